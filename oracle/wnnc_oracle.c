/*
 * wnnc_oracle.c -- plain FP64 CPU oracle for the WNNC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke() check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code
 * with the CUDA path (no headers, no helpers, no constants).
 *
 * What it computes (all in double precision, one OpenMP loop over targets
 * where the loop has no cross-target accumulation):
 *
 *  - or_normalize: the input normalisation of Sec. 5.1.1 (points scaled into
 *    [-1,1]^3 with a margin of 1/11).
 *  - or_direct: the plain O(N*M) sums of the three operators of Sec. 4.5,
 *      A(mu)_y   = sum_j gradPhi(y - x_j) . mu_j            (Eq. 5, Eq. 6)
 *      G(mu)_y   = -sum_j HPhi(y - x_j) mu_j               (Eq. 9, Eq. 10)
 *      AT(s)_y   = sum_i s_i gradPhi(x_i - y)              (Sec. 4.5, A^T)
 *    with gradPhi(y) = -y/(4 pi |y|^3) (Thm. 1) and
 *    HPhi(y) = -I/(4 pi |y|^3) + 3 y y^T/(4 pi |y|^5) (Eq. 9), every term set
 *    to zero when |y - x| < w (Sec. 4.4, operators A_w, G_w).
 *  - or_tree_*: the treecode approximation of Sec. 4.5 / Alg. 4: an octree
 *    over the sources that stops splitting at leaf_size points or depth D,
 *    node representatives (Eq. 13/14), and far / recurse / leaf-direct
 *    decisions.  Targets are evaluated in groups of consecutive Morton-sorted
 *    targets; a node is used as a far source for a whole group when the gap
 *    between the group's bounding box and the node's bounding box exceeds
 *    c * width(node), c = 1/theta.  Because both the target and the
 *    representative lie in those boxes, every far use also satisfies the
 *    per-target test of Alg. 4 (|x_i - x_B| > c * width(B)).
 *  - or_ptree_*: the paper's own treecode, Alg. 4 exactly as printed, with no
 *    design of this build in it: a plain geometric octree (cubes of
 *    [-1,1]^3 split into octants while a cube holds more than leaf_size
 *    points and is shallower than D; leaf_size 1 is the paper's), the
 *    nu-representatives of Eq. 13-14 recomputed for every call, and for
 *    every target separately a recursion from the root that takes node B
 *    as far iff |y - x_{B,nu}| > c * width(B).  A^T is the paper's
 *    s-representative treecode (nu = s).
 *  - or_iterate: Alg. 3 (width schedule, grad step of Alg. 2, WNNC update,
 *    rescale), on the direct sums, the group treecode or the paper's treecode.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

enum { OP_A = 0, OP_G = 1, OP_AT = 2 };

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Normalisation (Sec. 5.1.1): centre the bounding box, scale the largest    */
/* half-extent to 10/11.                                                     */
/* ------------------------------------------------------------------------ */
void or_normalize(const float* pts, int64_t n, double* xn, double* center, double* scale) {
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
        lo[k] = n > 0 ? (double)pts[k] : 0.0;
        hi[k] = lo[k];
    }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            double v = (double)pts[3 * i + k];
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    double hmax = 0.0;
    for (int k = 0; k < 3; ++k) {
        center[k] = (lo[k] + hi[k]) * 0.5;
        double h = (hi[k] - lo[k]) * 0.5;
        if (h > hmax) hmax = h;
    }
    double s = hmax > 0.0 ? (10.0 / 11.0) / hmax : 1.0;
    *scale = s;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k)
            xn[3 * i + k] = ((double)pts[3 * i + k] - center[k]) * s;
}

/* ------------------------------------------------------------------------ */
/* Pair terms.  d = y - x (target minus source).                              */
/* ------------------------------------------------------------------------ */

/* gradPhi(y - x) . mu  =  -(d . mu) / (4 pi r^3) */
static inline double term_A(const double d[3], double r2, const double* mu) {
    double r = sqrt(r2);
    return -(d[0] * mu[0] + d[1] * mu[1] + d[2] * mu[2]) / (4.0 * OR_PI * r2 * r);
}

/* -HPhi(d) mu = mu/(4 pi r^3) - 3 d (d.mu)/(4 pi r^5) */
static inline void term_G(const double d[3], double r2, const double* mu, double out[3]) {
    double r = sqrt(r2);
    double r3 = r2 * r, r5 = r3 * r2;
    double dm = d[0] * mu[0] + d[1] * mu[1] + d[2] * mu[2];
    for (int k = 0; k < 3; ++k)
        out[k] = mu[k] / (4.0 * OR_PI * r3) - 3.0 * d[k] * dm / (4.0 * OR_PI * r5);
}

/* s * gradPhi(x - y) = s * d / (4 pi r^3), d = y - x */
static inline void term_AT(const double d[3], double r2, double s, double out[3]) {
    double r = sqrt(r2);
    for (int k = 0; k < 3; ++k) out[k] = s * d[k] / (4.0 * OR_PI * r2 * r);
}

/* Cut-off of Sec. 4.4: a term counts iff |y - x| >= w.  Pairs closer than
 * MIN_SEP = 2^-20 (normalised units, about 1e-6 of the cloud) count as
 * coincident and never count either: this removes the self term, and it is the
 * only exclusion when w = 0 (Alg. 1), where the kernel is singular. */
#define MIN_SEP2 (1.0 / 1099511627776.0) /* (2^-20)^2 */
static inline double eff_w2(double w) { double w2 = w * w; return w2 > MIN_SEP2 ? w2 : MIN_SEP2; }
static inline int keep_pair(double r2, double w2) { return r2 >= w2; }

/* A pair is "cut-off ambiguous" when r^2 lies within amb_tol*w^2 of w^2: a
 * single-precision evaluation may take the other side of the test. */
static inline int ambiguous(double r2, double w2, double amb_tol) {
    return fabs(r2 - w2) <= amb_tol * w2;
}

/* ------------------------------------------------------------------------ */
/* Direct sums: targets y (nt x 3), sources x (ns x 3).                       */
/* nu: mu (ns x 3) for A and G, s (ns) for AT.                                */
/* out: nt for A, nt x 3 for G and AT.  amb (optional): per target, the sum   */
/* of |term| over cut-off-ambiguous pairs (the largest change a flipped       */
/* cut-off decision can make).                                               */
/* ------------------------------------------------------------------------ */
void or_direct(int op, const double* xs, int64_t ns, const double* nu,
               const double* yt, int64_t nt, double w, double amb_tol,
               double* out, double* amb, double* abssum) {
    const double w2 = eff_w2(w);
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        double acc[3] = {0, 0, 0}, ab = 0.0, as = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            double d[3] = {yt[3 * t] - xs[3 * j], yt[3 * t + 1] - xs[3 * j + 1],
                           yt[3 * t + 2] - xs[3 * j + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            int amb_p = amb && ambiguous(r2, w2, amb_tol);
            if (!keep_pair(r2, w2) && !amb_p) continue;
            double v[3] = {0, 0, 0};
            if (op == OP_A) v[0] = term_A(d, r2, nu + 3 * j);
            else if (op == OP_G) term_G(d, r2, nu + 3 * j, v);
            else term_AT(d, r2, nu[j], v);
            double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (amb_p) ab += vn;
            if (keep_pair(r2, w2)) {
                for (int k = 0; k < 3; ++k) acc[k] += v[k];
                as += vn;
            }
        }
        if (op == OP_A) out[t] = acc[0];
        else for (int k = 0; k < 3; ++k) out[3 * t + k] = acc[k];
        if (amb) amb[t] = ab;
        if (abssum) abssum[t] = as;
    }
}

/* ------------------------------------------------------------------------ */
/* Octree (Sec. 4.5): cells are the dyadic cubes of the root cube [-1,1]^3;  */
/* a cell at depth d has width 2/2^d.  A node is split into its non-empty    */
/* child cells while it holds more than leaf_size points and d < max_depth.  */
/* Points are ordered by a 45-bit Morton key (15 bits per axis, x the most   */
/* significant bit of each 3-bit digit), ties broken by input index.         */
/* ------------------------------------------------------------------------ */

static int64_t quant15(double v) {
    double q = floor((v + 1.0) * 16384.0);
    if (q < 0.0) q = 0.0;
    if (q > 32767.0) q = 32767.0;
    return (int64_t)q;
}

static uint64_t morton45(const double* x) {
    int64_t q[3] = {quant15(x[0]), quant15(x[1]), quant15(x[2])};
    uint64_t key = 0;
    for (int b = 14; b >= 0; --b) {
        uint64_t digit = (uint64_t)(((q[0] >> b) & 1) << 2 | ((q[1] >> b) & 1) << 1 | ((q[2] >> b) & 1));
        key = (key << 3) | digit;
    }
    return key;
}

typedef struct { uint64_t key; int64_t idx; } keyidx;

static int cmp_keyidx(const void* a, const void* b) {
    const keyidx* p = (const keyidx*)a;
    const keyidx* q = (const keyidx*)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

/* Sorted order of a point set: perm[k] = input index of the k-th point. */
static void morton_order(const double* x, int64_t n, int64_t* perm, uint64_t* keys) {
    keyidx* ki = (keyidx*)malloc(sizeof(keyidx) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { ki[i].key = morton45(x + 3 * i); ki[i].idx = i; }
    qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
    for (int64_t i = 0; i < n; ++i) { perm[i] = ki[i].idx; if (keys) keys[i] = ki[i].key; }
    free(ki);
}

typedef struct {
    int64_t n, nnodes, cap;
    int leaf_size, max_depth;
    double* x;          /* sources, normalised, sorted order (n x 3) */
    int64_t* perm;      /* sorted position -> input index */
    uint64_t* key;
    int64_t *start, *count, *parent, *child0;
    int *depth, *nchild;
    double *lo, *hi, *cent;   /* tight bounding box and point centroid per node */
} or_octree;

static int64_t new_node(or_octree* t) {
    if (t->nnodes == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->start = realloc(t->start, sizeof(int64_t) * t->cap);
        t->count = realloc(t->count, sizeof(int64_t) * t->cap);
        t->parent = realloc(t->parent, sizeof(int64_t) * t->cap);
        t->child0 = realloc(t->child0, sizeof(int64_t) * t->cap);
        t->depth = realloc(t->depth, sizeof(int) * t->cap);
        t->nchild = realloc(t->nchild, sizeof(int) * t->cap);
    }
    return t->nnodes++;
}

/* Breadth-first construction so that the children of a node are consecutive. */
static void build_octree(or_octree* t) {
    int64_t root = new_node(t);
    t->start[root] = 0; t->count[root] = t->n; t->parent[root] = -1;
    t->depth[root] = 0; t->nchild[root] = 0; t->child0[root] = -1;
    for (int64_t b = 0; b < t->nnodes; ++b) {
        if (t->count[b] <= t->leaf_size || t->depth[b] >= t->max_depth) continue;
        int d = t->depth[b];
        int shift = 3 * (14 - d);      /* digit of the child level d+1 */
        int64_t s = t->start[b], e = s + t->count[b];
        int64_t first = -1; int nc = 0;
        int64_t i = s;
        while (i < e) {
            uint64_t dig = (t->key[i] >> shift) & 7u;
            int64_t j = i;
            while (j < e && ((t->key[j] >> shift) & 7u) == dig) ++j;
            int64_t c = new_node(t);
            if (first < 0) first = c;
            t->start[c] = i; t->count[c] = j - i; t->parent[c] = b;
            t->depth[c] = d + 1; t->nchild[c] = 0; t->child0[c] = -1;
            ++nc;
            i = j;
        }
        t->child0[b] = first; t->nchild[b] = nc;
    }
    int64_t m = t->nnodes;
    t->lo = malloc(sizeof(double) * 3 * m);
    t->hi = malloc(sizeof(double) * 3 * m);
    t->cent = malloc(sizeof(double) * 3 * m);
    for (int64_t b = 0; b < m; ++b) {
        double sum[3] = {0, 0, 0};
        for (int k = 0; k < 3; ++k) { t->lo[3 * b + k] = INFINITY; t->hi[3 * b + k] = -INFINITY; }
        for (int64_t i = t->start[b]; i < t->start[b] + t->count[b]; ++i)
            for (int k = 0; k < 3; ++k) {
                double v = t->x[3 * i + k];
                if (v < t->lo[3 * b + k]) t->lo[3 * b + k] = v;
                if (v > t->hi[3 * b + k]) t->hi[3 * b + k] = v;
                sum[k] += v;
            }
        for (int k = 0; k < 3; ++k) t->cent[3 * b + k] = sum[k] / (double)t->count[b];
    }
}

/* Target groups: runs of at most group_size consecutive Morton-sorted
 * targets (group g = sorted targets goff[g] .. goff[g+1]-1), with their
 * interaction lists against the source octree. */
typedef struct {
    int64_t m, ngroups;
    int group_size;
    int64_t* goff;
    double* y;           /* targets, normalised, sorted (m x 3) */
    int64_t* perm;       /* sorted position -> input index */
    double *glo, *ghi;   /* group bounding boxes */
    int64_t *far_off, *far_id, *near_off, *near_id;   /* CSR lists per group */
    int64_t far_pairs, near_pairs;
} or_targets;

typedef struct { int64_t *v; int64_t n, cap; } ivec;
static void ivec_push(ivec* a, int64_t x) {
    if (a->n == a->cap) { a->cap = a->cap ? 2 * a->cap : 64; a->v = realloc(a->v, sizeof(int64_t) * a->cap); }
    a->v[a->n++] = x;
}

/* Far test for a target group box (glo, ghi) against node b: the gap between
 * the boxes, squared, must exceed (c * width(b))^2.  Evaluated as written, in
 * double precision, without fused multiply-adds. */
static double box_gap2(const or_octree* t, int64_t b, const double* glo, const double* ghi) {
    double g[3];
    for (int k = 0; k < 3; ++k) {
        double a = t->lo[3 * b + k] - ghi[k];
        double e = glo[k] - t->hi[3 * b + k];
        double m = a > e ? a : e;
        g[k] = m > 0.0 ? m : 0.0;
    }
    double gx = g[0] * g[0], gy = g[1] * g[1], gz = g[2] * g[2];
    return (gx + gy) + gz;
}

static int is_far(const or_octree* t, int64_t b, const double* glo, const double* ghi, double c) {
    if (!(c < INFINITY)) return 0;
    double d2 = box_gap2(t, b, glo, ghi);
    double width = ldexp(2.0, -t->depth[b]);
    double cw = c * width;
    return d2 > cw * cw;
}

/* Local-expansion test for a far node b of a group with box (glo, ghi): the
 * box gap, squared, must exceed (cL * e)^2, e the largest extent of the group
 * box (same evaluation rules as is_far).  cL = 0 switches local expansions off. */
static double group_extent(const double* glo, const double* ghi) {
    double e = ghi[0] - glo[0];
    if (ghi[1] - glo[1] > e) e = ghi[1] - glo[1];
    if (ghi[2] - glo[2] > e) e = ghi[2] - glo[2];
    return e;
}

static int is_local(const or_octree* t, int64_t b, const double* glo, const double* ghi, double cL) {
    if (!(cL > 0.0)) return 0;
    double ce = cL * group_extent(glo, ghi);
    return box_gap2(t, b, glo, ghi) > ce * ce;
}

static void traverse(const or_octree* t, int64_t b, const double* glo, const double* ghi, double c,
                     ivec* far, ivec* near) {
    if (is_far(t, b, glo, ghi, c)) { ivec_push(far, b); return; }
    if (t->nchild[b] == 0) { ivec_push(near, b); return; }
    for (int q = 0; q < t->nchild[b]; ++q) traverse(t, t->child0[b] + q, glo, ghi, c, far, near);
}

/* Number of leading 3-bit digits two 45-bit Morton keys share (0..15). */
static int common_digits(uint64_t a, uint64_t b) {
    int c = 0;
    for (int l = 14; l >= 0; --l) {
        if (((a >> (3 * l)) & 7u) != ((b >> (3 * l)) & 7u)) break;
        ++c;
    }
    return c;
}

/* Group boundaries.  Without a tree (slack < 0): fixed runs of group_size.
 * With the source tree (targets = sources, sorted alike): a new group also
 * starts before sorted point k when the leaves of points k-1 and k do not
 * share an ancestor within `slack` levels of the deeper leaf, i.e. when the
 * keys share fewer than max(depth(leaf(k-1)), depth(leaf(k))) - slack digits,
 * or fewer than min_depth digits (the two points lie in different cells of
 * depth min_depth).  A group then never straddles a jump of the Morton curve
 * between distant cells and stays inside one cell of depth min_depth, which
 * keeps its bounding box (and its interaction lists) compact. */
static int64_t group_offsets(const or_octree* t, const uint64_t* keys, int64_t m, int group_size,
                             int slack, int min_depth, int64_t* goff) {
    int* ldepth = NULL;
    if (slack >= 0) {
        ldepth = malloc(sizeof(int) * (m > 0 ? m : 1));
        for (int64_t b = 0; b < t->nnodes; ++b)
            if (t->nchild[b] == 0)
                for (int64_t i = t->start[b]; i < t->start[b] + t->count[b]; ++i) ldepth[i] = t->depth[b];
    }
    int64_t ng = 0, start = 0;
    for (int64_t k = 0; k < m; ++k) {
        int cut = (k == 0) || (k - start == group_size);
        if (!cut && slack >= 0) {
            int d = ldepth[k - 1] > ldepth[k] ? ldepth[k - 1] : ldepth[k];
            const int cd = common_digits(keys[k - 1], keys[k]);
            cut = cd < d - slack || cd < min_depth;
        }
        if (cut) {
            if (goff) goff[ng] = k;
            ++ng;
            start = k;
        }
    }
    if (goff) goff[ng] = m;
    free(ldepth);
    return ng;
}

static void build_targets(or_targets* T, const or_octree* t, const double* yn, int64_t m,
                          int group_size, double theta, int slack, int min_depth) {
    T->m = m; T->group_size = group_size;
    T->perm = malloc(sizeof(int64_t) * (m > 0 ? m : 1));
    uint64_t* keys = malloc(sizeof(uint64_t) * (m > 0 ? m : 1));
    morton_order(yn, m, T->perm, keys);
    T->y = malloc(sizeof(double) * 3 * (m > 0 ? m : 1));
    for (int64_t i = 0; i < m; ++i)
        for (int k = 0; k < 3; ++k) T->y[3 * i + k] = yn[3 * T->perm[i] + k];
    int64_t ng = group_offsets(t, keys, m, group_size, slack, min_depth, NULL);
    T->goff = malloc(sizeof(int64_t) * (ng + 1));
    group_offsets(t, keys, m, group_size, slack, min_depth, T->goff);
    free(keys);
    T->ngroups = ng;
    T->glo = malloc(sizeof(double) * 3 * (ng > 0 ? ng : 1));
    T->ghi = malloc(sizeof(double) * 3 * (ng > 0 ? ng : 1));
    double c = theta > 0.0 ? 1.0 / theta : INFINITY;
    ivec* fars = calloc((size_t)(ng > 0 ? ng : 1), sizeof(ivec));
    ivec* nears = calloc((size_t)(ng > 0 ? ng : 1), sizeof(ivec));
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t g = 0; g < ng; ++g) {
        int64_t s = T->goff[g], e = T->goff[g + 1];
        for (int k = 0; k < 3; ++k) { T->glo[3 * g + k] = INFINITY; T->ghi[3 * g + k] = -INFINITY; }
        for (int64_t i = s; i < e; ++i)
            for (int k = 0; k < 3; ++k) {
                double v = T->y[3 * i + k];
                if (v < T->glo[3 * g + k]) T->glo[3 * g + k] = v;
                if (v > T->ghi[3 * g + k]) T->ghi[3 * g + k] = v;
            }
        if (t->n > 0) traverse(t, 0, T->glo + 3 * g, T->ghi + 3 * g, c, &fars[g], &nears[g]);
    }
    T->far_off = malloc(sizeof(int64_t) * (ng + 1));
    T->near_off = malloc(sizeof(int64_t) * (ng + 1));
    T->far_off[0] = T->near_off[0] = 0;
    for (int64_t g = 0; g < ng; ++g) {
        T->far_off[g + 1] = T->far_off[g] + fars[g].n;
        T->near_off[g + 1] = T->near_off[g] + nears[g].n;
    }
    T->far_id = malloc(sizeof(int64_t) * (T->far_off[ng] > 0 ? T->far_off[ng] : 1));
    T->near_id = malloc(sizeof(int64_t) * (T->near_off[ng] > 0 ? T->near_off[ng] : 1));
    T->far_pairs = T->near_pairs = 0;
    for (int64_t g = 0; g < ng; ++g) {
        int64_t gs = T->goff[g], ge = T->goff[g + 1];
        memcpy(T->far_id + T->far_off[g], fars[g].v, sizeof(int64_t) * fars[g].n);
        memcpy(T->near_id + T->near_off[g], nears[g].v, sizeof(int64_t) * nears[g].n);
        T->far_pairs += (ge - gs) * fars[g].n;
        for (int64_t q = 0; q < nears[g].n; ++q) T->near_pairs += (ge - gs) * t->count[nears[g].v[q]];
        free(fars[g].v); free(nears[g].v);
    }
    free(fars); free(nears);
}

static void free_targets(or_targets* T) {
    free(T->y); free(T->perm); free(T->glo); free(T->ghi); free(T->goff);
    free(T->far_off); free(T->far_id); free(T->near_off); free(T->near_id);
}

/* The public tree handle: sources with their octree, and the sources
 * themselves as the on-surface target set. */
typedef struct {
    or_octree src;
    or_targets self;
    double theta;
    int far_order;      /* 0: monopole far terms (Eq. 13-14); 1: plus the first-order Taylor terms */
    double local_c;     /* > 0: first-order local expansions about the group box centre for far
                           nodes with box gap > local_c x group extent (far_order 0, rep_mode 1) */
    int local_cluster;  /* >= 2: also about the centres of clusters of that many groups */
    signed char* self_cls;   /* the class of every far entry of the points as targets */
} or_tree;

static signed char* local_classes(const or_octree* t, const or_targets* T, double c, int K);

/* group_slack, group_min_depth: the rule of group_offsets for the points as
 * targets (slack < 0: fixed runs of group_size). */
or_tree* or_tree_build(const double* xn, int64_t n, int leaf_size, int group_size, int max_depth,
                       double theta, int group_slack, int group_min_depth) {
    or_tree* T = calloc(1, sizeof(or_tree));
    or_octree* t = &T->src;
    t->n = n; t->leaf_size = leaf_size; t->max_depth = max_depth;
    t->perm = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    t->key = malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    morton_order(xn, n, t->perm, t->key);
    t->x = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) t->x[3 * i + k] = xn[3 * t->perm[i] + k];
    if (n > 0) build_octree(t);
    T->theta = theta;
    build_targets(&T->self, t, xn, n, group_size, theta, group_slack, group_min_depth);
    return T;
}

void or_tree_free(or_tree* T) {
    if (!T) return;
    or_octree* t = &T->src;
    free(t->x); free(t->perm); free(t->key); free(t->start); free(t->count); free(t->parent);
    free(t->child0); free(t->depth); free(t->nchild); free(t->lo); free(t->hi); free(t->cent);
    free_targets(&T->self);
    free(T->self_cls);
    free(T);
}

/* Order of the far-field expansion of the group treecode (rep_mode 1 only):
 * 0 = one term per far node at its point centroid x_B (Eq. 13-14);
 * 1 = plus the first-order Taylor term of the kernel about x_B. */
void or_tree_set_far_order(or_tree* T, int order) { T->far_order = order; }

/* Local expansions of the far field about the target group's box centre
 * (rep_mode 1, far_order 0): a far node b is expanded for a group when the box
 * gap exceeds 1/local_theta times the group box's largest extent; local_theta
 * 0 switches them off. */
/* The class of every far entry of the points as targets (in the order of
 * or_tree_lists): 0 summed pair by pair, 1 expanded about its group's centre,
 * 2 about its cluster's; all 0 without local expansions. */
void or_tree_local_classes(const or_tree* T, signed char* out) {
    const int64_t nf = T->self.far_off[T->self.ngroups];
    for (int64_t q = 0; q < nf; ++q) out[q] = T->self_cls ? T->self_cls[q] : 0;
}

void or_tree_set_local(or_tree* T, double local_theta, int cluster) {
    T->local_c = local_theta > 0.0 ? 1.0 / local_theta : 0.0;
    T->local_cluster = cluster;
    free(T->self_cls);
    T->self_cls = T->local_c > 0.0 ? local_classes(&T->src, &T->self, T->local_c, cluster) : NULL;
}

/* Structure queries (for the structural pins and for comparing list sizes). */
int64_t or_tree_nnodes(const or_tree* T) { return T->src.nnodes; }
void or_tree_nodes(const or_tree* T, int64_t* start, int64_t* count, int* depth, int* nchild,
                   int64_t* parent) {
    const or_octree* t = &T->src;
    for (int64_t b = 0; b < t->nnodes; ++b) {
        start[b] = t->start[b]; count[b] = t->count[b]; depth[b] = t->depth[b];
        nchild[b] = t->nchild[b]; parent[b] = t->parent[b];
    }
}
void or_tree_perm(const or_tree* T, int64_t* perm) { memcpy(perm, T->src.perm, sizeof(int64_t) * T->src.n); }
void or_tree_boxes(const or_tree* T, double* lo, double* hi, double* cent) {
    const or_octree* t = &T->src;
    memcpy(lo, t->lo, sizeof(double) * 3 * t->nnodes);
    memcpy(hi, t->hi, sizeof(double) * 3 * t->nnodes);
    memcpy(cent, t->cent, sizeof(double) * 3 * t->nnodes);
}
/* far / near list sizes and pair counts of the on-surface target set */
void or_tree_counts(const or_tree* T, int64_t* out4) {
    out4[0] = T->self.far_off[T->self.ngroups];
    out4[1] = T->self.near_off[T->self.ngroups];
    out4[2] = T->self.far_pairs;
    out4[3] = T->self.near_pairs;
}
int64_t or_tree_ngroups(const or_tree* T) { return T->self.ngroups; }
void or_tree_groups(const or_tree* T, int64_t* goff) {
    memcpy(goff, T->self.goff, sizeof(int64_t) * (T->self.ngroups + 1));
}
void or_tree_lists(const or_tree* T, int64_t* far_off, int64_t* far_id, int64_t* near_off, int64_t* near_id) {
    const or_targets* S = &T->self;
    memcpy(far_off, S->far_off, sizeof(int64_t) * (S->ngroups + 1));
    memcpy(near_off, S->near_off, sizeof(int64_t) * (S->ngroups + 1));
    memcpy(far_id, S->far_id, sizeof(int64_t) * S->far_off[S->ngroups]);
    memcpy(near_id, S->near_id, sizeof(int64_t) * S->near_off[S->ngroups]);
}

/* ------------------------------------------------------------------------ */
/* Node representatives (Eq. 13, Eq. 14).                                    */
/*  rep_mode 0 (as in the paper): x_B = sum |nu_i| x_i / sum |nu_j|          */
/*  rep_mode 1: x_B = plain centroid of the node's points (independent of    */
/*              nu, which makes the tree operator linear in nu).             */
/*  If sum |nu_j| = 0 the plain centroid is used (nu_B = 0 then anyway).     */
/*  nu_B = sum nu_i.  nu has dim 3 (mu) or 1 (s); nu is in sorted order.     */
/* ------------------------------------------------------------------------ */
static void node_reps(const or_octree* t, const double* nu, int dim, int rep_mode,
                      double* rep, double* nuB) {
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t b = 0; b < t->nnodes; ++b) {
        double sw = 0.0, sx[3] = {0, 0, 0}, sn[3] = {0, 0, 0};
        for (int64_t i = t->start[b]; i < t->start[b] + t->count[b]; ++i) {
            double a = 0.0;
            for (int k = 0; k < dim; ++k) { sn[k] += nu[dim * i + k]; a += nu[dim * i + k] * nu[dim * i + k]; }
            a = sqrt(a);
            sw += a;
            for (int k = 0; k < 3; ++k) sx[k] += a * t->x[3 * i + k];
        }
        for (int k = 0; k < 3; ++k)
            rep[3 * b + k] = (rep_mode == 0 && sw > 0.0) ? sx[k] / sw : t->cent[3 * b + k];
        for (int k = 0; k < dim; ++k) nuB[dim * b + k] = sn[k];
    }
}

/* ------------------------------------------------------------------------ */
/* First-order far field (rep_mode 1, about the point centroid x_B).  With   */
/* d = y - x_B and a source x_j = x_B + delta_j, Taylor's theorem gives       */
/*   gradPhi(d - delta) = gradPhi(d) - HPhi(d) delta + O(|delta|^2)           */
/*   HPhi(d - delta)    = HPhi(d) - T(d)[delta] + O(|delta|^2),               */
/* T_abc = d_c HPhi_ab = (3 (I_ab d_c + I_ac d_b + I_bc d_a)/r^5              */
/*                        - 15 d_a d_b d_c / r^7) / (4 pi),                   */
/* and summed over the node's sources the first-order terms need only the     */
/* symmetric moment S = sum_j sym(delta_j mu_j^T) (HPhi and T are symmetric): */
/*   A: - HPhi(d) : S = tr S/(4 pi r^3) - 3 d.S d/(4 pi r^5)                  */
/*   G: + T(d) : S    = (6 S d + 3 tr S d)/(4 pi r^5) - 15 (d.S d) d/(4 pi r^7) */
/* S is stored as (Sxx, Syy, Szz, Sxy, Sxz, Syz).                             */
/* ------------------------------------------------------------------------ */
static void node_dipoles(const or_octree* t, const double* nu, double* S) {
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t b = 0; b < t->nnodes; ++b) {
        double m[6] = {0, 0, 0, 0, 0, 0};
        const double* c = t->cent + 3 * b;
        for (int64_t i = t->start[b]; i < t->start[b] + t->count[b]; ++i) {
            const double dl[3] = {t->x[3 * i] - c[0], t->x[3 * i + 1] - c[1], t->x[3 * i + 2] - c[2]};
            const double* v = nu + 3 * i;
            m[0] += dl[0] * v[0];
            m[1] += dl[1] * v[1];
            m[2] += dl[2] * v[2];
            m[3] += 0.5 * (dl[0] * v[1] + dl[1] * v[0]);
            m[4] += 0.5 * (dl[0] * v[2] + dl[2] * v[0]);
            m[5] += 0.5 * (dl[1] * v[2] + dl[2] * v[1]);
        }
        for (int k = 0; k < 6; ++k) S[6 * b + k] = m[k];
    }
}

static inline void sym_mul(const double* S, const double d[3], double out[3]) {
    out[0] = S[0] * d[0] + S[3] * d[1] + S[4] * d[2];
    out[1] = S[3] * d[0] + S[1] * d[1] + S[5] * d[2];
    out[2] = S[4] * d[0] + S[5] * d[1] + S[2] * d[2];
}

/* First-order correction of a far term (op A: out[0]; op G: out[0..2]). */
static void far_correction(int op, const double d[3], double r2, const double* S, double out[3]) {
    const double r = sqrt(r2), r3 = r2 * r, r5 = r3 * r2, r7 = r5 * r2;
    const double tr = S[0] + S[1] + S[2];
    double Sd[3];
    sym_mul(S, d, Sd);
    const double dSd = d[0] * Sd[0] + d[1] * Sd[1] + d[2] * Sd[2];
    if (op == OP_A) {
        out[0] = tr / (4.0 * OR_PI * r3) - 3.0 * dSd / (4.0 * OR_PI * r5);
        out[1] = out[2] = 0.0;
    } else {
        for (int k = 0; k < 3; ++k)
            out[k] = (6.0 * Sd[k] + 3.0 * tr * d[k]) / (4.0 * OR_PI * r5) - 15.0 * dSd * d[k] / (4.0 * OR_PI * r7);
    }
}

/* ------------------------------------------------------------------------ */
/* Local (target-side) expansion of the far field, the counterpart on the     */
/* target side of the expansions named in Sec. 4.5 and Sec. 6.3 (rep_mode 1,  */
/* far_order 0).  For a far node B of group g with D = c_g - x_B (c_g the     */
/* centre of the group box) and a target y = c_g + delta, Taylor's theorem    */
/* about c_g gives, with a(d) = gradPhi(d) . mu_B and g(d) = -HPhi(d) mu_B    */
/* (the far terms of A and G, G = -grad A):                                   */
/*   a(D + delta) = a(D) - delta . g(D) + O(|delta|^2)                        */
/*   g(D + delta) = g(D) - J(D) delta   + O(|delta|^2),                       */
/* J_ac = sum_b d_c HPhi_ab(D) mu_b                                           */
/*      = (3 (mu D^T + D mu^T)_ac + 3 (D.mu) I_ac)/(4 pi r^5)                */
/*        - 15 (D.mu) D_a D_c/(4 pi r^7),                                     */
/* symmetric, stored as (xx, yy, zz, xy, xz, yz).  A group sums a, g and J    */
/* over its local entries once and evaluates the two polynomials per target.  */
/* The transpose (the adjoint A^T) gives node B, per local entry,             */
/*   S_g gradPhi(D) + HPhi(D) D_g,  S_g = sum_i s_i, D_g = sum_i s_i delta_i. */
/* An entry is expanded only when every one of its pairs clears the cut-off:  */
/* with rho_g the largest distance of the group's targets from c_g, every     */
/* pair distance is at least |D| - rho_g, so the test is |D| - rho_g >= w;    */
/* otherwise the entry is summed pair by pair like the other far entries.    */
/* ------------------------------------------------------------------------ */
static void local_coeffs(const double D[3], const double* mu, double out[10]) {
    const double r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    const double r = sqrt(r2), r5 = r2 * r2 * r, r7 = r5 * r2;
    out[0] = term_A(D, r2, mu);
    term_G(D, r2, mu, out + 1);
    const double dm = D[0] * mu[0] + D[1] * mu[1] + D[2] * mu[2];
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ic[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q) {
        const int a = ia[q], c = ic[q];
        const double diag = a == c ? 3.0 * dm : 0.0;
        out[4 + q] = (3.0 * (mu[a] * D[c] + D[a] * mu[c]) + diag) / (4.0 * OR_PI * r5)
                   - 15.0 * dm * D[a] * D[c] / (4.0 * OR_PI * r7);
    }
}

/* The transposed local term of one entry: S gradPhi(D) + HPhi(D) Dg. */
static void local_adjoint(const double D[3], double S, const double Dg[3], double out[3]) {
    const double r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    const double r = sqrt(r2), r3 = r2 * r, r5 = r3 * r2;
    const double dd = D[0] * Dg[0] + D[1] * Dg[1] + D[2] * Dg[2];
    for (int k = 0; k < 3; ++k)
        out[k] = -S * D[k] / (4.0 * OR_PI * r3) + (3.0 * D[k] * dd - r2 * Dg[k]) / (4.0 * OR_PI * r5);
}

/* Per group: the expansion centre c_g (the centre of the group box) and rho_g. */
typedef struct { double c[3], rho; } local_frame;

static local_frame group_frame(const or_targets* T, int64_t g) {
    local_frame L;
    const double* glo = T->glo + 3 * g;
    const double* ghi = T->ghi + 3 * g;
    for (int k = 0; k < 3; ++k) L.c[k] = 0.5 * (glo[k] + ghi[k]);
    L.rho = 0.0;
    for (int64_t i = T->goff[g]; i < T->goff[g + 1]; ++i) {
        const double* y = T->y + 3 * i;
        const double dl[3] = {y[0] - L.c[0], y[1] - L.c[1], y[2] - L.c[2]};
        const double r = sqrt(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]);
        if (r > L.rho) L.rho = r;
    }
    return L;
}

/* Whether a local entry with D = c_g - x_B is expanded at the effective
 * squared width w2 (*amb: the decision lies within amb_tol of its threshold). */
static int local_use(const double D[3], double rho, double w2, double amb_tol, int* amb) {
    const double m = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]) - rho;
    const double m2 = m > 0.0 ? m * m : 0.0;
    *amb = amb_tol > 0.0 && m > 0.0 && fabs(m2 - w2) <= amb_tol * w2;
    return m > 0.0 && m2 >= w2;
}

/* The expanded term of one entry at the target offset dl from c_g
 * (op A: out[0]; op G: out[0..2]) and a bound of its size. */
static double local_eval(int op, const double* ce, const double dl[3], double out[3]) {
    const double dn = sqrt(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]);
    if (op == OP_A) {
        out[0] = ce[0] - (dl[0] * ce[1] + dl[1] * ce[2] + dl[2] * ce[3]);
        out[1] = out[2] = 0.0;
        return fabs(ce[0]) + dn * sqrt(ce[1] * ce[1] + ce[2] * ce[2] + ce[3] * ce[3]);
    }
    double jd[3];
    sym_mul(ce + 4, dl, jd);
    for (int k = 0; k < 3; ++k) out[k] = ce[1 + k] - jd[k];
    return sqrt(ce[1] * ce[1] + ce[2] * ce[2] + ce[3] * ce[3])
         + dn * sqrt(ce[4] * ce[4] + ce[5] * ce[5] + ce[6] * ce[6]
                     + 2.0 * (ce[7] * ce[7] + ce[8] * ce[8] + ce[9] * ce[9]));
}

/* Clusters of K consecutive target groups (K >= 2; cluster C = groups
 * C K .. C K + K - 1, the last one possibly shorter).  A far node that lies in
 * the expanded part of every member group's list, and is itself local for the
 * cluster's box (the union of the members' boxes; the same test as for a
 * group), is expanded once about the cluster's centre c_C instead of once per
 * member: each member's target at c_C + d gets a(D_C) - d.g(D_C) and
 * g(D_C) + J(D_C) d, D_C = c_C - x_B, when |D_C| - rho_C >= w (rho_C the
 * largest distance of the cluster's targets from c_C); otherwise the entry is
 * summed pair by pair.  The transpose takes the cluster's sums of s and of
 * s (x_i - c_C), once per (node, cluster). */
static int64_t cluster_end(const or_targets* T, int64_t C, int K) {
    int64_t e = (C + 1) * K;
    return e < T->ngroups ? e : T->ngroups;
}

static void cluster_box(const or_targets* T, int64_t C, int K, double lo[3], double hi[3]) {
    for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t g = C * K; g < cluster_end(T, C, K); ++g)
        for (int k = 0; k < 3; ++k) {
            if (T->glo[3 * g + k] < lo[k]) lo[k] = T->glo[3 * g + k];
            if (T->ghi[3 * g + k] > hi[k]) hi[k] = T->ghi[3 * g + k];
        }
}

static local_frame cluster_frame(const or_targets* T, int64_t C, int K) {
    local_frame L;
    double lo[3], hi[3];
    cluster_box(T, C, K, lo, hi);
    for (int k = 0; k < 3; ++k) L.c[k] = 0.5 * (lo[k] + hi[k]);
    L.rho = 0.0;
    for (int64_t i = T->goff[C * K]; i < T->goff[cluster_end(T, C, K)]; ++i) {
        const double* y = T->y + 3 * i;
        const double dl[3] = {y[0] - L.c[0], y[1] - L.c[1], y[2] - L.c[2]};
        const double r = sqrt(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]);
        if (r > L.rho) L.rho = r;
    }
    return L;
}

/* The local expansions of one target set: c = 1/local_theta, the cluster size
 * K (0 or 1: groups only) and per far entry its class: 0 summed pair by pair,
 * 1 expanded about its group's centre, 2 about its cluster's centre. */
typedef struct { double c; int K; signed char* cls; } local_cfg;

typedef struct { int64_t b, q; } node_entry;
static int cmp_node_entry(const void* a, const void* b) {
    const int64_t x = ((const node_entry*)a)->b, y = ((const node_entry*)b)->b;
    return (x > y) - (x < y);
}

static signed char* local_classes(const or_octree* t, const or_targets* T, double c, int K) {
    const int64_t ng = T->ngroups, nf = T->far_off[ng];
    signed char* cls = calloc((size_t)(nf > 0 ? nf : 1), 1);
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < ng; ++g)
        for (int64_t q = T->far_off[g]; q < T->far_off[g + 1]; ++q)
            cls[q] = (signed char)is_local(t, T->far_id[q], T->glo + 3 * g, T->ghi + 3 * g, c);
    if (K < 2) return cls;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t C = 0; C < (ng + K - 1) / K; ++C) {
        const int64_t g0 = C * K, g1 = cluster_end(T, C, K), nm = g1 - g0;
        if (nm < 2) continue;
        double lo[3], hi[3];
        cluster_box(T, C, K, lo, hi);
        /* each member's expanded entries, sorted by node */
        node_entry** ent = malloc(sizeof(node_entry*) * nm);
        int64_t* cnt = calloc((size_t)nm, sizeof(int64_t));
        for (int64_t m = 0; m < nm; ++m) {
            const int64_t g = g0 + m;
            ent[m] = malloc(sizeof(node_entry) * (T->far_off[g + 1] - T->far_off[g] + 1));
            for (int64_t q = T->far_off[g]; q < T->far_off[g + 1]; ++q)
                if (cls[q] == 1) ent[m][cnt[m]++] = (node_entry){T->far_id[q], q};
            qsort(ent[m], (size_t)cnt[m], sizeof(node_entry), cmp_node_entry);
        }
        int64_t* qm = malloc(sizeof(int64_t) * nm);
        for (int64_t k = 0; k < cnt[0]; ++k) {
            const int64_t b = ent[0][k].b;
            if (!is_local(t, b, lo, hi, c)) continue;
            int all = 1;
            qm[0] = ent[0][k].q;
            for (int64_t m = 1; m < nm && all; ++m) {
                node_entry key = {b, 0};
                node_entry* f = bsearch(&key, ent[m], (size_t)cnt[m], sizeof(node_entry), cmp_node_entry);
                if (!f) all = 0;
                else qm[m] = f->q;
            }
            if (all)
                for (int64_t m = 0; m < nm; ++m) cls[qm[m]] = 2;
        }
        for (int64_t m = 0; m < nm; ++m) free(ent[m]);
        free(ent); free(cnt); free(qm);
    }
    return cls;
}

/* Gather-form treecode for targets T against the source octree:
 *   op A : out (m)    = sum_far gradPhi(y - x_B) . mu_B + sum_near gradPhi(y - x_j) . mu_j
 *   op G : out (m x 3) = sum_far -HPhi(y - x_B) mu_B  + sum_near -HPhi(y - x_j) mu_j
 *   op AT (rep_mode 0 only, the s-representative treecode of Sec. 4.5):
 *          out (m x 3) = sum_far s_B gradPhi(x_B - y) + sum_near s_i gradPhi(x_i - y)
 * nu_sorted: source attribute in sorted source order.  out: sorted target order.
 */
static void tree_gather(const or_octree* t, const or_targets* T, int op, int rep_mode, double w,
                        const double* nu_sorted, double* out_sorted, double amb_tol, double* amb_sorted,
                        double* abs_sorted, int far_order, const local_cfg* LC) {
    int dim = (op == OP_AT) ? 1 : 3;
    double* rep = malloc(sizeof(double) * 3 * (t->nnodes > 0 ? t->nnodes : 1));
    double* nuB = malloc(sizeof(double) * dim * (t->nnodes > 0 ? t->nnodes : 1));
    node_reps(t, nu_sorted, dim, rep_mode, rep, nuB);
    const int dip = far_order == 1 && rep_mode == 1 && op != OP_AT;
    double* S = dip ? malloc(sizeof(double) * 6 * (t->nnodes > 0 ? t->nnodes : 1)) : NULL;
    if (dip) node_dipoles(t, nu_sorted, S);
    const double w2 = eff_w2(w);
    const int loc = LC && LC->c > 0.0 && rep_mode == 1 && !dip && op != OP_AT;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t g = 0; g < T->ngroups; ++g) {
        int64_t s = T->goff[g], e = T->goff[g + 1];
        local_frame L[3] = {{{0, 0, 0}, 0.0}, {{0, 0, 0}, 0.0}, {{0, 0, 0}, 0.0}};   /* by class */
        if (loc) L[1] = group_frame(T, g);
        if (loc && LC->K >= 2) L[2] = cluster_frame(T, g / LC->K, LC->K);
        for (int64_t i = s; i < e; ++i) {
            const double* y = T->y + 3 * i;
            double acc[3] = {0, 0, 0}, ab = 0.0, as = 0.0;
            for (int64_t q = T->far_off[g]; q < T->far_off[g + 1]; ++q) {
                int64_t b = T->far_id[q];
                /* an expanded entry: its term expanded about the centre of its group
                 * (class 1) or cluster (class 2) when all its pairs clear the cut-off */
                int use = 0, lamb = 0;
                double ev[3] = {0, 0, 0}, evabs = 0.0;
                const int cl = loc ? LC->cls[q] : 0;
                if (cl) {
                    const local_frame* F = &L[cl];
                    const double D[3] = {F->c[0] - rep[3 * b], F->c[1] - rep[3 * b + 1], F->c[2] - rep[3 * b + 2]};
                    use = local_use(D, F->rho, w2, amb_sorted ? amb_tol : 0.0, &lamb);
                    if (use || lamb) {
                        double ce[10];
                        local_coeffs(D, nuB + 3 * b, ce);
                        const double dl[3] = {y[0] - F->c[0], y[1] - F->c[1], y[2] - F->c[2]};
                        evabs = local_eval(op, ce, dl, ev);
                    }
                }
                if (use && !lamb) {
                    for (int k = 0; k < 3; ++k) acc[k] += ev[k];
                    as += evabs;
                    continue;
                }
                double d[3] = {y[0] - rep[3 * b], y[1] - rep[3 * b + 1], y[2] - rep[3 * b + 2]};
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                int amb_p = amb_sorted && ambiguous(r2, w2, amb_tol);
                if (!keep_pair(r2, w2) && !amb_p && !lamb) continue;
                double v[3] = {0, 0, 0};
                if (op == OP_A) v[0] = term_A(d, r2, nuB + 3 * b);
                else if (op == OP_G) term_G(d, r2, nuB + 3 * b, v);
                else term_AT(d, r2, nuB[b], v);
                double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                if (dip) {
                    double cr[3];
                    far_correction(op, d, r2, S + 6 * b, cr);
                    for (int k = 0; k < 3; ++k) v[k] += cr[k];
                    vn += sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
                }
                if (lamb) {
                    /* either side of the decision may be taken: bound their difference */
                    const double kp = keep_pair(r2, w2) ? 1.0 : 0.0;
                    ab += sqrt((ev[0] - kp * v[0]) * (ev[0] - kp * v[0]) + (ev[1] - kp * v[1]) * (ev[1] - kp * v[1])
                               + (ev[2] - kp * v[2]) * (ev[2] - kp * v[2]));
                    if (use) {
                        for (int k = 0; k < 3; ++k) acc[k] += ev[k];
                        as += evabs;
                        continue;
                    }
                }
                if (amb_p) ab += vn;
                if (keep_pair(r2, w2)) {
                    for (int k = 0; k < 3; ++k) acc[k] += v[k];
                    as += vn;
                }
            }
            for (int64_t q = T->near_off[g]; q < T->near_off[g + 1]; ++q) {
                int64_t b = T->near_id[q];
                for (int64_t j = t->start[b]; j < t->start[b] + t->count[b]; ++j) {
                    const double* x = t->x + 3 * j;
                    double d[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    int amb_p = amb_sorted && ambiguous(r2, w2, amb_tol);
                    if (!keep_pair(r2, w2) && !amb_p) continue;
                    double v[3] = {0, 0, 0};
                    if (op == OP_A) v[0] = term_A(d, r2, nu_sorted + 3 * j);
                    else if (op == OP_G) term_G(d, r2, nu_sorted + 3 * j, v);
                    else term_AT(d, r2, nu_sorted[j], v);
                    double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                    if (amb_p) ab += vn;
                    if (keep_pair(r2, w2)) {
                        for (int k = 0; k < 3; ++k) acc[k] += v[k];
                        as += vn;
                    }
                }
            }
            if (op == OP_A) out_sorted[i] = acc[0];
            else for (int k = 0; k < 3; ++k) out_sorted[3 * i + k] = acc[k];
            if (amb_sorted) amb_sorted[i] = ab;
            if (abs_sorted) abs_sorted[i] = as;
        }
    }
    free(rep); free(nuB); free(S);
}

/* Exact transpose of the rep_mode-1 tree operator A (targets = sources):
 *   A_tree(mu)_i = sum_{B far for g(i)} gradPhi(x_i - x_B) . sum_{j in B} mu_j
 *                + sum_{L near for g(i)} sum_{j in L} gradPhi(x_i - x_j) . mu_j
 * so
 *   (A_tree^T s)_j = sum_{B containing j} V_B
 *                  + sum_{(g, L): L near for g, j in L} sum_{i in g} s_i gradPhi(x_i - x_j),
 *   V_B = sum_{g: B far for g} sum_{i in g} s_i gradPhi(x_i - x_B).
 * The node sums and the leaf sums are gathered through the transposed lists so
 * that each output is a sum in a fixed order (groups ascending, then i). */
/* With far_order 1 the tree operator A carries the first-order terms
 *   A_tree(mu)_i += - sum_{B far for g(i)} sum_{j in B} (HPhi(x_i - x_B) delta_jB) . mu_j,
 * delta_jB = x_j - x_B, whose transpose adds to every point j
 *   - sum_{B containing j} H_B delta_jB,   H_B = sum_{g: B far} sum_{i in g} s_i HPhi(x_i - x_B),
 * with the same cut-off decision as the node's monopole term. */
static void tree_adjoint_exact(const or_octree* t, const or_targets* T, double w,
                               const double* s_sorted, double* out_sorted, double amb_tol,
                               double* amb_sorted, double* abs_sorted, int far_order, const local_cfg* LC) {
    int64_t nn = t->nnodes, ng = T->ngroups;
    const double w2 = eff_w2(w);
    /* local expansions: per group (and per cluster) its centre, rho, S = sum s_i,
     * D = sum s_i (x_i - c) and the bounds of their terms */
    const int loc = LC && LC->c > 0.0 && far_order == 0;
    const int K = loc && LC->K >= 2 ? LC->K : 0;
    const int64_t ncl = K ? (ng + K - 1) / K : 0;
    local_frame* LS = calloc((size_t)(ng > 0 ? ng : 1), sizeof(local_frame));
    double* SD = calloc((size_t)(ng > 0 ? ng : 1) * 6, sizeof(double));   /* S, D[3], sum|s|, sum|s||delta| */
    local_frame* LSC = calloc((size_t)(ncl > 0 ? ncl : 1), sizeof(local_frame));
    double* SDC = calloc((size_t)(ncl > 0 ? ncl : 1) * 6, sizeof(double));
    if (loc) {
        #pragma omp parallel for schedule(dynamic, 16)
        for (int64_t u = 0; u < ng + ncl; ++u) {
            const int is_cl = u >= ng;
            const int64_t id = is_cl ? u - ng : u;
            const local_frame F = is_cl ? cluster_frame(T, id, K) : group_frame(T, id);
            double* sd = is_cl ? SDC + 6 * id : SD + 6 * id;
            const int64_t i0 = is_cl ? T->goff[id * K] : T->goff[id];
            const int64_t i1 = is_cl ? T->goff[cluster_end(T, id, K)] : T->goff[id + 1];
            for (int64_t i = i0; i < i1; ++i) {
                const double dl[3] = {T->y[3 * i] - F.c[0], T->y[3 * i + 1] - F.c[1], T->y[3 * i + 2] - F.c[2]};
                const double si = s_sorted[i];
                sd[0] += si;
                for (int k = 0; k < 3; ++k) sd[1 + k] += si * dl[k];
                sd[4] += fabs(si);
                sd[5] += fabs(si) * sqrt(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]);
            }
            if (is_cl) LSC[id] = F;
            else LS[id] = F;
        }
    }
    /* transposed lists: node -> groups using it (far), leaf -> groups using it (near) */
    int64_t* fcnt = calloc((size_t)nn + 1, sizeof(int64_t));
    int64_t* ncnt = calloc((size_t)nn + 1, sizeof(int64_t));
    for (int64_t q = 0; q < T->far_off[ng]; ++q) fcnt[T->far_id[q] + 1]++;
    for (int64_t q = 0; q < T->near_off[ng]; ++q) ncnt[T->near_id[q] + 1]++;
    for (int64_t b = 0; b < nn; ++b) { fcnt[b + 1] += fcnt[b]; ncnt[b + 1] += ncnt[b]; }
    int64_t* fg = malloc(sizeof(int64_t) * (fcnt[nn] > 0 ? fcnt[nn] : 1));
    int64_t* fq = malloc(sizeof(int64_t) * (fcnt[nn] > 0 ? fcnt[nn] : 1));   /* the far entry */
    int64_t* ngp = malloc(sizeof(int64_t) * (ncnt[nn] > 0 ? ncnt[nn] : 1));
    int64_t* fpos = malloc(sizeof(int64_t) * (nn > 0 ? nn : 1));
    int64_t* npos = malloc(sizeof(int64_t) * (nn > 0 ? nn : 1));
    memcpy(fpos, fcnt, sizeof(int64_t) * nn);
    memcpy(npos, ncnt, sizeof(int64_t) * nn);
    for (int64_t g = 0; g < ng; ++g) {
        for (int64_t q = T->far_off[g]; q < T->far_off[g + 1]; ++q) {
            fq[fpos[T->far_id[q]]] = q;
            fg[fpos[T->far_id[q]]++] = g;
        }
        for (int64_t q = T->near_off[g]; q < T->near_off[g + 1]; ++q) ngp[npos[T->near_id[q]]++] = g;
    }
    double* V = calloc((size_t)(nn > 0 ? nn : 1) * 3, sizeof(double));
    double* VA = calloc((size_t)(nn > 0 ? nn : 1), sizeof(double));
    double* VS = calloc((size_t)(nn > 0 ? nn : 1), sizeof(double));
    double* H = calloc((size_t)(nn > 0 ? nn : 1) * 6, sizeof(double));   /* (xx, yy, zz, xy, xz, yz) */
    double* HN = calloc((size_t)(nn > 0 ? nn : 1), sizeof(double));      /* sum of |s_i| |HPhi|_F */
    const double* rep = t->cent;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nn; ++b) {
        double acc[3] = {0, 0, 0}, ab = 0.0, as = 0.0, h[6] = {0, 0, 0, 0, 0, 0}, hn = 0.0;
        for (int64_t q = fcnt[b]; q < fcnt[b + 1]; ++q) {
            int64_t g = fg[q];
            const int cl = loc ? LC->cls[fq[q]] : 0;
            if (cl == 2 && g % K != 0) continue;     /* a cluster's entry: carried by its first member */
            /* the targets behind the entry: the group's, or for class 2 the cluster's */
            int64_t s = T->goff[g], e = cl == 2 ? T->goff[cluster_end(T, g / K, K)] : T->goff[g + 1];
            /* an expanded entry: the transposed expansion when all its pairs clear the cut-off */
            int use = 0, lamb = 0;
            double lv[3] = {0, 0, 0}, pw[3] = {0, 0, 0};
            if (cl) {
                const local_frame* F = cl == 2 ? &LSC[g / K] : &LS[g];
                const double D[3] = {F->c[0] - rep[3 * b], F->c[1] - rep[3 * b + 1], F->c[2] - rep[3 * b + 2]};
                use = local_use(D, F->rho, w2, amb_sorted ? amb_tol : 0.0, &lamb);
                const double* sd = cl == 2 ? SDC + 6 * (g / K) : SD + 6 * g;
                local_adjoint(D, sd[0], sd + 1, lv);
                if (use) {
                    const double r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
                    for (int k = 0; k < 3; ++k) acc[k] += lv[k];
                    as += sd[4] / (4.0 * OR_PI * r2) + 2.0 * sd[5] / (4.0 * OR_PI * r2 * sqrt(r2));
                    if (!lamb) continue;
                }
            }
            for (int64_t i = s; i < e; ++i) {
                /* s_i gradPhi(x_i - x_B) = s_i (x_B - x_i) / (4 pi r^3) */
                double d[3] = {rep[3 * b] - T->y[3 * i], rep[3 * b + 1] - T->y[3 * i + 1],
                               rep[3 * b + 2] - T->y[3 * i + 2]};
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                int amb_p = amb_sorted && ambiguous(r2, w2, amb_tol);
                if (!keep_pair(r2, w2) && !amb_p) continue;
                double v[3];
                term_AT(d, r2, s_sorted[i], v);
                double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                if (lamb) {
                    if (keep_pair(r2, w2)) for (int k = 0; k < 3; ++k) pw[k] += v[k];
                    if (use) continue;
                }
                if (amb_p) ab += vn;
                if (keep_pair(r2, w2)) {
                    for (int k = 0; k < 3; ++k) acc[k] += v[k];
                    as += vn;
                    if (far_order == 1) {
                        /* s_i HPhi(d), HPhi(d) = (3 d d^T - r^2 I)/(4 pi r^5), even in d */
                        const double r = sqrt(r2), f = s_sorted[i] / (4.0 * OR_PI * r2 * r2 * r);
                        h[0] += f * (3.0 * d[0] * d[0] - r2);
                        h[1] += f * (3.0 * d[1] * d[1] - r2);
                        h[2] += f * (3.0 * d[2] * d[2] - r2);
                        h[3] += f * 3.0 * d[0] * d[1];
                        h[4] += f * 3.0 * d[0] * d[2];
                        h[5] += f * 3.0 * d[1] * d[2];
                        hn += fabs(f) * sqrt(6.0) * r2;
                    }
                }
            }
            if (lamb)
                ab += sqrt((lv[0] - pw[0]) * (lv[0] - pw[0]) + (lv[1] - pw[1]) * (lv[1] - pw[1])
                           + (lv[2] - pw[2]) * (lv[2] - pw[2]));
        }
        for (int k = 0; k < 3; ++k) V[3 * b + k] = acc[k];
        for (int k = 0; k < 6; ++k) H[6 * b + k] = h[k];
        VA[b] = ab;
        VS[b] = as;
        HN[b] = hn;
    }
    /* near part, per source leaf, then add the far sums of all nodes containing j */
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nn; ++b) {
        if (t->nchild[b] != 0) continue;
        for (int64_t j = t->start[b]; j < t->start[b] + t->count[b]; ++j) {
            const double* x = t->x + 3 * j;
            double acc[3] = {0, 0, 0}, ab = 0.0, as = 0.0;
            for (int64_t q = ncnt[b]; q < ncnt[b + 1]; ++q) {
                int64_t g = ngp[q];
                int64_t s = T->goff[g], e = T->goff[g + 1];
                for (int64_t i = s; i < e; ++i) {
                    double d[3] = {x[0] - T->y[3 * i], x[1] - T->y[3 * i + 1], x[2] - T->y[3 * i + 2]};
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    int amb_p = amb_sorted && ambiguous(r2, w2, amb_tol);
                    if (!keep_pair(r2, w2) && !amb_p) continue;
                    double v[3];
                    term_AT(d, r2, s_sorted[i], v);
                    double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                    if (amb_p) ab += vn;
                    if (keep_pair(r2, w2)) {
                        for (int k = 0; k < 3; ++k) acc[k] += v[k];
                        as += vn;
                    }
                }
            }
            double far[3] = {0, 0, 0};
            for (int64_t a = b; a >= 0; a = t->parent[a]) {
                for (int k = 0; k < 3; ++k) far[k] += V[3 * a + k];
                ab += VA[a];
                as += VS[a];
                if (far_order == 1) {
                    const double dl[3] = {x[0] - rep[3 * a], x[1] - rep[3 * a + 1], x[2] - rep[3 * a + 2]};
                    double hd[3];
                    sym_mul(H + 6 * a, dl, hd);
                    for (int k = 0; k < 3; ++k) far[k] -= hd[k];
                    as += HN[a] * sqrt(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]);
                }
            }
            for (int k = 0; k < 3; ++k) out_sorted[3 * j + k] = acc[k] + far[k];
            if (amb_sorted) amb_sorted[j] = ab;
            if (abs_sorted) abs_sorted[j] = as;
        }
    }
    free(fcnt); free(ncnt); free(fg); free(ngp); free(fpos); free(npos); free(V); free(VA); free(VS);
    free(H); free(HN); free(LS); free(SD); free(LSC); free(SDC); free(fq);
}

/* On-surface application of an operator.  nu and out are in input order,
 * normalised units.  For op AT, rep_mode 1 gives the exact transpose of the
 * rep_mode-1 A, rep_mode 0 the paper's s-representative treecode. */
void or_tree_apply(const or_tree* T, int op, int rep_mode, double w, const double* nu, double* out,
                   double amb_tol, double* amb, double* abssum) {
    const or_octree* t = &T->src;
    int64_t n = t->n;
    int din = (op == OP_AT) ? 1 : 3, dout = (op == OP_A) ? 1 : 3;
    double* nus = malloc(sizeof(double) * din * (n > 0 ? n : 1));
    double* outs = malloc(sizeof(double) * dout * (n > 0 ? n : 1));
    double* ambs = amb ? malloc(sizeof(double) * (n > 0 ? n : 1)) : NULL;
    double* abss = abssum ? malloc(sizeof(double) * (n > 0 ? n : 1)) : NULL;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < din; ++k) nus[din * i + k] = nu[din * t->perm[i] + k];
    local_cfg cfg = {T->local_c, T->local_cluster, T->self_cls};
    if (op == OP_AT && rep_mode == 1)
        tree_adjoint_exact(t, &T->self, w, nus, outs, amb_tol, ambs, abss, T->far_order,
                           T->self_cls ? &cfg : NULL);
    else tree_gather(t, &T->self, op, rep_mode, w, nus, outs, amb_tol, ambs, abss, T->far_order,
                     T->self_cls ? &cfg : NULL);
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < dout; ++k) out[dout * T->self.perm[i] + k] = outs[dout * i + k];
        if (amb) amb[T->self.perm[i]] = ambs[i];
        if (abssum) abssum[T->self.perm[i]] = abss[i];
    }
    free(nus); free(outs); free(ambs); free(abss);
}

/* Off-surface targets (op A or G): the targets are grouped and listed
 * against the source octree exactly like the on-surface set. */
void or_tree_apply_at(const or_tree* T, int op, int rep_mode, double w, const double* nu,
                      const double* qn, int64_t m, double* out, int64_t* pairs2, double* abssum) {
    const or_octree* t = &T->src;
    or_targets Q;
    memset(&Q, 0, sizeof(Q));
    build_targets(&Q, t, qn, m, T->self.group_size, T->theta, -1, 0);
    int64_t n = t->n;
    int dout = (op == OP_A) ? 1 : 3;
    double* nus = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* outs = malloc(sizeof(double) * dout * (m > 0 ? m : 1));
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) nus[3 * i + k] = nu[3 * t->perm[i] + k];
    double* abss = abssum ? malloc(sizeof(double) * (m > 0 ? m : 1)) : NULL;
    local_cfg cfg = {T->local_c, T->local_cluster, NULL};
    if (T->local_c > 0.0) cfg.cls = local_classes(t, &Q, T->local_c, T->local_cluster);
    tree_gather(t, &Q, op, rep_mode, w, nus, outs, 0.0, NULL, abss, T->far_order, cfg.cls ? &cfg : NULL);
    free(cfg.cls);
    for (int64_t i = 0; i < m; ++i) {
        for (int k = 0; k < dout; ++k) out[dout * Q.perm[i] + k] = outs[dout * i + k];
        if (abssum) abssum[Q.perm[i]] = abss[i];
    }
    free(abss);
    if (pairs2) { pairs2[0] = Q.far_pairs; pairs2[1] = Q.near_pairs; }
    free(nus); free(outs);
    free_targets(&Q);
}

/* ------------------------------------------------------------------------ */
/* The paper's treecode (Sec. 4.5, Eq. 13-14, Alg. 4), per target.           */
/*                                                                          */
/* Octree: the root is the cube [-1,1]^3 (depth 0, width 2); a cube of      */
/* depth d has width 2/2^d and is split into its eight octants (a point     */
/* goes to the upper half of an axis iff its coordinate is >= the cube's    */
/* centre on that axis) while it holds more than leaf_size points and       */
/* d < max_depth.  Empty octants are dropped.  Each node's points are one   */
/* contiguous range of the permutation idx.                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n, nnodes, cap;
    int leaf_size, max_depth;
    const double* x;      /* sources, caller's array (n x 3), not copied */
    int64_t* idx;         /* node ranges index into this permutation of 0..n-1 */
    int64_t *start, *count;
    int64_t* child;       /* 8 per node, -1 for an empty octant */
    int* depth;
    int* nchild;
    double* ctr;          /* cube centre (3 per node) */
} or_ptree;

static int64_t pt_new_node(or_ptree* P) {
    if (P->nnodes == P->cap) {
        P->cap = P->cap ? 2 * P->cap : 1024;
        P->start = realloc(P->start, sizeof(int64_t) * P->cap);
        P->count = realloc(P->count, sizeof(int64_t) * P->cap);
        P->child = realloc(P->child, sizeof(int64_t) * 8 * P->cap);
        P->depth = realloc(P->depth, sizeof(int) * P->cap);
        P->nchild = realloc(P->nchild, sizeof(int) * P->cap);
        P->ctr = realloc(P->ctr, sizeof(double) * 3 * P->cap);
    }
    int64_t b = P->nnodes++;
    for (int q = 0; q < 8; ++q) P->child[8 * b + q] = -1;
    P->nchild[b] = 0;
    return b;
}

/* Split node b into octants (recursively).  tmp: scratch of n entries. */
static void pt_split(or_ptree* P, int64_t b, int64_t* tmp) {
    if (P->count[b] <= P->leaf_size || P->depth[b] >= P->max_depth) return;
    const int64_t s = P->start[b], e = s + P->count[b];
    const double* c = P->ctr + 3 * b;
    const double quarter = ldexp(1.0, -P->depth[b]) * 0.5;   /* child half-width = width/4 */
    int64_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int* oct = malloc(sizeof(int) * (size_t)(e - s));
    for (int64_t k = s; k < e; ++k) {
        const double* p = P->x + 3 * P->idx[k];
        int o = (p[0] >= c[0] ? 4 : 0) | (p[1] >= c[1] ? 2 : 0) | (p[2] >= c[2] ? 1 : 0);
        oct[k - s] = o;
        cnt[o]++;
    }
    int64_t off[8];
    off[0] = s;
    for (int o = 1; o < 8; ++o) off[o] = off[o - 1] + cnt[o - 1];
    int64_t pos[8];
    memcpy(pos, off, sizeof(pos));
    for (int64_t k = s; k < e; ++k) tmp[pos[oct[k - s]]++] = P->idx[k];
    memcpy(P->idx + s, tmp + s, sizeof(int64_t) * (size_t)(e - s));
    free(oct);
    for (int o = 0; o < 8; ++o) {
        if (cnt[o] == 0) continue;
        int64_t ch = pt_new_node(P);
        c = P->ctr + 3 * b;                       /* the node arrays may have moved */
        P->child[8 * b + o] = ch;
        P->nchild[b]++;
        P->start[ch] = off[o];
        P->count[ch] = cnt[o];
        P->depth[ch] = P->depth[b] + 1;
        P->ctr[3 * ch + 0] = c[0] + ((o & 4) ? quarter : -quarter);
        P->ctr[3 * ch + 1] = c[1] + ((o & 2) ? quarter : -quarter);
        P->ctr[3 * ch + 2] = c[2] + ((o & 1) ? quarter : -quarter);
    }
    for (int o = 0; o < 8; ++o)
        if (P->child[8 * b + o] >= 0) pt_split(P, P->child[8 * b + o], tmp);
}

or_ptree* or_ptree_build(const double* xs, int64_t n, int leaf_size, int max_depth) {
    or_ptree* P = calloc(1, sizeof(or_ptree));
    P->n = n; P->x = xs; P->leaf_size = leaf_size; P->max_depth = max_depth;
    P->idx = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) P->idx[i] = i;
    if (n > 0) {
        int64_t r = pt_new_node(P);
        P->start[r] = 0; P->count[r] = n; P->depth[r] = 0;
        P->ctr[0] = P->ctr[1] = P->ctr[2] = 0.0;
        int64_t* tmp = malloc(sizeof(int64_t) * (size_t)n);
        pt_split(P, r, tmp);
        free(tmp);
    }
    return P;
}

void or_ptree_free(or_ptree* P) {
    if (!P) return;
    free(P->idx); free(P->start); free(P->count); free(P->child); free(P->depth); free(P->nchild);
    free(P->ctr);
    free(P);
}

int64_t or_ptree_nnodes(const or_ptree* P) { return P->nnodes; }
/* per node: first index into idx, point count, depth, number of children */
void or_ptree_nodes(const or_ptree* P, int64_t* start, int64_t* count, int* depth, int* nchild, double* ctr,
                    int64_t* idx) {
    for (int64_t b = 0; b < P->nnodes; ++b) {
        start[b] = P->start[b]; count[b] = P->count[b]; depth[b] = P->depth[b]; nchild[b] = P->nchild[b];
        for (int k = 0; k < 3; ++k) ctr[3 * b + k] = P->ctr[3 * b + k];
    }
    memcpy(idx, P->idx, sizeof(int64_t) * (size_t)P->n);
}

/* Representatives of one call (Eq. 13, Eq. 14):
 *   x_{B,nu} = sum_i |nu_i| x_i / sum_j |nu_j|,   nu_B = sum_i nu_i,
 * |nu_i| the Euclidean length (dim 3) or the absolute value (dim 1).  A
 * node whose nu all vanish has nu_B = 0 and contributes nothing whichever
 * way it is used; its representative is then the plain centroid. */
static void pt_reps(const or_ptree* P, const double* nu, int dim, double* rep, double* nuB) {
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t b = 0; b < P->nnodes; ++b) {
        double sw = 0.0, sx[3] = {0, 0, 0}, sc[3] = {0, 0, 0}, sn[3] = {0, 0, 0};
        for (int64_t k = P->start[b]; k < P->start[b] + P->count[b]; ++k) {
            const int64_t i = P->idx[k];
            double a = 0.0;
            for (int q = 0; q < dim; ++q) { sn[q] += nu[dim * i + q]; a += nu[dim * i + q] * nu[dim * i + q]; }
            a = sqrt(a);
            sw += a;
            for (int q = 0; q < 3; ++q) { sx[q] += a * P->x[3 * i + q]; sc[q] += P->x[3 * i + q]; }
        }
        for (int q = 0; q < 3; ++q)
            rep[3 * b + q] = sw > 0.0 ? sx[q] / sw : sc[q] / (double)P->count[b];
        for (int q = 0; q < dim; ++q) nuB[dim * b + q] = sn[q];
    }
}

typedef struct {
    const or_ptree* P;
    int op, dim;
    double c, w2, amb_tol;
    const double* nu;
    const double *rep, *nuB;
} pt_ctx;

typedef struct { double v[3]; double amb, abssum; int64_t far, near; } pt_acc;

/* One term with the cut-off of Sec. 4.4 (kept iff r >= w), d = y - x. */
static void pt_term(const pt_ctx* C, const double d[3], const double* nu, pt_acc* a) {
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const int amb_p = C->amb_tol > 0.0 && ambiguous(r2, C->w2, C->amb_tol);
    if (!keep_pair(r2, C->w2) && !amb_p) return;
    double v[3] = {0, 0, 0};
    if (C->op == OP_A) v[0] = term_A(d, r2, nu);
    else if (C->op == OP_G) term_G(d, r2, nu, v);
    else term_AT(d, r2, nu[0], v);
    const double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (amb_p) a->amb += vn;
    if (keep_pair(r2, C->w2)) {
        for (int k = 0; k < 3; ++k) a->v[k] += v[k];
        a->abssum += vn;
    }
}

/* Alg. 4, apply(y, B): far term, else recurse into the children, else the
 * leaf's points.  A far decision whose squared distance lies within
 * amb_tol (c width)^2 of the threshold is "ambiguous": a lower-precision
 * evaluation may take the other branch, so both branches are evaluated and
 * their difference is added to the ambiguity budget. */
static void pt_apply(const pt_ctx* C, const double* y, int64_t b, pt_acc* a) {
    const or_ptree* P = C->P;
    const double* xb = C->rep + 3 * b;
    const double d[3] = {y[0] - xb[0], y[1] - xb[1], y[2] - xb[2]};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double cw = C->c * ldexp(2.0, -P->depth[b]);
    const int far = C->c < INFINITY && r2 > cw * cw;
    const int amb_far = C->amb_tol > 0.0 && C->c < INFINITY && fabs(r2 - cw * cw) <= C->amb_tol * cw * cw;
    pt_acc fa = {{0, 0, 0}, 0, 0, 0, 0}, re = {{0, 0, 0}, 0, 0, 0, 0};
    if (far || amb_far) {
        pt_term(C, d, C->nuB + C->dim * b, &fa);
        fa.far = 1;
    }
    if (!far || amb_far) {
        if (P->nchild[b] > 0) {
            for (int q = 0; q < 8; ++q)
                if (P->child[8 * b + q] >= 0) pt_apply(C, y, P->child[8 * b + q], &re);
        } else {
            for (int64_t k = P->start[b]; k < P->start[b] + P->count[b]; ++k) {
                const int64_t j = P->idx[k];
                const double dj[3] = {y[0] - P->x[3 * j], y[1] - P->x[3 * j + 1], y[2] - P->x[3 * j + 2]};
                pt_term(C, dj, C->nu + C->dim * j, &re);
                re.near++;
            }
        }
    }
    const pt_acc* take = far ? &fa : &re;
    for (int k = 0; k < 3; ++k) a->v[k] += take->v[k];
    a->abssum += take->abssum;
    a->amb += take->amb;
    a->far += take->far;
    a->near += take->near;
    if (amb_far) {
        const double dd[3] = {fa.v[0] - re.v[0], fa.v[1] - re.v[1], fa.v[2] - re.v[2]};
        const pt_acc* other = far ? &re : &fa;
        a->amb += sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]) + other->amb;
    }
}

/* Treecode sum of op at nt targets yt (nt x 3):
 *   op A : nu = mu (ns x 3), out (nt)        op G : nu = mu, out (nt x 3) = -sum HPhi mu
 *   op AT: nu = s (ns),      out (nt x 3) = sum_i s_i gradPhi(x_i - y)  (s-representatives)
 * theta = 1/c (0: never far, the direct sum).  amb, abssum (optional, per
 * target) as in or_direct, amb also covering ambiguous far decisions.
 * counts (optional): total far (target, node) and near (target, point) terms. */
void or_ptree_apply(const or_ptree* P, int op, double theta, double w, const double* nu, const double* yt,
                    int64_t nt, double* out, double amb_tol, double* amb, double* abssum, int64_t* counts) {
    const int dim = (op == OP_AT) ? 1 : 3;
    const int64_t nn = P->nnodes > 0 ? P->nnodes : 1;
    double* rep = malloc(sizeof(double) * 3 * (size_t)nn);
    double* nuB = malloc(sizeof(double) * (size_t)dim * (size_t)nn);
    pt_reps(P, nu, dim, rep, nuB);
    pt_ctx C = {P, op, dim, theta > 0.0 ? 1.0 / theta : INFINITY, eff_w2(w), amb_tol, nu, rep, nuB};
    int64_t tfar = 0, tnear = 0;
    #pragma omp parallel for schedule(dynamic, 16) reduction(+ : tfar, tnear)
    for (int64_t t = 0; t < nt; ++t) {
        pt_acc a = {{0, 0, 0}, 0, 0, 0, 0};
        if (P->nnodes > 0) pt_apply(&C, yt + 3 * t, 0, &a);
        if (op == OP_A) out[t] = a.v[0];
        else for (int k = 0; k < 3; ++k) out[3 * t + k] = a.v[k];
        if (amb) amb[t] = a.amb;
        if (abssum) abssum[t] = a.abssum;
        tfar += a.far;
        tnear += a.near;
    }
    if (counts) { counts[0] = tfar; counts[1] = tnear; }
    free(rep); free(nuB);
}

/* ------------------------------------------------------------------------ */
/* Alg. 3: n iterations of grad step (Alg. 2) + WNNC update + rescale, with  */
/* the width schedule of or_schedule_width2 (the paper's is the linear one). */
/*   T != NULL: the group treecode; else P != NULL: the paper's treecode    */
/*   (Alg. 4) at opening parameter ptheta; else the direct sums over xn.     */
/*   mu (n x 3, input order, normalised units) is updated in place.          */
/*   rescale 0: mu_i <- muhat_i |mu_i| / |muhat_i|  (Alg. 3)                 */
/*   rescale 1: mu_i <- muhat_i sigma_i / |muhat_i|  (Eq. 19, needs area)    */
/*   use_grad / use_wnnc switch the two halves off for the ablations of      */
/*   Sec. 5.5.2 / Sec. 6.1.3.                                                */
/*   stats (optional, per iteration): w, E = |A mu - b|^2 before the step,   */
/*   alpha, |r|^2.                                                           */
/* ------------------------------------------------------------------------ */
/* The operator of the iteration: the group treecode T, else the paper's
 * treecode P at opening parameter ptheta, else the direct sums. */
static void apply_op(const or_tree* T, const or_ptree* P, double ptheta, const double* xn, int64_t n, int op,
                     int rep_mode, double w, const double* nu, double* out) {
    if (T) or_tree_apply(T, op, rep_mode, w, nu, out, 0.0, NULL, NULL);
    else if (P) or_ptree_apply(P, op, ptheta, w, nu, xn, n, out, 0.0, NULL, NULL, NULL);
    else or_direct(op, xn, n, nu, xn, n, w, 0.0, out, NULL, NULL);
}

/* Width of iteration i of n (Sec. 4.4 and Alg. 3).  With t = (i-1)/(n-1)
 * running from 0 at the first iteration to 1 at the last:
 *   schedule 0, linear (the paper's):  w = w2 (1 - t) + w1 t
 *   schedule 1, cosine:                w = w1 + (w2 - w1) (1 + cos(pi t)) / 2
 *   schedule 2, exponential:           w = w2 (w1 / w2)^t   (w1, w2 > 0)
 * Sec. 6.1.2 reports that cosine and exponential decays were tried and gave
 * no clear difference; it prints no formula for them, so these are the
 * standard forms that fall smoothly from w2 to w1.  n = 1 gives w1. */
double or_schedule_width2(int i, int n_iter, double w1, double w2, int schedule) {
    if (n_iter <= 1) return w1;
    if (schedule == 0)
        return w2 * (double)(n_iter - i) / (double)(n_iter - 1) + w1 * (double)(i - 1) / (double)(n_iter - 1);
    const double t = (double)(i - 1) / (double)(n_iter - 1);
    if (schedule == 1) return w1 + (w2 - w1) * 0.5 * (1.0 + cos(acos(-1.0) * t));
    return w2 * pow(w1 / w2, t);
}

double or_schedule_width(int i, int n_iter, double w1, double w2) {
    return or_schedule_width2(i, n_iter, w1, w2, 0);
}

void or_iterate(const or_tree* T, const or_ptree* P, double ptheta, const double* xn, int64_t n, double* mu,
                int n_iter, int first_iter, int last_iter, double w1, double w2, int rep_mode, int rescale,
                const double* area, int use_grad, int use_wnnc, int schedule, double* stats) {
    double* a = malloc(sizeof(double) * (n > 0 ? n : 1));
    double* s = malloc(sizeof(double) * (n > 0 ? n : 1));
    double* r = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* q = malloc(sizeof(double) * (n > 0 ? n : 1));
    double* muhat = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    for (int it = first_iter; it <= last_iter; ++it) {
        double w = or_schedule_width2(it, n_iter, w1, w2, schedule);
        double E = 0.0, rr = 0.0, qq = 0.0, alpha = 0.0;
        if (use_grad) {
            /* Alg. 2:  r = A^T b - A^T A mu = A^T (b - A mu);  alpha = r.r / |A r|^2;  mu += alpha r */
            apply_op(T, P, ptheta, xn, n, OP_A, rep_mode, w, mu, a);
            for (int64_t i = 0; i < n; ++i) { s[i] = 0.5 - a[i]; E += s[i] * s[i]; }
            apply_op(T, P, ptheta, xn, n, OP_AT, rep_mode, w, s, r);
            for (int64_t i = 0; i < 3 * n; ++i) rr += r[i] * r[i];
            apply_op(T, P, ptheta, xn, n, OP_A, rep_mode, w, r, q);
            for (int64_t i = 0; i < n; ++i) qq += q[i] * q[i];
            alpha = qq > 0.0 ? rr / qq : 0.0;
            for (int64_t i = 0; i < 3 * n; ++i) mu[i] += alpha * r[i];
        }
        if (use_wnnc) {
            /* WNNC update muhat = G_w(mu), then rescale */
            apply_op(T, P, ptheta, xn, n, OP_G, rep_mode, w, mu, muhat);
            for (int64_t i = 0; i < n; ++i) {
                double hn = sqrt(muhat[3 * i] * muhat[3 * i] + muhat[3 * i + 1] * muhat[3 * i + 1] +
                                 muhat[3 * i + 2] * muhat[3 * i + 2]);
                if (!(hn > 0.0)) continue;
                double len;
                if (rescale == 1 && area) len = area[i];
                else len = sqrt(mu[3 * i] * mu[3 * i] + mu[3 * i + 1] * mu[3 * i + 1] + mu[3 * i + 2] * mu[3 * i + 2]);
                for (int k = 0; k < 3; ++k) mu[3 * i + k] = muhat[3 * i + k] * len / hn;
            }
        }
        if (stats) {
            double* st = stats + 4 * (it - first_iter);
            st[0] = w; st[1] = E; st[2] = alpha; st[3] = rr;
        }
    }
    free(a); free(s); free(r); free(q); free(muhat);
}

/* ------------------------------------------------------------------------ */
/* k nearest neighbours by exhaustive search (ties by index), excluding the  */
/* point itself.  out: n x k indices, dist2: n x k squared distances.        */
/* ------------------------------------------------------------------------ */
void or_knn(const double* x, int64_t n, int k, int64_t* out, double* dist2) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        int64_t* idx = out + (int64_t)k * i;
        double* dd = dist2 + (int64_t)k * i;
        int cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (cnt == k && !(r2 < dd[k - 1])) continue;
            int p = cnt < k ? cnt++ : k - 1;
            while (p > 0 && dd[p - 1] > r2) { dd[p] = dd[p - 1]; idx[p] = idx[p - 1]; --p; }
            dd[p] = r2; idx[p] = j;
        }
    }
}
