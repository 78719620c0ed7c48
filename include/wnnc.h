/*
 * wnnc.h -- C ABI of the B300 (sm_103a) WNNC treecode library.
 *
 * The library evaluates, on one GPU, the three linear operators of the
 * Winding-Number-Normal-Consistency normal-orientation method
 * (Lin, Shi, Liu, "Fast and Globally Consistent Normal Orientation based on
 * the Winding Number Normal Consistency", Sec. 4):
 *
 *   A(mu)_i  = sum_j gradPhi(x_i - x_j) . mu_j         winding number F(x_i; mu)  (Eq. 5, Eq. 6)
 *   G(mu)_i  = -sum_j HPhi(x_i - x_j) mu_j              = -grad F(x_i; mu)          (Eq. 9, Eq. 10)
 *   A^T(s)_j = sum_i s_i gradPhi(x_i - x_j)             adjoint of A (Sec. 4.5)
 *
 *   gradPhi(y) = -y / (4 pi |y|^3)                        (Thm. 1)
 *   HPhi(y)    = -I/(4 pi |y|^3) + 3 y y^T / (4 pi |y|^5) (Eq. 9)
 *
 * with every pair term set to zero when |x_i - x_j| < w (smoothing width,
 * Sec. 4.4), accelerated by a treecode over an octree of the points
 * (Sec. 4.5, Eq. 13-14, Alg. 4), and the iteration of Alg. 3 (width
 * schedule, gradient step of Alg. 2, WNNC update, rescale).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers marked "device" are CUDA device pointers; "host" are host
 *    pointers.  Arrays of points/normals are row-major float32 [n][3]
 *    (a contiguous torch tensor of shape (n, 3)), in the caller's input order.
 *  - The caller owns every input and output buffer.  The library owns only
 *    wnnc_tree objects (and the device memory inside them).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Evaluation and iteration calls are asynchronous on that stream; build
 *    and free synchronise with it.  Calls that use the same tree must not run
 *    concurrently (they share the tree's work buffers).
 *  - Units: positions and normals are in the caller's units.  The tree
 *    normalises the cloud into [-1,1]^3 with a 1/11 margin (Sec. 5.1.1):
 *    x' = (x - c) * s.  The smoothing width w is given in those normalised
 *    units, as in the paper.  mu scales like area (mu' = s^2 mu); results are
 *    returned in caller units (F is dimensionless, grad F scales by s,
 *    A^T v by s^2, so that <A mu, v> = <mu, A^T v> in caller units).
 *  - Errors: every call returns a wnnc_status.  Argument and launch errors
 *    are reported at once.  Conditions detected on the device (a non-finite
 *    step length in the iteration) are latched in the tree and returned by
 *    wnnc_sync_status.  wnnc_last_error() returns a thread-local text for the
 *    last failure.  No exception crosses this boundary.
 */
#ifndef WNNC_H
#define WNNC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wnnc_tree wnnc_tree;

typedef enum {
    WNNC_OK = 0,
    WNNC_EINVAL = 1,      /* bad argument (NULL pointer, n < 1, w < 0, theta < 0, ...) */
    WNNC_ENOMEM = 2,      /* device or host allocation failed */
    WNNC_ECUDA = 3,       /* a CUDA runtime call failed */
    WNNC_ENONFINITE = 4,  /* the iteration produced a non-finite step length */
    WNNC_ECAPACITY = 5,   /* a traversal stack or list capacity was exceeded */
    WNNC_ETIMEOUT = 6     /* a bounded device wait gave up (single-pass scans and sorts of a build) */
} wnnc_status;

/* Tree parameters (Sec. 5.1.1 defaults: D = 15, c = 2 i.e. theta = 0.5). */
typedef struct {
    int max_depth;     /* maximum octree depth D, root = depth 0; 1..15 (default 15) */
    int leaf_size;     /* a node is split while it holds more than this many points
                          (the paper splits down to 1 point); 1..1024 (default 8, the
                          fastest measured on B300 at 50k-2M points) */
    float theta;       /* opening parameter, 1/c of Alg. 4; 0 = exact direct sums (default 0.5) */
    int rep_mode;      /* node representative (Eq. 13): 1 = point centroid, which makes the
                          tree operator linear so that A^T is its exact transpose (default);
                          0 = |nu|-weighted centroid as in the paper (A^T is then the paper's
                          s-representative treecode, not an exact transpose) */
    int moments_fp64;  /* 1 = sum node moments in double precision, and sum the moments of
                          every G step directly instead of deriving them from those of mu
                          and r by linearity (default 0: single precision) */
    int near_bf16;     /* 1 = round the near-field coordinates (offsets in the target group's
                          frame, sources and targets) to bfloat16 before the pair terms of A, G
                          and the fused A+G; the adjoint stays in float, so A^T is then not the
                          exact transpose.  A precision study, not a fast path (default 0) */
    int criterion;     /* far-field decisions (Alg. 4):
                          0 = once per group of at most 32 Morton-consecutive targets: node B is
                              far when the gap between the group's box and B's box exceeds
                              width(B)/theta, so every target also passes Alg. 4's test; the
                              lists are built once with the tree and reused by every call
                              (default, the fast path);
                          1 = the paper's own test, per target and per call: every target walks
                              the octree from the root and takes B as far iff
                              |x_i - x_{B,nu}| > width(B)/theta with the representative of that
                              call (Eq. 13).  Needs rep_mode 0 and near_bf16 0 (else
                              WNNC_EINVAL).  With leaf_size 1 this is Alg. 4 as printed.  A
                              reference mode: warps diverge, several times slower.
                              wnnc_get_stats still counts the group lists' pairs */
    int far_order;     /* order of each far node's term (criterion 0, rep_mode 1):
                          0 = the node's summed nu at its point centroid x_B (Eq. 13-14; default);
                          1 = plus the first-order Taylor terms of gradPhi and HPhi about x_B,
                              from the node moment S = sum_j sym((x_j - x_B) nu_j^T); A^T stays
                              the exact transpose (per-node sums of s HPhi pushed down as
                              -H_B (x_j - x_B)).  The step toward the expansions of an FMM that
                              Sec. 4.5 and Sec. 6.3 name for precision control: the far-field
                              error falls as (h/R)^2 instead of h/R.  Other values, or
                              far_order 1 with rep_mode 0 or criterion 1: WNNC_EINVAL */
    float local_theta; /* local expansions of the far field about each target group (criterion 0,
                          rep_mode 1, far_order 0): a far node B whose box gap to a group's
                          box exceeds the box's largest extent / local_theta is not summed
                          against each target; its terms of A and G are expanded to first order
                          about the group box centre c_g (value and gradient of A, value and
                          Jacobian of G = -grad A, summed over those nodes once per group and
                          evaluated at each target), and A^T takes the exact transpose
                          (per entry, S_g gradPhi + HPhi D_g from the group's sum of s and of
                          s (x_i - c_g)).  An entry is expanded only when every one of its pairs
                          clears the cut-off (|c_g - x_B| - rho_g >= w, rho_g the group's
                          radius about c_g); otherwise it is summed pair by pair.  The
                          target-side counterpart of the expansions that Sec. 4.5 and Sec. 6.3
                          name; its error is second order in (group extent / distance).
                          0 = off (default); negative, non-finite, or > 0 with rep_mode 0,
                          criterion 1 or far_order 1: WNNC_EINVAL */
    int local_cluster; /* with local_theta > 0, a second level of local expansions: clusters of
                          local_cluster consecutive target groups (2..8; 0 = none, the default).
                          A far node that lies in the expanded part of every member group's list
                          and is itself local for the cluster's box (the union of the members'
                          boxes, the same test) is expanded once about the cluster's box centre
                          instead of once per member, and its A^T term is taken once per
                          cluster; the cut-off rule is the group's with the cluster's radius
                          (otherwise the entry's pairs are summed).  Other values: WNNC_EINVAL */
} wnnc_tree_params;

/* Iteration parameters (Alg. 3; Sec. 5.1.1 defaults n = 40, w1 = 0.002, w2 = 0.016). */
typedef struct {
    int n_iter;        /* n of the width schedule (linear: w_i = w2 (n-i)/(n-1) + w1 (i-1)/(n-1)) */
    int first_iter;    /* first i to run (1 = from the start; >1 resumes a saved run) */
    int last_iter;     /* last i to run (0 = n_iter) */
    float w1, w2;      /* final and initial smoothing widths, normalised units */
    int init;          /* 0 = start from mu = 0 (the paper); 1 = start from mu_inout */
    int rescale;       /* 0 = |mu_i| kept across the WNNC update (Alg. 3);
                          1 = |mu_i| set to the given area sigma_i (Eq. 19) */
    int use_grad;      /* 1 = gradient step of Alg. 2 (default); 0 = skip it (ablation) */
    int use_wnnc;      /* 1 = WNNC update + rescale (default); 0 = skip it (ablation) */
    int schedule;      /* width schedule from w2 down to w1, with t = (i-1)/(n-1) (n = 1: w1):
                          0 = linear w2 (1-t) + w1 t (Alg. 3, default);
                          1 = cosine w1 + (w2-w1)(1 + cos(pi t))/2;
                          2 = exponential w2 (w1/w2)^t, needs w1, w2 > 0.
                          Sec. 6.1.2 names cosine and exponential decays as tried
                          alternatives without giving formulas; these are the standard
                          smooth forms.  Other values: WNNC_EINVAL */
} wnnc_iter_params;

/* Fill p with the defaults listed above.  Returns WNNC_EINVAL if p is NULL. */
wnnc_status wnnc_tree_params_default(wnnc_tree_params* p);
wnnc_status wnnc_iter_params_default(wnnc_iter_params* p);

/*
 * Build the octree (Sec. 4.5: split until leaf_size points or depth D),
 * node boxes and centroids, and the interaction lists of the points as
 * targets (Alg. 4's far / recurse / leaf-direct decisions, taken once per
 * group of at most 32 Morton-consecutive targets against its bounding box).
 *   pts    device, float32 [n][3], caller units, all finite; read during the
 *          call only.
 *   n      number of points, >= 1.
 *   params host, may be NULL for the defaults.
 *   out    host; receives the new tree (NULL on failure).
 * Synchronises with `stream`.  Errors: WNNC_EINVAL (also for a NaN or
 * infinite coordinate), WNNC_ENOMEM, WNNC_ECUDA, WNNC_ECAPACITY.
 */
wnnc_status wnnc_build_tree(const float* pts, int64_t n, const wnnc_tree_params* params,
                            void* stream, wnnc_tree** out);

/* Release a tree and its device memory (synchronises with the device). NULL is a no-op. */
wnnc_status wnnc_tree_free(wnnc_tree* tree);

/*
 * F(x_i; mu) = A_w(mu)_i at every input point (Eq. 5 with the cut-off of Sec. 4.4).
 *   mu  device, float32 [n][3], caller units (oriented area elements).
 *   w   smoothing width (normalised units), >= 0; w = 0 only drops coincident pairs.
 *   out device, float32 [n].
 */
wnnc_status wnnc_eval_w(const wnnc_tree* tree, const float* mu, float w, float* out, void* stream);

/*
 * grad F(x_i; mu) = -G_w(mu)_i at every input point (Eq. 8-10).
 *   mu  device, float32 [n][3];  out device, float32 [n][3] (caller units).
 */
wnnc_status wnnc_eval_grad(const wnnc_tree* tree, const float* mu, float w, float* out, void* stream);

/*
 * A_w^T(s) at every input point (Sec. 4.5; the backward of F with respect to mu).
 *   s   device, float32 [n];  out device, float32 [n][3] (caller units).
 * With rep_mode 1 this is the exact transpose of wnnc_eval_w's operator.
 */
wnnc_status wnnc_eval_adjoint(const wnnc_tree* tree, const float* s, float w, float* out, void* stream);

/*
 * F(q_k; mu) (grad = 0) or grad F(q_k; mu) (grad = 1) at m query points that
 * need not be input points (Thm. 1: 1 inside, 0 outside, 1/2 on the surface).
 *   q   device, float32 [m][3], caller units, all finite (else WNNC_EINVAL);  m >= 1.
 *   out device, float32 [m] (grad = 0) or [m][3] (grad = 1).
 * Builds the queries' interaction lists (allocates) and synchronises with `stream`.
 */
wnnc_status wnnc_eval_at(const wnnc_tree* tree, const float* mu, const float* q, int64_t m,
                         float w, int grad, float* out, void* stream);

/*
 * Run iterations first_iter..last_iter of Alg. 3 on the tree's points.
 *   mu_inout device, float32 [n][3], caller units: the initial field when
 *            init = 1 (ignored when init = 0), the result on return.
 *   area     device, float32 [n] (caller units) for rescale = 1, else NULL.
 *   params   host; NULL for the defaults.
 *   stats    device, float32 [last-first+1][4] or NULL: per iteration the width
 *            w_i, the energy E = |A mu - b|^2 before the step (Eq. 12, b = 1/2),
 *            the step length alpha and |r|^2 (Alg. 2), in normalised units.
 * Asynchronous; a non-finite alpha is latched (WNNC_ENONFINITE).
 */
wnnc_status wnnc_iterate(wnnc_tree* tree, float* mu_inout, const float* area,
                         const wnnc_iter_params* params, void* stream, float* stats);

/*
 * The whole orientation from host memory to host memory (Sec. 4.5 + Alg. 3):
 * copy the points to the device, build the tree, run iterations first..last of
 * Alg. 3, copy the field back.  For callers without device buffers; the
 * copies are faster from pinned (page-locked) host memory.
 *   pts_host  host, float32 [n][3], caller units, all finite.
 *   tree_params, iter_params  host, either may be NULL for the defaults.
 *   area_host host, float32 [n] (rescale = 1), else NULL.
 *   mu_host   host, float32 [n][3]: the initial field when init = 1, the
 *             oriented field (caller units) on return.
 * Allocates its device buffers and the tree, frees them before returning, and
 * synchronises with `stream`.  Errors: those of wnnc_build_tree,
 * wnnc_iterate and wnnc_sync_status; mu_host is unspecified after an error.
 */
wnnc_status wnnc_orient(const float* pts_host, int64_t n, const wnnc_tree_params* tree_params,
                        const wnnc_iter_params* iter_params, const float* area_host, float* mu_host,
                        void* stream);

/* Interaction counts of one on-surface operator evaluation: far (target, node)
 * pairs and near (target, source) pairs summed pair by pair, cut-off ones
 * included (far entries expanded about their group's centre are counted by
 * wnnc_get_local_stats instead).  host out. */
wnnc_status wnnc_get_stats(const wnnc_tree* tree, int64_t* far_pairs, int64_t* near_pairs);

/* Far entries that the local expansions (local_theta > 0) evaluate once per
 * target group instead of per target, and the (target, node) pairs they stand
 * for; both 0 when local_theta = 0.  An entry that the cut-off reaches on a
 * call is summed pair by pair on that call but still counted here.  host out. */
wnnc_status wnnc_get_local_stats(const wnnc_tree* tree, int64_t* local_entries, int64_t* local_pairs);

/* With local_cluster > 0: the (cluster, node) expansions of the second level
 * and the (target, node) pairs they stand for (not counted by
 * wnnc_get_local_stats); both 0 otherwise.  host out. */
wnnc_status wnnc_get_cluster_stats(const wnnc_tree* tree, int64_t* cluster_entries, int64_t* cluster_pairs);

/*
 * Sizes of the tree (host out, any may be NULL): points, nodes, leaves,
 * target groups, far-list entries, merged near ranges, transposed near entries,
 * maximum depth reached.
 */
wnnc_status wnnc_tree_info(const wnnc_tree* tree, int64_t* n, int64_t* nnodes, int64_t* nleaves,
                           int64_t* ngroups, int64_t* far_entries, int64_t* near_ranges,
                           int64_t* tnear_entries, int* depth);

/*
 * How the interaction-list traversal of the tree's own points ran (Alg. 4's
 * decisions for every target group; either way the lists are the same).  Each
 * group is first walked breadth first, which writes its far nodes in
 * ascending id; a group whose walk grows too wide for the per-warp buffer
 * finishes depth first and has its far list sorted afterwards
 * (*stack_walk_groups counts them).  If a depth-first walk overflows as well,
 * every group runs again depth first with a larger buffer and all far lists
 * are sorted (*big_stack = 1, *stack_walk_groups = 0).  Either output may be
 * NULL.  Errors: WNNC_EINVAL for a NULL tree.
 */
wnnc_status wnnc_tree_walk_stats(const wnnc_tree* tree, int* stack_walk_groups, int* big_stack);

/*
 * Copy the tree's structure to host buffers (any may be NULL), for checking
 * against an independent construction:
 *   perm        int64 [n]        sorted position -> input index
 *   node_start  int32 [nnodes]   first sorted point of each node (breadth-first order)
 *   node_count  int32 [nnodes]
 *   node_depth  int32 [nnodes]
 *   node_nchild int32 [nnodes]   0 for leaves
 *   far_off     int32 [ngroups+1], far_id int32 [far_entries]  per group, ascending node id
 *               (local_theta > 0: two ascending parts, see wnnc_tree_export_local)
 *   near_off    int32 [ngroups+1], near_rng int32 [near_ranges][2]  [start,end) point ranges
 *               (consecutive near leaves merged, then cut to at most 256 points)
 *   group_off   int32 [ngroups+1]  target group g = sorted points group_off[g]..group_off[g+1]-1
 *               (at most 32; a new group starts where consecutive points' leaves share no
 *               ancestor within 3 levels of the deeper leaf, or lie in different depth-3 cells)
 *   center_scale float64 [4]     normalisation centre c (3) and scale s
 */
wnnc_status wnnc_tree_export(const wnnc_tree* tree, int64_t* perm, int32_t* node_start,
                             int32_t* node_count, int32_t* node_depth, int32_t* node_nchild,
                             int32_t* far_off, int32_t* far_id, int32_t* near_off,
                             int32_t* near_rng, int32_t* group_off, double* center_scale);

/* With local_theta > 0 each group's far list holds first the entries summed
 * pair by pair, then (from far_lsplit[g] on) the entries expanded about the
 * group's centre, then (from far_csplit[g] on, local_cluster > 0) those
 * expanded about its cluster's centre, each part ascending by node id.
 * far_lsplit, far_csplit: int32 [ngroups], host out (far_off[g + 1] where a
 * part is absent).  WNNC_EINVAL if either is NULL. */
wnnc_status wnnc_tree_export_local(const wnnc_tree* tree, int32_t* far_lsplit, int32_t* far_csplit);

/*
 * Kernel timing (not in the paper; the tracing facility of this library).
 * When enabled, every kernel launch of the evaluation and iteration calls is
 * bracketed by CUDA events on the launching stream and attributed to one of
 * the classes below.  wnnc_profile_read synchronises with those events and
 * returns, per class, the number of launches and their summed device time in
 * milliseconds since the last reset (host out, arrays of WNNC_PROF_CLASSES
 * entries, either may be NULL).  Enabling adds two event records per launch.
 */
enum {
    WNNC_PROF_MOMENTS = 0,   /* node moments (Eq. 13, Eq. 14) */
    WNNC_PROF_A = 1,         /* treecode sum of A (Eq. 5, Alg. 4) */
    WNNC_PROF_ADJ_FAR = 2,   /* adjoint: far (target group, node) sums */
    WNNC_PROF_ADJ_NODE = 3,  /* adjoint: per-node reduction */
    WNNC_PROF_ADJ_NEAR = 4,  /* adjoint: near sums + push-down of node sums */
    WNNC_PROF_G = 5,         /* treecode sum of G + rescale (Eq. 10, Alg. 3) */
    WNNC_PROF_SMALL = 6,     /* permutations, step length, axpy, WNNC update */
    WNNC_PROF_AG = 7,        /* fused treecode sums of A and G on one field (the default
                                iteration: A(mu) with G(mu), A(r) with G(r)) */
    WNNC_PROF_LOCAL = 8,     /* far entries expanded about their target group's centre
                                (local_theta > 0): the terms of A and G, and of A^T */
    WNNC_PROF_CLASSES = 9
};
wnnc_status wnnc_profile_enable(wnnc_tree* tree, int enable);
/* Restrict the recording to the classes whose bit is set in mask (bit k:
 * class k above); the default is every class.  Each recorded launch group
 * costs two events on its stream, so a caller timing a long run can record
 * only the class it needs.  Errors: WNNC_EINVAL for a NULL tree. */
wnnc_status wnnc_profile_classes(wnnc_tree* tree, unsigned mask);
wnnc_status wnnc_profile_read(wnnc_tree* tree, int64_t* launches, double* total_ms);
wnnc_status wnnc_profile_reset(wnnc_tree* tree);

/* ------------------------------------------------------------------------ */
/* Learned warm start (not in the paper).  A point-patch MLP maps the 16      */
/* nearest neighbours of a point (offsets divided by the 16th neighbour's     */
/* distance, nearest first, 48 values) through 128-128-128 ReLU layers to an  */
/* oriented normal; it is trained on the method's own converged normals and   */
/* starts the iteration (init = 1) on the tail of the width schedule.         */
/* ------------------------------------------------------------------------ */

/*
 * k = 16 nearest neighbours of every tree point (the point itself excluded)
 * and its patch features.  Exact neighbours (FP32 distances in local frames).
 *   idx  device, int32 [n][16] (input indices, nearest first) or NULL
 *   feat device, float32 [n][48]: (x_j - x_i) / |x_j16 - x_i| for the 16
 *        neighbours j1..j16 in order, or NULL.  Synchronises with `stream`.
 */
wnnc_status wnnc_knn16(const wnnc_tree* tree, int32_t* idx, float* feat, void* stream);

typedef struct wnnc_mlp wnnc_mlp;
enum { WNNC_MLP_PARAMS = 39683 };   /* 48*128+128 + 2*(128*128+128) + 128*3+3 */

/*
 * Parameter layout (FP32, flat): W1 [128][48], b1 [128], W2 [128][128], b2,
 * W3 [128][128], b3, W4 [3][128], b4 [3].  Every parameter (weights and
 * biases) is rounded to BF16 when read; products accumulate in FP32.  The
 * forward runs on the BF16 tensor cores (activations enter as BF16 hi + lo
 * pairs, ~16 significant bits).  max_batch bounds the rows of one gradient or
 * training call (forward calls take any number of rows).  The MLP owns its
 * work buffers (allocated here).
 */
wnnc_status wnnc_mlp_create(int64_t max_batch, wnnc_mlp** out);
wnnc_status wnnc_mlp_free(wnnc_mlp* mlp);
/* Copy parameters in (device [WNNC_MLP_PARAMS]); resets the Adam state. */
wnnc_status wnnc_mlp_set_params(wnnc_mlp* mlp, const float* params, void* stream);
wnnc_status wnnc_mlp_get_params(const wnnc_mlp* mlp, float* params, void* stream);
/* y [B][3] = network(x [B][48]) (device pointers). */
wnnc_status wnnc_mlp_forward(wnnc_mlp* mlp, const float* x, int64_t B, float* y, void* stream);
/*
 * Training loss per row, with c = (y/|y|).label: mode 0 (default) 1 - c,
 * mode 1 1 - c^2 (indifferent to the sign of y).  Other modes: WNNC_EINVAL.
 */
wnnc_status wnnc_mlp_set_loss(wnnc_mlp* mlp, int mode);
/*
 * Gradient of the mean loss over B <= max_batch rows with
 * respect to the parameters.  grad device [WNNC_MLP_PARAMS] or NULL (kept
 * inside for the next train step); loss device [1] or NULL.
 */
wnnc_status wnnc_mlp_grad(wnnc_mlp* mlp, const float* x, const float* label, int64_t B, float* grad,
                          float* loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the gradient of (x, label). */
wnnc_status wnnc_mlp_train_step(wnnc_mlp* mlp, const float* x, const float* label, int64_t B, float lr,
                                float* loss, void* stream);
/*
 * Warm-start field: mu_i = L_i * dir_i / |dir_i|, negated where
 * dir_i . ref_i < 0 (ref: the field after one iteration of the method, or
 * NULL for no sign correction), with L_i = area if area > 0, else |ref_i|.
 * dir, ref, mu device float32 [n][3].
 */
wnnc_status wnnc_warm_init(const float* dir, const float* ref, int64_t n, float area, float* mu,
                           void* stream);

/* Number of kernels this library has launched in this process so far (all
 * threads, all trees); for counting the launches inside a timed region. */
int64_t wnnc_kernel_launches(void);

/*
 * Diagnostic (no counterpart in the paper): the FP32 FMA throughput of the
 * current device in TFLOP/s, measured with eight independent FMA chains per
 * thread on all SMs and timed with CUDA events on `stream` (synchronises).
 * The pair kernels are bound by FP32 issue; this is their measured ceiling.
 */
wnnc_status wnnc_probe_fp32(double* tflops, void* stream);

/*
 * Diagnostic (no counterpart in the paper): runs one block of the build's
 * single-pass scan on `stream` with the tile before its own never published
 * (a look-back word that nothing sets), so that its bounded wait gives up,
 * then synchronises and reads the device's timeout count.  Returns
 * WNNC_ETIMEOUT when the wait gave up and was reported as the builds report
 * it (the count is cleared and the context stays usable; the wait lasts about
 * a second at most); any other status means that the bound or the report
 * failed.  Used by the tests of the failure paths.
 */
wnnc_status wnnc_selftest_wait_timeout(void* stream);

/*
 * F(q_k; mu) at m query points by direct summation over all n points, with no
 * tree and no device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc (a host application
 * that owns all device memory through its own pool, a plugin sandbox, or a
 * latency-critical path where an allocation that may synchronise the device is
 * not acceptable).  It uses the normalisation, cut-off and units of the tree
 * entry points, and its results agree with wnnc_eval_at on a tree built with
 * theta = 0 from the same points within the FP32 rounding of the two sums
 * (the sums run in different frames and orders, so a pair at r = w can fall
 * on either side of the cut-off).
 *   pts device, float32 [n][3], all finite; mu device, float32 [n][3];
 *   q   device, float32 [m][3], all finite;  out device, float32 [m];
 *   w   smoothing width (normalised units), >= 0
 *   n   at most 32768 points (larger n returns WNNC_EINVAL with a message).
 * A NaN or infinite point or query coordinate returns WNNC_EINVAL (out is
 * then unspecified).  Scratch lives in a fixed array of about 1 MiB inside
 * the library's device image (held by every GPU that loads the library until
 * the process exits).  The first call on a device looks up that array's
 * device address; make that first call before any stream capture.  All calls
 * on a device share the array: calls whose kernels may overlap on the GPU
 * (different streams without ordering) race, so order them.  The call waits
 * for its stream before it returns (it reads back the non-finite flags).
 */
wnnc_status wnnc_eval_w_direct_noalloc(const float* pts, int64_t n, const float* mu, const float* q,
                                       int64_t m, float w, float* out, void* stream);

/*
 * Fault injection for tests (no counterpart in the paper): after `after` more
 * successful device allocations by the library, the next one fails as if the
 * device were out of memory, and the call that made it returns WNNC_ENOMEM
 * (then the injection switches itself off).  after < 0 switches it off.
 * Building a tree allocates; evaluation and iteration do not (wnnc_eval_at
 * allocates its query lists).  A process-wide setting: do not use it while
 * other threads call the library.  Returns WNNC_OK.
 */
wnnc_status wnnc_debug_fail_alloc(int64_t after);

/* Wait for the stream and return (and clear) any condition latched on the device. */
wnnc_status wnnc_sync_status(wnnc_tree* tree, void* stream);

/* Thread-local description of the last failed call ("" if none). */
const char* wnnc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WNNC_H */
