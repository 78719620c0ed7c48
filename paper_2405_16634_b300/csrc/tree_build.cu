// tree_build.cu -- normalisation, Morton order, octree, node boxes and
// centroids, target groups and interaction lists (forward and transposed).
//
// Sec. 4.5 builds an octree that stops splitting at one point or at depth D,
// and Alg. 4 decides, per target and node, between a far (representative)
// interaction, recursion, and a leaf direct sum.  Here the decision is taken
// once per group of 32 Morton-consecutive targets (one warp), against the
// group's bounding box: node B is far for the group when the gap between the
// two bounding boxes exceeds c * width(B).  Every target and the node's
// representative lie inside those boxes, so each far use also passes the
// per-target test of Alg. 4.  The test is evaluated in double precision with
// explicit round-to-nearest operations (no contraction), so that any
// implementation of the same rule takes identical decisions.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace wnnc {

namespace {

constexpr int kTB = 256;

// ---------------------------------------------------------------------------
// Normalisation (Sec. 5.1.1) and Morton keys
// ---------------------------------------------------------------------------

__global__ void k_bbox_partial(const float* pts, int64_t n, double* part) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double v = (double)pts[3 * i + k];
            if (!isfinite(v)) {          // the box becomes infinite: the host rejects the cloud
                lo[k] = -INFINITY;
                hi[k] = INFINITY;
            }
            lo[k] = fmin(lo[k], v);
            hi[k] = fmax(hi[k], v);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    __shared__ double s[2][3][32];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) { s[0][k][warp] = lo[k]; s[1][k][warp] = hi[k]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            for (int k = 0; k < 3; ++k) {
                lo[k] = fmin(lo[k], s[0][k][w]);
                hi[k] = fmax(hi[k], s[1][k][w]);
            }
        for (int k = 0; k < 3; ++k) { part[6 * blockIdx.x + k] = lo[k]; part[6 * blockIdx.x + 3 + k] = hi[k]; }
    }
}

// centre (3) and scale: centre of the bounding box, largest half-extent -> 10/11
// One block: thread b takes partial b, then a tree reduction (min and max are
// exact, so the result does not depend on the order).
__global__ void __launch_bounds__(1024) k_bbox_final(const double* part, int nparts, double* cs) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], part[6 * b + k]);
            hi[k] = fmax(hi[k], part[6 * b + 3 + k]);
        }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    __shared__ double sh[2][3][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) { sh[0][k][warp] = lo[k]; sh[1][k][warp] = hi[k]; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], sh[0][k][w]);
            hi[k] = fmax(hi[k], sh[1][k][w]);
        }
    double hmax = 0.0;
    for (int k = 0; k < 3; ++k) {
        cs[k] = __dmul_rn(__dadd_rn(lo[k], hi[k]), 0.5);
        double h = __dmul_rn(__dsub_rn(hi[k], lo[k]), 0.5);
        if (h > hmax) hmax = h;
    }
    cs[3] = hmax > 0.0 ? (10.0 / 11.0) / hmax : 1.0;
}

__device__ __forceinline__ int64_t quant15(double v) {
    double q = floor(__dmul_rn(__dadd_rn(v, 1.0), 16384.0));
    q = fmin(fmax(q, 0.0), 32767.0);
    return (int64_t)q;
}

// 45-bit key, 15 bits per axis, x the high bit of each 3-bit digit.
__device__ __forceinline__ uint64_t morton45(double x, double y, double z) {
    int64_t q[3] = {quant15(x), quant15(y), quant15(z)};
    uint64_t key = 0;
#pragma unroll
    for (int b = 14; b >= 0; --b) {
        uint64_t dig = (uint64_t)((((q[0] >> b) & 1) << 2) | (((q[1] >> b) & 1) << 1) | ((q[2] >> b) & 1));
        key = (key << 3) | dig;
    }
    return key;
}

// Normalised coordinates (double) and Morton keys of float32 caller-unit points.
__global__ void k_normalize_keys(const float* pts, int64_t n, const double* cs, double* xn,
                                 uint64_t* keys, uint32_t* idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = cs[3];
    double v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = __dmul_rn(__dsub_rn((double)pts[3 * i + k], cs[k]), s);
        xn[3 * i + k] = v[k];
    }
    keys[i] = morton45(v[0], v[1], v[2]);
    idx[i] = (uint32_t)i;
}

__global__ void k_keys_from_xn(const double* xn, int64_t n, uint64_t* keys, uint32_t* idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = morton45(xn[3 * i], xn[3 * i + 1], xn[3 * i + 2]);
    idx[i] = (uint32_t)i;
}

__global__ void k_gather_sorted(const double* xn, const uint32_t* idx, int64_t n, double* xs,
                                int64_t* perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = idx[i];
    perm[i] = j;
#pragma unroll
    for (int k = 0; k < 3; ++k) xs[3 * i + k] = xn[3 * j + k];
}

// ---------------------------------------------------------------------------
// Octree, level by level (breadth-first numbering, children in digit order)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int digit_at(uint64_t key, int depth_of_parent) {
    return (int)((key >> (3 * (14 - depth_of_parent))) & 7u);
}

// First index in [s, e) whose digit (below the parent's depth) is >= c.
__device__ __forceinline__ int first_digit_ge(const uint64_t* keys, int s, int e, int d, int c) {
    int lo = s, hi = e;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (digit_at(keys[mid], d) < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One level of the octree: eight threads per node, thread q finding by binary
// search the first point of the node whose digit at this depth is > q (the
// end of child q's range), all eight searches at once; a node splits if it
// holds more than leaf_size points and is above the maximum depth.  bnd[8i+q]
// keeps the ends for k_split_write; nkids[i] counts the non-empty children.
__global__ void k_split_count(const uint64_t* keys, const int* start, const int* count, int base,
                              int m, int depth, int leaf_size, int max_depth, int* nkids, int* bnd) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t >> 3), q = (int)(t & 7);
    const unsigned lane = threadIdx.x & 31u;
    const bool act = i < m;
    int s = 0, e = 0;
    bool split = false;
    if (act) {
        const int b = base + i;
        s = start[b];
        e = s + count[b];
        split = count[b] > leaf_size && depth < max_depth;
    }
    int p = e;
    if (split && q < 7) p = first_digit_ge(keys, s, e, depth, q + 1);
    int pp = __shfl_up_sync(0xffffffffu, p, 1, 8);   // the end of child q - 1
    if (q == 0) pp = s;
    const unsigned nonempty = __ballot_sync(0xffffffffu, split && p > pp);
    if (act) {
        bnd[(int64_t)8 * i + q] = p;
        if (q == 0) nkids[i] = __popc((nonempty >> (lane & ~7u)) & 0xffu);
    }
}

__global__ void k_split_write(int* start, int* count, int* parent, int* child0, int* nchild, int* ndepth,
                              int base, int m, int depth, int next_base, const int* koff, const int* nkids,
                              const int* bnd) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int b = base + i;
    int nk = nkids[i];
    if (nk == 0) {
        child0[b] = -1;
        nchild[b] = 0;
        return;
    }
    int c0 = next_base + koff[i];
    child0[b] = c0;
    nchild[b] = nk;
    int prev = start[b], w = 0;
    for (int q = 0; q < 8; ++q) {
        const int p = bnd[(int64_t)8 * i + q];
        if (p > prev) {
            int c = c0 + w++;
            start[c] = prev;
            count[c] = p - prev;
            parent[c] = b;
            ndepth[c] = depth + 1;
        }
        prev = p;
    }
}

// ---------------------------------------------------------------------------
// The whole octree in one cooperative launch (every block resident): level by
// level as k_split_count / k_split_write do, the blocks meeting at a grid
// barrier after the child counts of a level (phase A) and after its children
// are written (phase B).  Block k takes a contiguous slice of the level's
// nodes; a node's children go after the children of every node before it
// (the slices' totals, then a scan inside the slice), so the ids are those of
// the launch-per-level build.  If the nodes would pass the capacity, no
// children of that level are written and the caller builds by launches.
// ---------------------------------------------------------------------------
struct GridBar {
    unsigned count;
    unsigned gen;
    int err;            // a wait gave up
};
constexpr int kBarrierPolls = 1 << 20;   // with back-off: well under a second of polling

// Barrier of all blocks of a cooperative launch: each block arrives on the
// counter; the last to arrive resets it and bumps the generation, which the
// others poll (at most kBarrierPolls times: then the error flag, and on).
__device__ void grid_barrier(GridBar* gb) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &gb->gen;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(&gb->count, 1u) == gridDim.x - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            int polls = 0;
            while (*gen == g) {
                if (++polls > kBarrierPolls) {
                    atomicOr(&gb->err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

constexpr int kOctThreads = 256;
constexpr int kOctMaxLevels = kMaxDepth + 2;

struct OctArgs {
    const uint64_t* keys;
    int n, leaf_size, max_depth, cap;
    int *start, *count, *parent, *child0, *nchild, *depth;
    int* bnd;           // [8 x largest level]
    int* nkids;         // [largest level]
    int* block_tot;     // [gridDim.x]
    int* lvl;           // [kOctMaxLevels] nodes per level
    GridBar* bar;
    int* status;        // [0] nodes, [1] capacity exceeded
};

// Sum over the block of one value per thread, and the exclusive scan.
__device__ __forceinline__ int oct_block_scan(int v, int* total) {
    __shared__ int ws[kOctThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    int before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kOctThreads / 32; ++w) {
        if (w < warp) before += ws[w];
        all += ws[w];
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

__global__ void __launch_bounds__(kOctThreads) k_octree(OctArgs A) {
    const int G = (int)gridDim.x, blk = (int)blockIdx.x, tid = (int)threadIdx.x;
    const unsigned lane = threadIdx.x & 31u;
    if (blk == 0 && tid == 0) {
        A.start[0] = 0;
        A.count[0] = A.n;
        A.parent[0] = -1;
        A.depth[0] = 0;
        A.lvl[0] = 1;
    }
    grid_barrier(A.bar);
    int base = 0, m = 1, d = 0, total = 1;
    for (;;) {
        const int chunk = (m + G - 1) / G;
        const int B0 = min(blk * chunk, m), B1 = min(B0 + chunk, m);
        // phase A: eight threads per node, thread q finding the end of child q
        int mine = 0;
        for (int i0 = B0; i0 < B1; i0 += kOctThreads / 8) {
            const int i = i0 + (tid >> 3), q = tid & 7;
            const bool act = i < B1;
            int s = 0, e = 0;
            bool split = false;
            if (act) {
                const int b = base + i;
                s = A.start[b];
                e = s + A.count[b];
                split = A.count[b] > A.leaf_size && d < A.max_depth;
            }
            int p = e;
            if (split && q < 7) p = first_digit_ge(A.keys, s, e, d, q + 1);
            int pp = __shfl_up_sync(0xffffffffu, p, 1, 8);
            if (q == 0) pp = s;
            const unsigned nonempty = __ballot_sync(0xffffffffu, split && p > pp);
            if (act) {
                A.bnd[(int64_t)8 * i + q] = p;
                if (q == 0) {
                    const int nk = __popc((nonempty >> (lane & ~7u)) & 0xffu);
                    A.nkids[i] = nk;
                    mine += nk;
                }
            }
        }
        int bsum = 0;
        oct_block_scan(mine, &bsum);
        if (tid == 0) A.block_tot[blk] = bsum;
        grid_barrier(A.bar);
        // phase B: this slice's first child id, then the children
        int before = 0, all = 0;
        for (int k = tid; k < G; k += kOctThreads) {
            const int v = A.block_tot[k];
            all += v;
            if (k < blk) before += v;
        }
        int pre = 0, tot = 0;
        oct_block_scan(before, &pre);
        oct_block_scan(all, &tot);
        const bool overflow = (int64_t)total + tot > (int64_t)A.cap;
        if (!overflow) {
            int carry = 0;
            for (int i0 = B0; i0 < B1; i0 += kOctThreads) {
                const int i = i0 + tid;
                const int v = i < B1 ? A.nkids[i] : 0;
                int tile = 0;
                const int ex = oct_block_scan(v, &tile);
                if (i < B1) {
                    const int b = base + i;
                    if (v == 0) {
                        A.child0[b] = -1;
                        A.nchild[b] = 0;
                    } else {
                        const int c0 = total + pre + carry + ex;
                        A.child0[b] = c0;
                        A.nchild[b] = v;
                        int prev = A.start[b], w = 0;
                        for (int q = 0; q < 8; ++q) {
                            const int p = A.bnd[(int64_t)8 * i + q];
                            if (p > prev) {
                                const int c = c0 + w++;
                                A.start[c] = prev;
                                A.count[c] = p - prev;
                                A.parent[c] = b;
                                A.depth[c] = d + 1;
                            }
                            prev = p;
                        }
                    }
                }
                carry += tile;
            }
        }
        if (blk == 0 && tid == 0) {
            A.lvl[d + 1] = overflow ? 0 : tot;
            if (overflow) A.status[1] = 1;
        }
        grid_barrier(A.bar);
        if (overflow) break;
        base = total;
        total += tot;
        m = tot;
        ++d;
        if (m == 0 || d + 1 >= kOctMaxLevels) break;
    }
    if (blk == 0 && tid == 0) A.status[0] = total;
}

// Bounding boxes and point sums of all nodes in one launch, from the leaves
// up: a thread takes a leaf (its points in order), then climbs while it is
// the last of its parent's children to finish (a counter per node); the last
// child sums the parent from all its children in child order, so the sums
// are those of a level-by-level pass.  Children's values are written before
// the counter is raised (fence) and read by the last one past L1 (__ldcg).
__device__ __forceinline__ void node_box_store(double* lo, double* hi, double* sum, int b, const double* l,
                                               const double* h, const double* sm) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[3 * b + k] = l[k];
        hi[3 * b + k] = h[k];
        sum[3 * b + k] = sm[k];
    }
}

__global__ void k_node_boxes(const double* xs, const int* start, const int* count, const int* child0,
                             const int* nchild, const int* parent, int nn, double* lo, double* hi, double* sum,
                             int* arrive) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nn || nchild[b] != 0) return;
    double l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
    double sm[3] = {0, 0, 0};
    for (int j = start[b]; j < start[b] + count[b]; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double v = xs[3 * (int64_t)j + k];
            l[k] = fmin(l[k], v);
            h[k] = fmax(h[k], v);
            sm[k] += v;
        }
    node_box_store(lo, hi, sum, b, l, h, sm);
    for (;;) {
        const int p = parent[b];
        if (p < 0) break;
        __threadfence();
        const int nc = nchild[p];
        if (atomicAdd(&arrive[p], 1) != nc - 1) break;
        __threadfence();
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            l[k] = INFINITY;
            h[k] = -INFINITY;
            sm[k] = 0.0;
        }
        for (int q = 0; q < nc; ++q) {
            const int c = child0[p] + q;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                l[k] = fmin(l[k], __ldcg(lo + 3 * c + k));
                h[k] = fmax(h[k], __ldcg(hi + 3 * c + k));
                sm[k] += __ldcg(sum + 3 * c + k);
            }
        }
        node_box_store(lo, hi, sum, p, l, h, sm);
        b = p;
    }
}

// Cell centre (exact dyadic), width, centroid offset; leaf ownership of points.
__global__ void k_node_cells(const uint64_t* keys, const int* start, const int* count,
                             const int* ndepth, const int* nchild, const double* sum, int nn,
                             float4* cell, float4* cent, int* leaf_of) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nn) return;
    int d = ndepth[b];
    uint64_t key = keys[start[b]];
    int q[3] = {0, 0, 0};
    for (int bit = 14; bit >= 0; --bit) {
        int dig = (int)((key >> (3 * bit)) & 7u);
        q[0] = (q[0] << 1) | ((dig >> 2) & 1);
        q[1] = (q[1] << 1) | ((dig >> 1) & 1);
        q[2] = (q[2] << 1) | (dig & 1);
    }
    double width = ldexp(2.0, -d);
    double c[3];
    for (int k = 0; k < 3; ++k) c[k] = -1.0 + ((double)(q[k] >> (15 - d)) + 0.5) * width;
    cell[b] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)width);
    double inv = 1.0 / (double)count[b];
    cent[b] = make_float4((float)(sum[3 * b] * inv - c[0]), (float)(sum[3 * b + 1] * inv - c[1]),
                          (float)(sum[3 * b + 2] * inv - c[2]), 0.f);
    if (nchild[b] == 0)
        for (int j = start[b]; j < start[b] + count[b]; ++j) leaf_of[j] = b;
}

// ---------------------------------------------------------------------------
// Target groups and coordinate frames
// ---------------------------------------------------------------------------

__device__ __forceinline__ double dyadic12(double v) { return rint(v * 4096.0) * 0x1p-12; }   // exact scaling

// Warp minimum and maximum of doubles without the (slow) FP64 pipe: finite
// doubles and infinities map to signed 64-bit integers in the same order
// (negative values with their magnitude bits flipped), an involution.
__device__ __forceinline__ long long dord(double v) {
    const long long k = __double_as_longlong(v);
    return k ^ ((k >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dord_inv(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
__device__ __forceinline__ void warp_minmax_d(double& l, double& h) {
    long long a = dord(l), b = dord(h);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a = min(a, __shfl_xor_sync(0xffffffffu, a, d));
        b = max(b, __shfl_xor_sync(0xffffffffu, b, d));
    }
    l = dord_inv(a);
    h = dord_inv(b);
}

// Number of leading 3-bit digits two 45-bit keys share (0..15).
__device__ __forceinline__ int common_digits(uint64_t a, uint64_t b) {
    uint64_t x = a ^ b;
    if (x == 0) return 15;
    int hb = 63 - __clzll((long long)x);
    return 14 - hb / 3;
}

// Group rule for the points as targets: a new group starts before sorted
// point k when the leaves of k-1 and k share no ancestor within `slack`
// levels of the deeper leaf (the keys share fewer than that many digits), or
// when the two points lie in different cells of depth `min_depth`.
__global__ void k_group_cuts(const uint64_t* keys, const int* leaf_of, const int* ndepth, int64_t m,
                             int slack, int min_depth, int* cut) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    int c = 1;
    if (k > 0) {
        int d = max(ndepth[leaf_of[k - 1]], ndepth[leaf_of[k]]);
        const int cd = common_digits(keys[k - 1], keys[k]);
        c = cd < d - slack || cd < min_depth;
    }
    cut[k] = c;
}

// out[scan[k]] = k for every flagged k.
__global__ void k_compact(const int* flag, const int* scan, int64_t m, int* out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m && flag[k]) out[scan[k]] = (int)k;
}

// Runs between cuts are cut again into groups of at most 32.
__global__ void k_run_ngroups(const int* run_start, int nruns, int64_t m, int* cnt) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns) return;
    int e = r + 1 < nruns ? run_start[r + 1] : (int)m;
    cnt[r] = (e - run_start[r] + kGroup - 1) / kGroup;
}

__global__ void k_run_goff(const int* run_start, int nruns, int64_t m, const int* cnt_off, int* goff) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns) return;
    int e = r + 1 < nruns ? run_start[r + 1] : (int)m;
    int b = cnt_off[r];
    for (int s = run_start[r], j = 0; s < e; s += kGroup, ++j) goff[b + j] = s;
    if (r == nruns - 1) goff[cnt_off[nruns]] = (int)m;
}

__global__ void k_fixed_goff(int ng, int64_t m, int* goff) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g <= ng) goff[g] = (int)min((int64_t)g * kGroup, m);
}

// Warp per fixed chunk of 32 sorted targets: dyadic origin and float offsets.
__global__ void k_chunk_frames(const double* ys, int64_t m, int nchunks, float4* corig, float4* pos) {
    int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (c >= nchunks) return;
    int64_t i = (int64_t)c * kGroup + lane;
    bool valid = i < m;
    double o[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = valid ? ys[3 * i + k] : 0.0;
        double l = valid ? v : INFINITY, h = valid ? v : -INFINITY;
        warp_minmax_d(l, h);
        o[k] = dyadic12(0.5 * (l + h));
    }
    if (lane == 0) corig[c] = make_float4((float)o[0], (float)o[1], (float)o[2], 0.f);
    if (valid)
        pos[i] = make_float4((float)(ys[3 * i] - o[0]), (float)(ys[3 * i + 1] - o[1]),
                             (float)(ys[3 * i + 2] - o[2]), 0.f);
}

// Warp per group: bounding box and dyadic origin, the box in the group's
// frame rounded outward to float (it contains every target of the group), and
// for the local expansions (gctr, may be null) the box centre in that frame
// with the group's radius about it, rounded up.
__global__ void k_group_boxes(const double* ys, const int* goff, int ng, double* glo, double* ghi,
                              float4* gorig, float4* gbl, float4* gbh, float4* gctr) {
    int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (g >= ng) return;
    int64_t i = (int64_t)goff[g] + lane;
    bool valid = i < goff[g + 1];
    double o[3], bl[3], bh[3], v[3], c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = valid ? ys[3 * i + k] : 0.0;
        double l = valid ? v[k] : INFINITY, h = valid ? v[k] : -INFINITY;
        warp_minmax_d(l, h);
        if (lane == 0) { glo[3 * g + k] = l; ghi[3 * g + k] = h; }
        c[k] = 0.5 * (l + h);
        o[k] = dyadic12(c[k]);
        bl[k] = l - o[k];
        bh[k] = h - o[k];
    }
    if (gctr) {
        // the largest distance from the centre: the square root of the largest
        // square (the same value: sqrt is monotone and correctly rounded)
        double r2 = 0.0;
        if (valid) {
            const double dx = v[0] - c[0], dy = v[1] - c[1], dz = v[2] - c[2];
            r2 = dx * dx + dy * dy + dz * dz;
        }
        double lo2 = r2;
        warp_minmax_d(lo2, r2);
        const double r = sqrt(r2);
        if (lane == 0)
            gctr[g] = make_float4((float)(c[0] - o[0]), (float)(c[1] - o[1]), (float)(c[2] - o[2]),
                                  __double2float_ru(r));
    }
    if (lane == 0) {
        gorig[g] = make_float4((float)o[0], (float)o[1], (float)o[2], 0.f);
        gbl[g] = make_float4(__double2float_rd(bl[0]), __double2float_rd(bl[1]), __double2float_rd(bl[2]), 0.f);
        gbh[g] = make_float4(__double2float_ru(bh[0]), __double2float_ru(bh[1]), __double2float_ru(bh[2]), 0.f);
    }
}

// Float copies of the node boxes, rounded outward.
__global__ void k_node_fbox(const double* lo, const double* hi, int nn, float4* lof, float4* hif) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nn) return;
    lof[b] = make_float4(__double2float_rd(lo[3 * b]), __double2float_rd(lo[3 * b + 1]),
                         __double2float_rd(lo[3 * b + 2]), 0.f);
    hif[b] = make_float4(__double2float_ru(hi[3 * b]), __double2float_ru(hi[3 * b + 1]),
                         __double2float_ru(hi[3 * b + 2]), 0.f);
}

// FP32 pre-test of the far criterion on outward-rounded boxes: 1 = far, 0 = not
// far, -1 = undecided.  Node coordinates lie in [-1, 1] and the group's within
// [-S, S] (S > 1 only for query points outside the cloud), so each outward
// rounding moves a face by less than 1.2e-7 S and each float subtraction
// rounds by at most 1.2e-7 (1 + S): the float gap per axis is within
// 4.8e-7 (1 + S) of the exact one, the distance within 8.4e-7 (1 + S) (plus a
// relative 1e-7 from the float sum of squares).  With a margin of
// 1e-6 (1 + S) + 1e-6 cw a decision here is the one the exact FP64 test would
// take; the rest goes to that test.
__device__ __forceinline__ float gap2_f(const float4& nl, const float4& nh, const float4& gl, const float4& gh) {
    const float ax = fmaxf(fmaxf(nl.x - gh.x, gl.x - nh.x), 0.f);
    const float ay = fmaxf(fmaxf(nl.y - gh.y, gl.y - nh.y), 0.f);
    const float az = fmaxf(fmaxf(nl.z - gh.z, gl.z - nh.z), 0.f);
    return fmaf(ax, ax, fmaf(ay, ay, az * az));
}

// The same pre-test of d2 (the float gap squared) against a threshold cwf.
__device__ __forceinline__ int far_pretest(float d2, float cwf, float mscale) {
    const float m = mscale + 1e-6f * cwf;
    const float up = cwf + m, dn = cwf - m;
    if (d2 > up * up) return 1;
    if (dn > 0.f && d2 < dn * dn) return 0;
    return -1;
}

// Squared gap between a group box and node b's box, in double precision as
// written (no fused multiply-adds).
__device__ __forceinline__ double box_gap2_d(const double* nlo, const double* nhi, int b, const double* glo,
                                             const double* ghi) {
    double gq[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double a = __dsub_rn(nlo[3 * b + k], ghi[k]);
        double e = __dsub_rn(glo[k], nhi[3 * b + k]);
        double mm = a > e ? a : e;
        gq[k] = mm > 0.0 ? mm : 0.0;
    }
    double gx = __dmul_rn(gq[0], gq[0]), gy = __dmul_rn(gq[1], gq[1]), gz = __dmul_rn(gq[2], gq[2]);
    return __dadd_rn(__dadd_rn(gx, gy), gz);
}

// Far test of a group box against node b (see the file comment).
__device__ __forceinline__ bool is_far(const double* nlo, const double* nhi, const int* ndepth,
                                       int b, const double* glo, const double* ghi, double c) {
    double d2 = box_gap2_d(nlo, nhi, b, glo, ghi);
    double cw = __dmul_rn(c, ldexp(2.0, -ndepth[b]));
    return d2 > __dmul_rn(cw, cw);
}

// Local-expansion test of a far node b: its squared box gap to the group
// exceeds (cL e)^2, e the group box's largest extent (cle = cL e).
__device__ __forceinline__ bool is_local(const double* nlo, const double* nhi, int b, const double* glo,
                                         const double* ghi, double cle) {
    return box_gap2_d(nlo, nhi, b, glo, ghi) > __dmul_rn(cle, cle);
}

constexpr int kTravWarps = 2;
// Per-warp traversal buffer (shared memory): the first-in first-out walk uses
// the smaller, which allows more resident warps; a walk that overflows it runs
// again as a stack walk with the larger.
constexpr int kStackSmall = 2048;
constexpr int kStackBig = 4096;

// Warp-cooperative traversal of the octree for one target group, one pass:
// it writes far node ids and, for near leaves, keys (group << nsh | first
// point) with the leaf id, both in chunks (below); the near lists are sorted
// by first point afterwards.
// Up to 32 nodes are tested at once; children of opened nodes go into a
// per-warp shared buffer whose capacity is checked before a push.
//
// FIFO = true: the buffer is a ring visited first-in first-out.  Nodes are
// numbered level by level, children of one parent consecutively and child
// blocks in the order of their parents, so a first-in first-out walk from the
// root visits nodes in ascending id and each group's far nodes come out
// ascending.  The width of that walk grows with the group's box (a box
// spanning many cells opens many nodes per level); when fewer than 256 free
// slots (32 nodes x 8 children) remain, the warp finishes its group as a
// stack walk in the same ring and appends the group to `unsorted`, whose far
// lists the caller sorts by node afterwards.  FIFO = false: a stack walk
// (last-in first-out) throughout, whose depth grows far more slowly as theta
// shrinks; all its far lists are sorted afterwards.
//
// Far ids collect in per-warp shared buffers, one for the entries summed pair
// by pair (class 0) and, with local expansions, one for the expanded entries
// (class 1).  A buffer is flushed to the global pool with one atomic
// reservation, and the flush writes a chunk record (pool position, count,
// group, class << 31 | the number of the group's entries of that class
// flushed before).  A warp's flushes take ascending pool positions, so the
// records place every chunk in its group's list with no sort: the list is the
// class-0 entries, then the class-1 ones, each in the order of the walk.  At
// the end the warp writes its group's two counts.  Past a pool's capacity
// nothing is written but the counters still count, so that the caller can
// size the pools exactly and run the traversal again.
constexpr int kTravBuf = 128;

__device__ __forceinline__ void trav_flush_far(const int* buf, int cnt, int* pool, int64_t cap,
                                               unsigned long long* counter, int4* chunks, int64_t chunk_cap,
                                               unsigned long long* chunk_counter, int g, int cls, int prefix,
                                               int lane) {
    unsigned long long base = 0, ck = 0;
    if (lane == 0) {
        base = atomicAdd(counter, (unsigned long long)cnt);
        ck = atomicAdd(chunk_counter, 1ull);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    ck = __shfl_sync(0xffffffffu, ck, 0);
    if ((int64_t)(base + cnt) <= cap && (int64_t)ck < chunk_cap) {
        for (int k = lane; k < cnt; k += 32) pool[base + k] = buf[k];
        if (lane == 0) chunks[ck] = make_int4((int)base, cnt, g, (cls << 31) | prefix);
    }
    __syncwarp();
}

__device__ __forceinline__ void trav_flush_near(const uint64_t* buf, const uint32_t* vbuf, int cnt, uint64_t* pool,
                                                uint32_t* vpool, int64_t cap, unsigned long long* counter,
                                                int4* chunks, int64_t chunk_cap, unsigned long long* chunk_counter,
                                                int g, int prefix, int lane) {
    unsigned long long base = 0, ck = 0;
    if (lane == 0) {
        base = atomicAdd(counter, (unsigned long long)cnt);
        ck = atomicAdd(chunk_counter, 1ull);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    ck = __shfl_sync(0xffffffffu, ck, 0);
    if ((int64_t)(base + cnt) <= cap) {
        for (int k = lane; k < cnt; k += 32) {
            pool[base + k] = buf[k];
            vpool[base + k] = vbuf[k];
        }
        if (lane == 0 && (int64_t)ck < chunk_cap) chunks[ck] = make_int4((int)base, cnt, g, prefix);
    }
    __syncwarp();
}

struct TravOut {
    int* far_pool;                    // far node ids, in chunks
    int64_t far_cap;
    unsigned long long* far_count;
    int4* chunks;                     // chunk records
    int64_t chunk_cap;
    unsigned long long* chunk_count;
    int2* gcount;                     // per group: class-0 and class-1 far entries
    uint64_t* near_pool;              // near keys (group << nsh | first point)
    uint32_t* near_vpool;             //   and leaf ids, in chunks
    int64_t near_cap;
    unsigned long long* near_count;
    int4* near_chunks;                // their chunk records (pool position, count, group, prefix)
    int64_t near_chunk_cap;
    unsigned long long* near_chunk_count;
    int* ncount;                      // per group: near leaves
    int nsh;
    int* err;                         // [0] error flags, [1] stack-walk groups, [2] most near leaves of a group
    uint64_t* unsorted;               // groups whose walk was finished as a stack walk
    int* unsorted_count;
};

template <int STACK, bool FIFO>
__global__ void __launch_bounds__(32 * kTravWarps)
k_traverse(const double* nlo, const double* nhi, const float4* nlof, const float4* nhif, const int* ndepth,
           const int* nchild, const int* child0, const int* nstart, const double* glo, const double* ghi, int ng,
           double theta, double clocal, TravOut out) {
    __shared__ int stack[kTravWarps][STACK];
    __shared__ int fbuf_all[kTravWarps][kTravBuf];
    __shared__ int lbuf_all[kTravWarps][kTravBuf];
    __shared__ uint64_t nbuf_all[kTravWarps][kTravBuf];
    __shared__ uint32_t nvbuf_all[kTravWarps][kTravBuf];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * kTravWarps + wl;
    if (g >= ng) return;
    const unsigned lt = (1u << lane) - 1u;
    double bl[3], bh[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) { bl[k] = glo[3 * g + k]; bh[k] = ghi[3 * g + k]; }
    const double c = 1.0 / theta;
    const float cf = (float)c;
    const float4 gl = make_float4(__double2float_rd(bl[0]), __double2float_rd(bl[1]), __double2float_rd(bl[2]), 0.f);
    const float4 gh = make_float4(__double2float_ru(bh[0]), __double2float_ru(bh[1]), __double2float_ru(bh[2]), 0.f);
    const float gs = fmaxf(fmaxf(fmaxf(fabsf(gl.x), fabsf(gl.y)), fmaxf(fabsf(gl.z), fabsf(gh.x))),
                           fmaxf(fabsf(gh.y), fabsf(gh.z)));
    const float mscale = 1e-6f * (1.f + fmaxf(gs, 1.f));
    // local expansions (clocal = 1/local_theta, 0 = off): a far node is expanded
    // about the group centre when its box gap exceeds clocal x the group box's
    // largest extent (class 1)
    double ext = __dsub_rn(bh[0], bl[0]);
    if (__dsub_rn(bh[1], bl[1]) > ext) ext = __dsub_rn(bh[1], bl[1]);
    if (__dsub_rn(bh[2], bl[2]) > ext) ext = __dsub_rn(bh[2], bl[2]);
    const double cle = __dmul_rn(clocal, ext);
    const float clef = (float)cle;
    int* st = stack[wl];
    int* fbuf = fbuf_all[wl];
    int* lbuf = lbuf_all[wl];
    uint64_t* nbuf = nbuf_all[wl];
    uint32_t* nvbuf = nvbuf_all[wl];
    static_assert((STACK & (STACK - 1)) == 0, "ring size must be a power of two");
    if (lane == 0) st[0] = 0;
    __syncwarp();
    // live entries are [head, head + top) modulo STACK; pushes append at the
    // end; first-in first-out pops from head, the stack walk from the end
    int head = 0, top = 1, fcnt = 0, lcnt = 0, ncnt = 0, fdone = 0, ldone = 0, ndone = 0;
    bool fifo = FIFO;
    while (top > 0) {
        if (fifo && top > STACK - 256) {
            fifo = false;
            if (lane == 0) out.unsorted[atomicAdd(out.unsorted_count, 1)] = (uint64_t)g;
        }
        int take = min(top, 32);
        int b = -1;
        if (lane < take) b = st[(head + (fifo ? 0 : top - take) + lane) & (STACK - 1)];
        top -= take;
        if (fifo) head += take;
        __syncwarp();
        bool far = false, leaf = false, open = false, loc = false;
        if (b >= 0) {
            const float d2f = gap2_f(nlof[b], nhif[b], gl, gh);
            const int q = far_pretest(d2f, cf * ldexpf(2.f, -ndepth[b]), mscale);
            far = q < 0 ? is_far(nlo, nhi, ndepth, b, bl, bh, c) : q == 1;
            if (far && clocal > 0.0) {
                const int ql = far_pretest(d2f, clef, mscale);
                loc = ql < 0 ? is_local(nlo, nhi, b, bl, bh, cle) : ql == 1;
            }
            if (!far) {
                if (nchild[b] == 0) leaf = true; else open = true;
            }
        }
        const unsigned fm = __ballot_sync(0xffffffffu, far && !loc), xm = __ballot_sync(0xffffffffu, loc);
        const unsigned lm = __ballot_sync(0xffffffffu, leaf);
        if (fcnt + 32 > kTravBuf) {
            trav_flush_far(fbuf, fcnt, out.far_pool, out.far_cap, out.far_count, out.chunks, out.chunk_cap,
                           out.chunk_count, g, 0, fdone, lane);
            fdone += fcnt;
            fcnt = 0;
        }
        if (lcnt + 32 > kTravBuf) {
            trav_flush_far(lbuf, lcnt, out.far_pool, out.far_cap, out.far_count, out.chunks, out.chunk_cap,
                           out.chunk_count, g, 1, ldone, lane);
            ldone += lcnt;
            lcnt = 0;
        }
        if (ncnt + 32 > kTravBuf) {
            trav_flush_near(nbuf, nvbuf, ncnt, out.near_pool, out.near_vpool, out.near_cap, out.near_count,
                            out.near_chunks, out.near_chunk_cap, out.near_chunk_count, g, ndone, lane);
            ndone += ncnt;
            ncnt = 0;
        }
        if (far && !loc) fbuf[fcnt + __popc(fm & lt)] = b;
        if (loc) lbuf[lcnt + __popc(xm & lt)] = b;
        if (leaf) {
            const int p = ncnt + __popc(lm & lt);
            nbuf[p] = ((uint64_t)g << out.nsh) | (uint32_t)nstart[b];
            nvbuf[p] = (uint32_t)b;
        }
        fcnt += __popc(fm);
        lcnt += __popc(xm);
        ncnt += __popc(lm);
        int nc = open ? nchild[b] : 0;
        int inc = nc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        int total = __shfl_sync(0xffffffffu, inc, 31);
        if (top + total > STACK) {
            if (lane == 0) atomicOr(out.err, kErrCapacity);
            break;
        }
        if (open) {
            int c0 = child0[b], p = head + top + inc - nc;
            for (int q = 0; q < nc; ++q) st[(p + q) & (STACK - 1)] = c0 + q;
        }
        top += total;
        __syncwarp();
    }
    __syncwarp();
    if (fcnt)
        trav_flush_far(fbuf, fcnt, out.far_pool, out.far_cap, out.far_count, out.chunks, out.chunk_cap,
                       out.chunk_count, g, 0, fdone, lane);
    if (lcnt)
        trav_flush_far(lbuf, lcnt, out.far_pool, out.far_cap, out.far_count, out.chunks, out.chunk_cap,
                       out.chunk_count, g, 1, ldone, lane);
    if (ncnt)
        trav_flush_near(nbuf, nvbuf, ncnt, out.near_pool, out.near_vpool, out.near_cap, out.near_count,
                        out.near_chunks, out.near_chunk_cap, out.near_chunk_count, g, ndone, lane);
    if (lane == 0) {
        out.gcount[g] = make_int2(fdone + fcnt, ldone + lcnt);
        out.ncount[g] = ndone + ncnt;
        atomicMax(out.err + 2, ndone + ncnt);
    }
}

// Far list offsets from the per-group counts: tot[g] = class 0 + class 1.
__global__ void k_gcount_tot(const int2* gcount, int ng, int* tot) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ng) tot[g] = gcount[g].x + gcount[g].y;
}

// Each chunk of the pool to its place in its group's list (warp per chunk);
// with local expansions also lsplit[g] = the start of the group's class-1 part.
__global__ void k_far_place(const int4* chunks, int64_t nchunks, const int* pool, const int* far_off,
                            const int2* gcount, int* far_id) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= nchunks) return;
    const int4 c = chunks[k];
    const int cls = (unsigned)c.w >> 31, prefix = c.w & 0x7fffffff;
    const int dst = far_off[c.z] + (cls ? gcount[c.z].x : 0) + prefix;
    for (int i = lane; i < c.y; i += 32) far_id[dst + i] = pool[c.x + i];
}
// Each near chunk of the pool to its place in its group's list (warp per
// chunk), in the walk's order.
__global__ void k_near_place(const int4* chunks, int64_t nchunks, const uint64_t* pool, const uint32_t* vpool,
                             const int* off, uint64_t* keys, uint32_t* vals) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= nchunks) return;
    const int4 c = chunks[k];
    const int dst = off[c.z] + c.w;
    for (int i = lane; i < c.y; i += 32) {
        keys[dst + i] = pool[c.x + i];
        vals[dst + i] = vpool[c.x + i];
    }
}

// Each group's near list sorted by first point in shared memory, one block
// per group: (first point << 32 | leaf) keys, padded to a power of two, by a
// bitonic network (first points are distinct within a group).  Lists longer
// than kNearSortCap are left to the caller, which then sorts all near keys.
constexpr int kNearSortCap = 2048;
constexpr int kNearSortThreads = 256;
__global__ void __launch_bounds__(kNearSortThreads) k_near_group_sort(const int* off, int nsh, uint64_t* keys,
                                                                      uint32_t* vals) {
    __shared__ uint64_t sk[kNearSortCap];
    const int g = blockIdx.x, t = threadIdx.x;
    const int e0 = off[g], n = off[g + 1] - e0;
    if (n <= 1 || n > kNearSortCap) return;
    int P = 2;
    while (P < n) P <<= 1;
    const uint64_t low = (uint64_t(1) << nsh) - 1;
    for (int i = t; i < P; i += kNearSortThreads)
        sk[i] = i < n ? ((keys[e0 + i] & low) << 32) | vals[e0 + i] : ~0ull;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = t; i < P; i += kNearSortThreads) {
                const int ij = i ^ j;
                if (ij > i) {
                    const uint64_t a = sk[i], b = sk[ij];
                    if ((a > b) == ((i & k) == 0)) {
                        sk[i] = b;
                        sk[ij] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    const uint64_t hi = (uint64_t)g << nsh;
    for (int i = t; i < n; i += kNearSortThreads) {
        keys[e0 + i] = hi | (sk[i] >> 32);
        vals[e0 + i] = (uint32_t)(sk[i] & 0xffffffffu);
    }
}

__global__ void k_lsplit_from_counts(const int* far_off, const int2* gcount, int ng, int* lsplit) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ng) lsplit[g] = far_off[g] + gcount[g].x;
}


// theta = 0: every leaf is near for every group (one merged range [0, n),
// cut into pieces later).
__global__ void k_all_near(int ng, int n, int* near_off, int2* rng) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g > ng) return;
    near_off[g] = g;
    if (g < ng) rng[g] = make_int2(0, n);
}

__global__ void k_set_i32(int* p, int v) { *p = v; }

__global__ void k_gather_tot3(const int* a, const int* b, const int* c, int* out) {
    if (threadIdx.x == 0) {
        out[0] = *a;
        out[1] = *b;
        out[2] = *c;
    }
}

// Classes of the node moments (see build_tree): flags per node in four
// arrays of nn + 1 (the exclusive sums put the totals in the last entry):
// warp class (mid), top, front, leaf.
__global__ void k_mom_flags(const int* nchild, const int* count, const int* parent, int nn, int* fl) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nn) return;
    const int64_t st = (int64_t)nn + 1;
    const int cnt = count[b], nc = nchild[b], p = parent[b];
    const bool top = cnt > kMomDirect && nc > 0;
    const bool ptop = p >= 0 && count[p] > kMomDirect;   // a parent always has children
    fl[b] = !top && cnt > kMomSmall;
    fl[st + b] = top;
    fl[2 * st + b] = !top && ptop;
    fl[3 * st + b] = nc == 0;
}

__global__ void k_mom_totals(const int* fl, int nn, int* tot) {
    const int c = threadIdx.x;
    if (c < 4) tot[c] = fl[c * ((int64_t)nn + 1) + nn];
}

// The lists from the exclusive sums of the flags (a node is in a list where
// its offset differs from the next one); front keys = (first point, node).
__global__ void k_mom_lists(const int* off, int nn, const int* start, int* mid, int* top, uint64_t* fkeys) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nn) return;
    const int64_t st = (int64_t)nn + 1;
    if (off[b + 1] != off[b]) mid[off[b]] = b;
    if (off[st + b + 1] != off[st + b]) top[off[st + b]] = b;
    if (off[2 * st + b + 1] != off[2 * st + b])
        fkeys[off[2 * st + b]] = ((uint64_t)(uint32_t)start[b] << 32) | (uint32_t)b;
}

// Per top node: the range of the (sorted) front that covers its points.
__global__ void k_mom_top_ranges(const int* top, int ntop, const int* start, const int* count,
                                 const uint64_t* fkeys, int nfront, int2* rng) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ntop) return;
    const int b = top[k];
    auto lower = [&](uint32_t v) {
        int lo = 0, hi = nfront;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((uint32_t)(fkeys[mid] >> 32) < v) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    rng[k] = make_int2(lower((uint32_t)start[b]), lower((uint32_t)(start[b] + count[b])));
}

__global__ void k_low32(const uint64_t* keys, int64_t n, int* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)(uint32_t)(keys[i] & 0xffffffffu);
}

// Near leaves (sorted by group, then first point) -> merged ranges.
// head[e] = 1 where entry e starts a range (first of its group, or not
// contiguous with the previous leaf).
__global__ void k_near_heads(const uint64_t* keys, const uint32_t* leaf, int64_t n, int nsh,
                             const int* ncount, int* head) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const uint64_t low = (uint64_t(1) << nsh) - 1;
    int h = 1;
    if (e > 0 && (keys[e] >> nsh) == (keys[e - 1] >> nsh)) {
        uint32_t prev = leaf[e - 1];
        int prev_end = (int)(keys[e - 1] & low) + ncount[prev];
        if (prev_end == (int)(keys[e] & low)) h = 0;
    }
    head[e] = h;
}

// hscan = exclusive scan of head over n+1 entries (head[n] = 1 sentinel).
// Entry e belongs to range hscan[e+1]-1; it starts it if head[e], and ends
// it if head[e+1].
__global__ void k_near_ranges(const uint64_t* keys, const uint32_t* leaf, int64_t n, int nsh,
                              const int* ncount, const int* hscan, int2* rng) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int r = hscan[e + 1] - 1;
    int s = (int)(keys[e] & ((uint64_t(1) << nsh) - 1));
    if (hscan[e + 1] != hscan[e]) rng[r].x = s;
    if (hscan[e + 2] - hscan[e + 1] == 1) rng[r].y = s + ncount[leaf[e]];
}

// Cut ranges longer than kMaxRange into pieces.
__global__ void k_cap_count(const int2* rng, int64_t nr, int* cnt) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nr) cnt[q] = (rng[q].y - rng[q].x + kMaxRange - 1) / kMaxRange;
}
__global__ void k_cap_write(const int2* rng, int64_t nr, const int* off, int2* out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr) return;
    int2 r = rng[q];
    int p = off[q];
    for (int s = r.x; s < r.y; s += kMaxRange) out[p++] = make_int2(s, min(s + kMaxRange, r.y));
}

__global__ void k_gather_i32(const int* src, const int* idx, int n, int* dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// Interaction counts: far pairs = sum_g |g| * (far entries summed pair by
// pair), near = sum_g |g| * sum |range|, the expanded entries and the pairs
// they stand for.
__global__ void k_pair_counts(int ng, const int* goff, const int* far_off, const int* lsplit, const int* csplit,
                              int K, const int* near_off, const int2* rng, unsigned long long* out) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    int64_t sz = goff[g + 1] - goff[g];
    const int fl = lsplit ? lsplit[g] : far_off[g + 1];
    const int fc = csplit ? csplit[g] : far_off[g + 1];
    int64_t nf = fl - far_off[g], nl = fc - fl;
    int64_t nn = 0;
    for (int q = near_off[g]; q < near_off[g + 1]; ++q) nn += rng[q].y - rng[q].x;
    atomicAdd(&out[0], (unsigned long long)(sz * nf));
    atomicAdd(&out[1], (unsigned long long)(sz * nn));
    if (nl) {
        atomicAdd(&out[2], (unsigned long long)nl);
        atomicAdd(&out[3], (unsigned long long)(sz * nl));
    }
    if (csplit && g % K == 0 && far_off[g + 1] > fc) {
        // a cluster's (cluster, node) expansions, counted at its first member
        const int64_t nce = far_off[g + 1] - fc;
        const int64_t csz = goff[min(g + K, ng)] - goff[g];
        atomicAdd(&out[4], (unsigned long long)nce);
        atomicAdd(&out[5], (unsigned long long)(csz * nce));
    }
}

// Clusters of K consecutive target groups (local_cluster = K): warp per
// cluster.  The FP64 box (union of the members' boxes), its largest extent
// times clocal (cle), a dyadic frame origin and, in that frame, the box
// centre and the largest distance of the cluster's targets from it (FP64,
// rounded up).
__global__ void k_cluster_frames(const double* ys, const int* goff, const double* glo, const double* ghi, int ng,
                                 int K, double clocal, double* clo, double* chi, double* cle, float4* cctr,
                                 float4* cexp) {
    const int C = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nc = (ng + K - 1) / K;
    if (C >= nc) return;
    const int g0 = C * K, g1 = min(g0 + K, ng);
    double lo[3], hi[3], c[3], o[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double l = INFINITY, h = -INFINITY;
        if (g0 + lane < g1) { l = glo[3 * (g0 + lane) + k]; h = ghi[3 * (g0 + lane) + k]; }
        warp_minmax_d(l, h);
        lo[k] = l;
        hi[k] = h;
        c[k] = 0.5 * (l + h);
        o[k] = dyadic12(c[k]);
    }
    // the largest distance from the centre: the square root of the largest
    // square (sqrt is monotone and correctly rounded; squares compare as their
    // bit patterns)
    long long r2k = 0;
    for (int i = goff[g0] + lane; i < goff[g1]; i += 32) {
        const double dx = ys[3 * (int64_t)i] - c[0], dy = ys[3 * (int64_t)i + 1] - c[1], dz = ys[3 * (int64_t)i + 2] - c[2];
        r2k = max(r2k, __double_as_longlong(dx * dx + dy * dy + dz * dz));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) r2k = max(r2k, __shfl_xor_sync(0xffffffffu, r2k, d));
    const double r = sqrt(__longlong_as_double(r2k));
    if (lane == 0) {
        double e = __dsub_rn(hi[0], lo[0]);
        if (__dsub_rn(hi[1], lo[1]) > e) e = __dsub_rn(hi[1], lo[1]);
        if (__dsub_rn(hi[2], lo[2]) > e) e = __dsub_rn(hi[2], lo[2]);
        for (int k = 0; k < 3; ++k) { clo[3 * C + k] = lo[k]; chi[3 * C + k] = hi[k]; }
        cle[C] = __dmul_rn(clocal, e);
        cctr[C] = make_float4((float)o[0], (float)o[1], (float)o[2], 0.f);
        cexp[C] = make_float4((float)(c[0] - o[0]), (float)(c[1] - o[1]), (float)(c[2] - o[2]), __double2float_ru(r));
    }
}

// Warp per cluster of at least two groups: the entries of the first member's
// expanded part whose node is local for the cluster's box (the exact FP64
// test of the group's: squared box gap > cle^2) and also lies in every other
// member's expanded part (each ascending: binary search) are flagged in every
// member.
__global__ void k_cluster_classes(const int* far_off, const int* lsplit, const int* far_id, int ng, int K,
                                  const double* nlo, const double* nhi, const float4* nlof, const float4* nhif,
                                  const double* clo, const double* chi, const double* cle, unsigned char* moved) {
    const int C = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nc = (ng + K - 1) / K;
    if (C >= nc) return;
    const int g0 = C * K, g1 = min(g0 + K, ng);
    if (g1 - g0 < 2) return;
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) { lo[k] = clo[3 * C + k]; hi[k] = chi[3 * C + k]; }
    const double c2 = __dmul_rn(cle[C], cle[C]);
    // the traversal's FP32 pre-test on outward-rounded boxes; the exact FP64
    // test only within its margin of the threshold
    const float4 cl = make_float4(__double2float_rd(lo[0]), __double2float_rd(lo[1]), __double2float_rd(lo[2]), 0.f);
    const float4 ch = make_float4(__double2float_ru(hi[0]), __double2float_ru(hi[1]), __double2float_ru(hi[2]), 0.f);
    const float cs = fmaxf(fmaxf(fmaxf(fabsf(cl.x), fabsf(cl.y)), fmaxf(fabsf(cl.z), fabsf(ch.x))),
                           fmaxf(fabsf(ch.y), fabsf(ch.z)));
    const float mscale = 1e-6f * (1.f + fmaxf(cs, 1.f));
    const float clef = (float)cle[C];
    for (int e = lsplit[g0] + lane; e < far_off[g0 + 1]; e += 32) {
        const int b = far_id[e];
        const int q = far_pretest(gap2_f(nlof[b], nhif[b], cl, ch), clef, mscale);
        if (q == 0 || (q < 0 && !(box_gap2_d(nlo, nhi, b, lo, hi) > c2))) continue;
        int qm[kMaxCluster];
        bool all = true;
        for (int m = 1; m < g1 - g0 && all; ++m) {
            int a = lsplit[g0 + m], z = far_off[g0 + m + 1];    // search [a, z)
            while (a < z) {
                const int mid = (a + z) >> 1;
                if (far_id[mid] < b) a = mid + 1; else z = mid;
            }
            if (a < far_off[g0 + m + 1] && far_id[a] == b) qm[m] = a;
            else all = false;
        }
        if (!all) continue;
        moved[e] = 1;
        for (int m = 1; m < g1 - g0; ++m) moved[qm[m]] = 1;
    }
}

// Warp per group: its expanded part [lsplit, end) reordered stably into the
// entries not flagged, then the flagged ones (from csplit on), into out; the
// rest of the list copied.
__global__ void k_cluster_partition(const int* far_off, const int* lsplit, const int* far_id,
                                    const unsigned char* moved, int ng, int* out, int* csplit) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= ng) return;
    const unsigned lt = (1u << lane) - 1u;
    const int f0 = far_off[g], l0 = lsplit[g], f1 = far_off[g + 1];
    for (int e = f0 + lane; e < l0; e += 32) out[e] = far_id[e];
    int nstay = 0;
    for (int e = l0; e < f1; e += 32) {
        const bool v = e + lane < f1 && !moved[e + lane];
        nstay += __popc(__ballot_sync(0xffffffffu, v));
    }
    int ps = l0, pm = l0 + nstay;
    for (int base = l0; base < f1; base += 32) {
        const int e = base + lane;
        const bool v = e < f1;
        const bool mv = v && moved[e];
        const unsigned bs = __ballot_sync(0xffffffffu, v && !mv), bm = __ballot_sync(0xffffffffu, mv);
        if (v && !mv) out[ps + __popc(bs & lt)] = far_id[e];
        if (mv) out[pm + __popc(bm & lt)] = far_id[e];
        ps += __popc(bs);
        pm += __popc(bm);
    }
    if (lane == 0) csplit[g] = l0 + nstay;
}

// Transposed far lists: one key per far entry, (node << 32 | the entry's
// value in the transposed list), written by one warp per group.  The value is
// the entry index; with local expansions class << 30 | id: class 0 for an
// entry summed pair by pair (id = the entry), 1 for one expanded about its
// group (from lsplit on; id = the group), 2 for one expanded about its cluster
// (from csplit on; id = the cluster), kept only in the first member's copy
// (the other members' copies get node = nnodes and sort past every node).  A
// stable sort on the node and class bits then leaves each node's values by
// class, each class in entry order.
__global__ void k_tfar_keys(const int* far_off, const int* far_id, int ng, const int* lsplit, const int* csplit,
                            int K, int nnodes, uint64_t* keys) {
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= ng) return;
    const int f0 = far_off[g], f1 = far_off[g + 1];
    const int l0 = lsplit ? lsplit[g] : f1, c0 = csplit ? csplit[g] : f1;
    for (int e = f0 + lane; e < f1; e += 32) {
        uint32_t node = (uint32_t)far_id[e];
        uint32_t v = (uint32_t)e;
        if (e >= c0) {   // only with clusters (K >= 2)
            v = (2u << 30) | (uint32_t)(g / K);
            if (g % K != 0) node = (uint32_t)nnodes;
        } else if (e >= l0) {
            v = (1u << 30) | (uint32_t)g;
        }
        keys[e] = ((uint64_t)node << 32) | v;
    }
}

// Sorted transposed keys -> tfar_ent (the low words, dropped copies
// excluded) and the offsets of every node's run.
__global__ void k_tfar_finish(const uint64_t* keys, int64_t n, int nnodes, int* tfar_ent, int* off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = keys[i];
    const int64_t b = (int64_t)(k >> 32);
    if (b < nnodes) tfar_ent[i] = (int)(uint32_t)(k & 0xffffffffu);
    const int64_t bp = i > 0 ? (int64_t)(keys[i - 1] >> 32) : -1;
    for (int64_t q = bp + 1; q <= b && q <= nnodes; ++q) off[q] = (int)i;
    if (i == n - 1)
        for (int64_t q = b + 1; q <= nnodes; ++q) off[q] = (int)n;
}

__global__ void k_tnear_count(const int2* rng, int64_t nr, int* cnt) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr) return;
    int2 r = rng[q];
    cnt[q] = r.y > r.x ? (r.y - 1) / kAdjChunk - r.x / kAdjChunk + 1 : 0;
}

__global__ void k_range_len(const int2* rng, int64_t nr, int* len) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nr) len[q] = rng[q].y - rng[q].x;
}

// One thread per near range; its group is found by binary search in near_off.
// Each entry also records the near slot of its first point and its index
// (the sort's value).
__global__ void k_tnear_fill(const int2* rng, int64_t nr, const int* near_off, int ng, const int* cnt_off,
                             const int* rng_slot, uint64_t* keys, uint32_t* masks, int* slots,
                             uint32_t* idx) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr) return;
    int lo_g = 0, hi_g = ng - 1;   // the last group g with near_off[g] <= q
    while (lo_g < hi_g) {
        const int mid = (lo_g + hi_g + 1) >> 1;
        if (near_off[mid] <= q) lo_g = mid; else hi_g = mid - 1;
    }
    const int g = lo_g;
    const int2 r = rng[q];
    if (r.y <= r.x) return;
    int p = cnt_off[q];
    for (int sc = r.x / kAdjChunk; sc <= (r.y - 1) / kAdjChunk; ++sc, ++p) {
        int lo = max(r.x, sc * kAdjChunk) - sc * kAdjChunk, hi = min(r.y, (sc + 1) * kAdjChunk) - sc * kAdjChunk;
        uint32_t m = ((1u << hi) - 1u) & ~((1u << lo) - 1u);
        keys[p] = ((uint64_t)(uint32_t)sc << 32) | (uint32_t)g;
        masks[p] = m;
        slots[p] = rng_slot[q] + (sc * kAdjChunk + lo - r.x);
        idx[p] = (uint32_t)p;
    }
}

__global__ void k_key_heads(const uint64_t* keys, int64_t n, int* head) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) head[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1 : 0;
}

// Equal (source chunk, target group) keys: OR their masks into one entry.
// They come from ranges of one group that share the chunk, in range order
// (the sort is stable), so the first one's slot is the slot of the chunk's
// first point in the group's near lists, and the chunk's points in those
// lists hold consecutive slots.
__global__ void k_tnear_merge(const uint64_t* keys, const uint32_t* idx, const uint32_t* masks,
                              const int* slots, int64_t n, const int* head_scan, int2* ent, uint64_t* ukeys) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    if (e > 0 && keys[e] == keys[e - 1]) return;
    uint32_t m = 0;
    for (int64_t f = e; f < n && keys[f] == keys[e]; ++f) m |= masks[idx[f]];
    int r = head_scan[e];
    ent[r] = make_int2(slots[idx[e]], (int)m);
    ukeys[r] = keys[e];
}

// ---------------------------------------------------------------------------
// Work lists: each segment's lists (near units, then far entries in blocks of
// 32) are cut greedily into items of about `cap` lane-slots.
//   mode 0: near units are ranges costing their length (gather kernels)
//   mode 1: near units are transposed entries costing 8 each (adjoint near:
//           a quarter of a target group per lane)
//   mode 2: far entries only (adjoint far)
// ---------------------------------------------------------------------------
// Work items of segment g: its units in order (near ranges, then the
// pair-by-pair far entries in chunks of 32), cut greedily: a unit that would
// take a non-empty item past the cap starts a new item.  One warp per
// segment: the lanes take 32 consecutive units at a time, an inclusive prefix
// sum of their costs gives each unit's cost within the current item, and the
// cuts follow one at a time by ballot (the first unit past the cap after the
// last cut), so the items are those of the walk unit by unit.  Far entries
// expanded about the group centre (from lsplit[g] on) are not in the items:
// the local-expansion kernels take them.  Returns the number of items; with
// out set, lane 0 writes them.
__device__ int walk_items(int mode, int g, const int* near_off, const int2* rng, const int* far_off,
                          const int* lsplit, int cap, Item* out, int base, int pslot_base, int nparts, int split,
                          bool partials, int lane) {
    const int qb = near_off ? near_off[g] : 0, qe = near_off ? near_off[g + 1] : 0;
    const int fb = far_off ? far_off[g] : 0;
    const int fe = far_off ? (lsplit ? min(max(lsplit[g], fb), far_off[g + 1]) : far_off[g + 1]) : 0;
    const int nq = qe - qb, nu = nq + (fe - fb + 31) / 32;
    // unit u starts at near range q_at(u) and far entry f_at(u)
    auto q_at = [&](int u) { return u < nq ? qb + u : qe; };
    auto f_at = [&](int u) { return u < nq ? fb : fb + 32 * (u - nq); };
    int k = 0, u_start = 0, carry = 0;    // items so far; the current item's first unit and cost before the batch
    auto emit = [&](int u_end, int cost) {
        if (out && lane == 0) {
            Item it;
            it.g = g;
            it.q0 = q_at(u_start);
            it.q1 = u_end < nu ? q_at(u_end) : qe;
            it.f0 = f_at(u_start);
            it.f1 = u_end < nu ? f_at(u_end) : fe;
            it.pslot = (partials && nparts > 1) ? pslot_base + k : -1;
            it.cost = cost;
            it.split = it.pslot >= 0 ? split : -1;
            out[base + k] = it;
        }
        ++k;
        u_start = u_end;
    };
    for (int u0 = 0; u0 < nu; u0 += 32) {
        const int u = u0 + lane;
        int c = 0;
        if (u < nu) c = u < nq ? (mode == 1 ? 8 : rng[qb + u].y - rng[qb + u].x) : min(32, fe - f_at(u));
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int excl = incl - c;
        int s = 0, ex_s = 0;      // first pending lane of the batch and its exclusive prefix
        for (;;) {
            const int cur = carry + excl - ex_s;      // the item's cost before this unit
            const unsigned cut = __ballot_sync(0xffffffffu, u < nu && lane >= s && cur > 0 && cur + c > cap);
            if (!cut) break;
            const int j = __ffs(cut) - 1;
            emit(u0 + j, __shfl_sync(0xffffffffu, cur, j));
            ex_s = __shfl_sync(0xffffffffu, excl, j);
            s = j;
            carry = 0;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        carry += tot - ex_s;
    }
    if (carry > 0 || k == 0) emit(nu, carry);
    return k;
}

// Total cost of segment g (its walk without a cap); one warp per segment.
__global__ void k_seg_cost(int mode, int nseg, const int* near_off, const int2* rng, const int* far_off,
                           const int* lsplit, int64_t* cost) {
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= nseg) return;
    int64_t c = 0;
    if (near_off)
        for (int q = near_off[g] + lane; q < near_off[g + 1]; q += 32) c += mode == 1 ? 8 : rng[q].y - rng[q].x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
        if (far_off) {
            const int fb = far_off[g];
            c += (lsplit ? min(max(lsplit[g], fb), far_off[g + 1]) : far_off[g + 1]) - fb;
        }
        cost[g] = c;
    }
}

__global__ void k_items_count(int mode, int nseg, const int* near_off, const int2* rng, const int* far_off,
                              const int* lsplit, const int* capp, int* cnt, int* slots) {
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= nseg) return;
    const int c = walk_items(mode, g, near_off, rng, far_off, lsplit, *capp, nullptr, 0, 0, 0, -1, false, lane);
    if (lane == 0) {
        cnt[g] = c;
        slots[g] = c > 1 ? c : 0;
    }
}

__global__ void k_items_fill(int mode, int nseg, const int* near_off, const int2* rng, const int* far_off,
                             const int* lsplit, const int* capp, const int* cnt, const int* item_off,
                             const int* slot_off, bool partials, Item* items, int4* splits, const int* split_off) {
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= nseg) return;
    walk_items(mode, g, near_off, rng, far_off, lsplit, *capp, items, item_off[g], slot_off[g], cnt[g],
               (partials && cnt[g] > 1) ? split_off[g] : -1, partials, lane);
    if (lane == 0 && partials && cnt[g] > 1) splits[split_off[g]] = make_int4(g, slot_off[g], cnt[g], 0);
}

__global__ void k_group_splits(const int* cnt, const int* split_off, int nseg, int* gsplit) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < nseg) gsplit[g] = cnt[g] > 1 ? split_off[g] : -1;
}

__global__ void k_split_flags(const int* cnt, int nseg, int* flag) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < nseg) flag[g] = cnt[g] > 1;
}

// Heaviest first: key = (kCostKeyMax - cost) << 32 | item index; an item
// costs at most the cap plus one near unit (a range of at most kMaxRange
// points or 32 far entries), so the cost field fits kCostKeyBits bits.
constexpr int kCostKeyBits = 13;
constexpr int kCostKeyMax = (1 << kCostKeyBits) - 1;
static_assert(kItemCostMax + kMaxRange <= kCostKeyMax, "item cost key too narrow");
__global__ void k_item_keys(const Item* items, int n, uint64_t* keys) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = ((uint64_t)(uint32_t)(kCostKeyMax - min(items[i].cost, kCostKeyMax)) << 32) | (uint32_t)i;
}
__global__ void k_item_permute(const Item* in, const uint64_t* keys, int n, Item* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[(uint32_t)(keys[i] & 0xffffffffu)];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host orchestration
// ---------------------------------------------------------------------------

// Temporaries go back to the pool in the order of its stream: no wait is
// needed before pool_free when that stream is s (every build entry point
// sets it so).
static void wait_before_free(cudaStream_t s) {
    if (alloc_stream() != s) WNNC_CUDA(cudaStreamSynchronize(s));
}

// Page-locked host memory for the build's read-backs (one block per host
// thread, kept for the thread's life): copies into it are asynchronous, so
// several can share one synchronisation.
struct PinnedScratch {
    void* p = nullptr;
    ~PinnedScratch() {
        if (p) cudaFreeHost(p);
    }
};
constexpr size_t kPinnedBytes = 4096;
static char* pinned_scratch() {
    thread_local PinnedScratch ps;
    if (!ps.p) WNNC_CUDA(cudaMallocHost(&ps.p, kPinnedBytes));
    return static_cast<char*>(ps.p);
}

static int read_int(const int* dptr, cudaStream_t s) {
    int* h = reinterpret_cast<int*>(pinned_scratch());
    WNNC_CUDA(cudaMemcpyAsync(h, dptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    WNNC_CUDA(cudaStreamSynchronize(s));
    return *h;
}

static int bits_for(int64_t v) {
    int b = 0;
    while ((int64_t(1) << b) <= v) ++b;
    return b;
}

void free_work(WorkList& w) {
    dfree(w.items);
    dfree(w.splits);
    dfree(w.split_cnt);
    dfree(w.gsplit);
    w.nitems = w.nsplit = w.nslots = 0;
}

// The item cap of a work list from the total cost of its segments: about
// total / kItemsTarget, a power of two within [kItemCostMin, kItemCostMax].
__global__ void k_item_cap(const int64_t* total, int* cap) {
    int c = kItemCostMin;
    while (c < kItemCostMax && (int64_t)c * 2 * kItemsTarget <= *total) c *= 2;
    *cap = c;
}

// A work list of nseg segments (see walk_items), heaviest item first, built
// in two phases so that several lists share one read-back of their sizes:
// work_count queues the cap, the per-segment item counts and their scans, and
// leaves the list's three totals (items, partial slots, cut groups) in tot;
// work_fill, given those totals on the host, allocates and fills the list.
struct WorkBuild {
    int mode = 0, nseg = 0;
    const int* near_off = nullptr;
    const int2* rng = nullptr;
    const int* far_off = nullptr;
    const int* lsplit = nullptr;
    bool partials = false;
    int *cnt = nullptr, *slots = nullptr, *item_off = nullptr, *slot_off = nullptr, *flag = nullptr,
        *split_off = nullptr, *cap = nullptr, *tot = nullptr;
};

static void work_count(WorkBuild& b, int mode, int nseg, const int* near_off, const int2* rng, const int* far_off,
                       const int* lsplit, bool partials, cudaStream_t s) {
    b.mode = mode;
    b.nseg = nseg;
    b.near_off = near_off;
    b.rng = rng;
    b.far_off = far_off;
    b.lsplit = lsplit;
    b.partials = partials;
    b.cnt = dalloc<int>(nseg + 1);
    b.slots = dalloc<int>(nseg + 1);
    b.item_off = dalloc<int>(nseg + 2);
    b.slot_off = dalloc<int>(nseg + 2);
    b.flag = dalloc<int>(nseg + 1);
    b.split_off = dalloc<int>(nseg + 2);
    b.cap = dalloc<int>(1);
    b.tot = dalloc<int>(3);
    int64_t* seg_cost = dalloc<int64_t>(nseg + 1);
    int64_t* cost_scan = dalloc<int64_t>(nseg + 2);
    k_seg_cost<<<ceil_div((int64_t)nseg * 32, kTB), kTB, 0, s>>>(mode, nseg, near_off, rng, far_off, lsplit, seg_cost);
    WNNC_LAUNCH_CHECK();
    exclusive_scan_i64(seg_cost, cost_scan, nseg, s);
    k_item_cap<<<1, 1, 0, s>>>(cost_scan + nseg, b.cap);
    WNNC_LAUNCH_CHECK();
    k_items_count<<<ceil_div((int64_t)nseg * 32, kTB), kTB, 0, s>>>(mode, nseg, near_off, rng, far_off, lsplit,
                                                                   b.cap, b.cnt, b.slots);
    WNNC_LAUNCH_CHECK();
    exclusive_scan_i32(b.cnt, b.item_off, nseg, s);
    exclusive_scan_i32(b.slots, b.slot_off, nseg, s);
    k_split_flags<<<ceil_div(nseg, kTB), kTB, 0, s>>>(b.cnt, nseg, b.flag);
    WNNC_LAUNCH_CHECK();
    exclusive_scan_i32(b.flag, b.split_off, nseg, s);
    k_gather_tot3<<<1, 32, 0, s>>>(b.item_off + nseg, b.slot_off + nseg, b.split_off + nseg, b.tot);
    WNNC_LAUNCH_CHECK();
    pool_free(seg_cost);
    pool_free(cost_scan);
}

static void work_fill(WorkList& w, WorkBuild& b, const int* htot, cudaStream_t s) {
    const int nseg = b.nseg;
    w.nitems = htot[0];
    w.nslots = b.partials ? htot[1] : 0;
    w.nsplit = b.partials ? htot[2] : 0;
    Item* tmp = dalloc<Item>(w.nitems);
    w.splits = dalloc<int4>(w.nsplit);
    w.split_cnt = dalloc<unsigned>(w.nsplit);
    if (b.partials) {
        w.gsplit = dalloc<int>(nseg);
        k_group_splits<<<ceil_div(nseg, kTB), kTB, 0, s>>>(b.cnt, b.split_off, nseg, w.gsplit);
        WNNC_LAUNCH_CHECK();
    }
    WNNC_CUDA(cudaMemsetAsync(w.split_cnt, 0, sizeof(unsigned) * (size_t)std::max(w.nsplit, 1), s));
    k_items_fill<<<ceil_div((int64_t)nseg * 32, kTB), kTB, 0, s>>>(b.mode, nseg, b.near_off, b.rng, b.far_off,
                                                                  b.lsplit, b.cap, b.cnt, b.item_off, b.slot_off,
                                                                  b.partials, tmp, w.splits, b.split_off);
    WNNC_LAUNCH_CHECK();
    uint64_t* keys = dalloc<uint64_t>(w.nitems);
    k_item_keys<<<ceil_div(w.nitems, kTB), kTB, 0, s>>>(tmp, w.nitems, keys);
    WNNC_LAUNCH_CHECK();
    radix_sort_pairs(keys, nullptr, w.nitems, 32 + kCostKeyBits, s, 32);   // indices already ascending
    w.items = dalloc<Item>(w.nitems);
    k_item_permute<<<ceil_div(w.nitems, kTB), kTB, 0, s>>>(tmp, keys, w.nitems, w.items);
    WNNC_LAUNCH_CHECK();
    wait_before_free(s);
    pool_free(b.cnt); pool_free(b.slots); pool_free(b.item_off); pool_free(b.slot_off); pool_free(b.flag);
    pool_free(b.split_off); pool_free(b.cap); pool_free(b.tot); pool_free(tmp); pool_free(keys);
    b = WorkBuild();
}

// Far lists of the groups that a first-in first-out walk finished as stack
// walks (or of every group after stack walks throughout): each class part of
// such a list is sorted by node.  The parts are copied one after another with
// compact keys (k << nbits | node), k = 2 x the group's place in `groups` +
// the class, sorted, and written back into their own places.
__device__ __forceinline__ void far_part(const int* far_off, const int* lsplit, int g, int cls, int& e0, int& e1) {
    const int mid = lsplit ? lsplit[g] : far_off[g + 1];
    e0 = cls ? mid : far_off[g];
    e1 = cls ? far_off[g + 1] : mid;
}
__global__ void k_seg_sizes(const uint64_t* groups, int nu, const int* far_off, const int* lsplit, int* sz) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * nu) return;
    int e0, e1;
    far_part(far_off, lsplit, (int)groups[k >> 1], k & 1, e0, e1);
    sz[k] = e1 - e0;
}
__global__ void k_seg_pack(const int* far_id, const uint64_t* groups, const int* far_off, const int* lsplit,
                           const int* pos, int nbits, uint64_t* tmp) {
    const int k = blockIdx.x;
    int e0, e1;
    far_part(far_off, lsplit, (int)groups[k >> 1], k & 1, e0, e1);
    const int p0 = pos[k];
    for (int i = threadIdx.x; i < e1 - e0; i += blockDim.x)
        tmp[p0 + i] = ((uint64_t)k << nbits) | (uint32_t)far_id[e0 + i];
}
__global__ void k_seg_unpack(const uint64_t* tmp, const uint64_t* groups, const int* far_off, const int* lsplit,
                             const int* pos, int nbits, int* far_id) {
    const int k = blockIdx.x;
    int e0, e1;
    far_part(far_off, lsplit, (int)groups[k >> 1], k & 1, e0, e1);
    const int p0 = pos[k];
    const uint64_t low = (uint64_t(1) << nbits) - 1;
    for (int i = threadIdx.x; i < e1 - e0; i += blockDim.x) far_id[e0 + i] = (int)(tmp[p0 + i] & low);
}
__global__ void k_iota_u64(uint64_t* p, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (uint64_t)i;
}

static void sort_far_segments(int* far_id, const int* far_off, const int* lsplit, const uint64_t* groups, int nu,
                              int nbits, cudaStream_t s) {
    const int nseg = 2 * nu;
    int* sz = dalloc<int>(nseg + 1);
    int* pos = dalloc<int>(nseg + 2);
    k_seg_sizes<<<ceil_div(nseg, kTB), kTB, 0, s>>>(groups, nu, far_off, lsplit, sz);
    WNNC_LAUNCH_CHECK();
    exclusive_scan_i32(sz, pos, nseg, s);
    const int total = read_int(pos + nseg, s);
    if (total > 0) {
        uint64_t* tmp = dalloc<uint64_t>(total);
        k_seg_pack<<<nseg, 256, 0, s>>>(far_id, groups, far_off, lsplit, pos, nbits, tmp);
        WNNC_LAUNCH_CHECK();
        radix_sort_pairs(tmp, nullptr, total, nbits + bits_for(nseg), s);
        k_seg_unpack<<<nseg, 256, 0, s>>>(tmp, groups, far_off, lsplit, pos, nbits, far_id);
        WNNC_LAUNCH_CHECK();
        pool_free(tmp);
    }
    pool_free(sz);
    pool_free(pos);
}

void build_target_set(const Tree& t, TargetSet& ts, const double* yn, int64_t m, bool self,
                      cudaStream_t s, const int64_t* self_perm, const std::function<void()>& after_far) {
    ts.m = m;
    ts.nchunks = ceil_div(m, kGroup);
    // Morton order of the targets: for the tree's own points it is the
    // sources' order, already computed by the tree build
    const bool reuse = self && self_perm != nullptr;
    uint64_t* keys = nullptr;
    uint32_t* idx = nullptr;
    double* ys = nullptr;
    ts.perm = dalloc<int64_t>(m);
    if (reuse) {
        keys = t.keys;
        ys = t.xs;
        WNNC_CUDA(cudaMemcpyAsync(ts.perm, self_perm, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, s));
    } else {
        keys = dalloc<uint64_t>(m);
        idx = dalloc<uint32_t>(m);
        k_keys_from_xn<<<ceil_div(m, kTB), kTB, 0, s>>>(yn, m, keys, idx);
        WNNC_LAUNCH_CHECK();
        radix_sort_pairs(keys, idx, m, kKeyBits, s);
        ys = dalloc<double>(3 * m);
        k_gather_sorted<<<ceil_div(m, kTB), kTB, 0, s>>>(yn, idx, m, ys, ts.perm);
        WNNC_LAUNCH_CHECK();
    }
    // coordinate frames of the fixed chunks
    ts.corig = dalloc<float4>(ts.nchunks);
    ts.pos = dalloc<float4>(m);
    k_chunk_frames<<<ceil_div((int64_t)ts.nchunks * 32, kTB), kTB, 0, s>>>(ys, m, ts.nchunks, ts.corig, ts.pos);
    WNNC_LAUNCH_CHECK();
    // groups
    if (self) {
        int* cut = dalloc<int>(m + 1);
        int* cscan = dalloc<int>(m + 2);
        k_group_cuts<<<ceil_div(m, kTB), kTB, 0, s>>>(keys, t.leaf_of, t.node_depth, m, kGroupSlack,
                                                      kGroupMinDepth, cut);
        WNNC_LAUNCH_CHECK();
        exclusive_scan_i32(cut, cscan, m, s);
        int nruns = read_int(cscan + m, s);
        int* run_start = dalloc<int>(nruns);
        k_compact<<<ceil_div(m, kTB), kTB, 0, s>>>(cut, cscan, m, run_start);
        WNNC_LAUNCH_CHECK();
        int* rcnt = dalloc<int>(nruns + 1);
        int* roff = dalloc<int>(nruns + 2);
        k_run_ngroups<<<ceil_div(nruns, kTB), kTB, 0, s>>>(run_start, nruns, m, rcnt);
        WNNC_LAUNCH_CHECK();
        exclusive_scan_i32(rcnt, roff, nruns, s);
        ts.ngroups = read_int(roff + nruns, s);
        ts.goff = dalloc<int>(ts.ngroups + 1);
        k_run_goff<<<ceil_div(nruns, kTB), kTB, 0, s>>>(run_start, nruns, m, roff, ts.goff);
        WNNC_LAUNCH_CHECK();
        wait_before_free(s);
        pool_free(cut); pool_free(cscan); pool_free(run_start); pool_free(rcnt); pool_free(roff);
    } else {
        ts.ngroups = ts.nchunks;
        ts.goff = dalloc<int>(ts.ngroups + 1);
        k_fixed_goff<<<ceil_div(ts.ngroups + 1, kTB), kTB, 0, s>>>(ts.ngroups, m, ts.goff);
        WNNC_LAUNCH_CHECK();
    }
    const int ng = ts.ngroups;
    ts.glo = dalloc<double>(3 * (size_t)ng);
    ts.ghi = dalloc<double>(3 * (size_t)ng);
    ts.gorig = dalloc<float4>(ng);
    ts.gbl = dalloc<float4>(ng);
    ts.gbh = dalloc<float4>(ng);
    const bool local = t.params.local_theta > 0.f && t.params.theta > 0.f;
    const double clocal = local ? 1.0 / (double)t.params.local_theta : 0.0;
    ts.gctr = local ? dalloc<float4>(ng) : nullptr;
    k_group_boxes<<<ceil_div((int64_t)ng * 32, kTB), kTB, 0, s>>>(ys, ts.goff, ng, ts.glo, ts.ghi, ts.gorig,
                                                                   ts.gbl, ts.gbh, ts.gctr);
    WNNC_LAUNCH_CHECK();
    // clusters of the second expansion level: boxes, frames, radii (targets still in FP64)
    const int K = (local && t.params.local_cluster >= 2) ? t.params.local_cluster : 0;
    double *cl_lo = nullptr, *cl_hi = nullptr, *cl_e = nullptr;
    if (K) {
        ts.cluster_k = K;
        ts.nclusters = (ng + K - 1) / K;
        cl_lo = dalloc<double>(3 * (size_t)ts.nclusters);
        cl_hi = dalloc<double>(3 * (size_t)ts.nclusters);
        cl_e = dalloc<double>(ts.nclusters);
        ts.cctr = dalloc<float4>(ts.nclusters);
        ts.cexp = dalloc<float4>(ts.nclusters);
        k_cluster_frames<<<ceil_div((int64_t)ts.nclusters * 32, kTB), kTB, 0, s>>>(
            ys, ts.goff, ts.glo, ts.ghi, ng, K, clocal, cl_lo, cl_hi, cl_e, ts.cctr, ts.cexp);
        WNNC_LAUNCH_CHECK();
    }
    wait_before_free(s);
    if (!reuse) {
        pool_free(ys);
        pool_free(keys);
        pool_free(idx);
    }

    ts.far_off = dalloc<int>(ng + 1);
    int* near_off0 = dalloc<int>(ng + 1);     // merged (uncut) ranges
    int2* rng0 = nullptr;
    int64_t nr0 = 0;
    const double theta = (double)t.params.theta;
    if (theta <= 0.0) {
        ts.far_entries = 0;
        ts.far_id = dalloc<int>(1);
        WNNC_CUDA(cudaMemsetAsync(ts.far_off, 0, sizeof(int) * (ng + 1), s));
        rng0 = dalloc<int2>(ng);
        nr0 = ng;
        k_all_near<<<ceil_div(ng + 1, kTB), kTB, 0, s>>>(ng, (int)t.n, near_off0, rng0);
        WNNC_LAUNCH_CHECK();
        if (after_far) after_far();
    } else {
        int* leaf_off = dalloc<int>(ng + 1);
        int* err = dalloc<int>(3);        // [0] error flags, [1] groups finished as stack walks, [2] longest near list
        uint64_t* unsorted = dalloc<uint64_t>(ng);
        unsigned long long* counts = dalloc<unsigned long long>(4);   // far ids, far chunks, near entries, near chunks
        int2* gcount = dalloc<int2>(ng);
        int* ncount = dalloc<int>(ng + 1);
        const int tgrid = ceil_div(ng, kTravWarps);
        const int nsh = bits_for(t.n);    // near keys: group << nsh | first point
        // pool estimates (per target); a second pass runs with exact sizes if exceeded
        int64_t far_cap = std::min<int64_t>(48 * m + 4096, INT32_MAX), near_cap = 8 * m + 4096;
        int* fpool = nullptr;
        int4* chunks = nullptr;
        int4* nchunks = nullptr;
        uint64_t* nkeys = nullptr;
        uint32_t* nvals = nullptr;
        int64_t nfar = 0, nchunk = 0, nleafent = 0, nnchunk = 0;
        int longest_near = 0;
        // first the first-in first-out walk (far ids come out ascending within
        // each group, except in the groups it lists as unsorted); if a stack
        // walk overflows its buffer, everything again as stack walks with the
        // larger buffer, whose far lists are all sorted afterwards
        int nunsorted = 0;
        bool big_stack = false;
        for (int attempt = 0; attempt < 4; ++attempt) {
            // a flush other than a class's last holds > kTravBuf - 32 entries
            const int64_t chunk_cap = far_cap / (kTravBuf - 31) + 2 * (int64_t)ng + 64;
            const int64_t nchunk_cap = near_cap / (kTravBuf - 31) + (int64_t)ng + 64;
            fpool = dalloc<int>(far_cap);
            chunks = dalloc<int4>(chunk_cap);
            nkeys = dalloc<uint64_t>(near_cap);
            nvals = dalloc<uint32_t>(near_cap);
            nchunks = dalloc<int4>(nchunk_cap);
            WNNC_CUDA(cudaMemsetAsync(err, 0, 3 * sizeof(int), s));
            WNNC_CUDA(cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), s));
            TravOut o;
            o.far_pool = fpool;
            o.far_cap = far_cap;
            o.far_count = counts;
            o.chunks = chunks;
            o.chunk_cap = chunk_cap;
            o.chunk_count = counts + 1;
            o.gcount = gcount;
            o.near_pool = nkeys;
            o.near_vpool = nvals;
            o.near_cap = near_cap;
            o.near_count = counts + 2;
            o.near_chunks = nchunks;
            o.near_chunk_cap = nchunk_cap;
            o.near_chunk_count = counts + 3;
            o.ncount = ncount;
            o.nsh = nsh;
            o.err = err;
            o.unsorted = unsorted;
            o.unsorted_count = err + 1;
#define WNNC_TRAVERSE(STK, FIFO)                                                                               \
    k_traverse<STK, FIFO><<<tgrid, 32 * kTravWarps, 0, s>>>(t.node_lo, t.node_hi, t.node_lof, t.node_hif,           \
                                                      t.node_depth, t.node_nchild, t.node_child0,            \
                                                      t.node_start, ts.glo, ts.ghi, ng, theta, clocal, o)
            if (big_stack) WNNC_TRAVERSE(kStackBig, false); else WNNC_TRAVERSE(kStackSmall, true);
#undef WNNC_TRAVERSE
            WNNC_LAUNCH_CHECK();
            unsigned long long* hc = reinterpret_cast<unsigned long long*>(pinned_scratch());
            int* herr = reinterpret_cast<int*>(hc + 4);
            WNNC_CUDA(cudaMemcpyAsync(hc, counts, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            WNNC_CUDA(cudaMemcpyAsync(herr, err, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
            WNNC_CUDA(cudaStreamSynchronize(s));
            nunsorted = herr[1];
            longest_near = herr[2];
            if (herr[0]) {
                pool_free(fpool); pool_free(chunks); pool_free(nkeys); pool_free(nvals); pool_free(nchunks);
                if (!big_stack) {   // again with the larger stack
                    big_stack = true;
                    continue;
                }
                pool_free(leaf_off); pool_free(err); pool_free(unsorted); pool_free(counts); pool_free(gcount);
                pool_free(ncount); pool_free(near_off0);
                fail(WNNC_ECAPACITY, "interaction-list traversal stack overflow (theta too small)");
            }
            nfar = (int64_t)hc[0];
            nchunk = (int64_t)hc[1];
            nleafent = (int64_t)hc[2];
            nnchunk = (int64_t)hc[3];
            if (nfar <= far_cap && nchunk <= chunk_cap && nleafent <= near_cap && nnchunk <= nchunk_cap) break;
            pool_free(fpool); pool_free(chunks); pool_free(nkeys); pool_free(nvals); pool_free(nchunks);
            if (attempt == 3 || nfar > INT32_MAX || nleafent > INT32_MAX) {
                pool_free(leaf_off); pool_free(err); pool_free(unsorted); pool_free(counts); pool_free(gcount);
                pool_free(ncount); pool_free(near_off0);
                fail(WNNC_ECAPACITY, "interaction lists too long");
            }
            far_cap = std::max<int64_t>(nfar, 1);
            near_cap = std::max<int64_t>(nleafent, 1);
        }
        const int gbits = bits_for(ng);
        // far lists: offsets from the per-group counts, chunks to their places
        {
            int* tot = dalloc<int>(ng + 1);
            k_gcount_tot<<<ceil_div(ng, kTB), kTB, 0, s>>>(gcount, ng, tot);
            WNNC_LAUNCH_CHECK();
            exclusive_scan_i32(tot, ts.far_off, ng, s);
            wait_before_free(s);
            pool_free(tot);
        }
        ts.far_entries = nfar;
        ts.far_id = dalloc<int>(std::max<int64_t>(nfar, 1));
        if (nchunk) {
            k_far_place<<<ceil_div(nchunk * 32, kTB), kTB, 0, s>>>(chunks, nchunk, fpool, ts.far_off, gcount,
                                                                  ts.far_id);
            WNNC_LAUNCH_CHECK();
        }
        if (local) {
            ts.far_lsplit = dalloc<int>(ng);
            k_lsplit_from_counts<<<ceil_div(ng, kTB), kTB, 0, s>>>(ts.far_off, gcount, ng, ts.far_lsplit);
            WNNC_LAUNCH_CHECK();
        }
        if (big_stack) {
            k_iota_u64<<<ceil_div(ng, kTB), kTB, 0, s>>>(unsorted, ng);
            WNNC_LAUNCH_CHECK();
            nunsorted = ng;
        }
        if (nunsorted > 0 && nfar > 0)
            sort_far_segments(ts.far_id, ts.far_off, ts.far_lsplit, unsorted, nunsorted, bits_for(t.nnodes), s);
        ts.walk_stack_groups = big_stack ? 0 : nunsorted;
        ts.walk_big_stack = big_stack ? 1 : 0;
        if (K) {
            // entries expanded about their cluster: flagged, then each group's expanded
            // part reordered into [group | cluster] (csplit)
            ts.far_csplit = dalloc<int>(ng);
            unsigned char* moved = dalloc<unsigned char>(std::max<int64_t>(nfar, 1));
            WNNC_CUDA(cudaMemsetAsync(moved, 0, std::max<int64_t>(nfar, 1), s));
            k_cluster_classes<<<ceil_div((int64_t)ts.nclusters * 32, kTB), kTB, 0, s>>>(
                ts.far_off, ts.far_lsplit, ts.far_id, ng, K, t.node_lo, t.node_hi, t.node_lof, t.node_hif, cl_lo,
                cl_hi, cl_e, moved);
            WNNC_LAUNCH_CHECK();
            int* reordered = dalloc<int>(std::max<int64_t>(nfar, 1));
            k_cluster_partition<<<ceil_div((int64_t)ng * 32, kTB), kTB, 0, s>>>(
                ts.far_off, ts.far_lsplit, ts.far_id, moved, ng, reordered, ts.far_csplit);
            WNNC_LAUNCH_CHECK();
            wait_before_free(s);
            pool_free(ts.far_id);
            ts.far_id = reordered;
            pool_free(moved);
        }
        if (after_far) after_far();
        // near leaves by (group, first point): the chunks to their groups' lists and each
        // list sorted in shared memory, or, if a list is longer than that holds, a radix
        // sort of all near keys
        if (longest_near <= kNearSortCap) {
            exclusive_scan_i32(ncount, leaf_off, ng, s);
            uint64_t* pk = dalloc<uint64_t>(std::max<int64_t>(nleafent, 1));
            uint32_t* pv = dalloc<uint32_t>(std::max<int64_t>(nleafent, 1));
            if (nnchunk) {
                k_near_place<<<ceil_div(nnchunk * 32, kTB), kTB, 0, s>>>(nchunks, nnchunk, nkeys, nvals, leaf_off, pk,
                                                                        pv);
                WNNC_LAUNCH_CHECK();
            }
            k_near_group_sort<<<ng, kNearSortThreads, 0, s>>>(leaf_off, nsh, pk, pv);
            WNNC_LAUNCH_CHECK();
            pool_free(nkeys);
            pool_free(nvals);
            nkeys = pk;
            nvals = pv;
        } else {
            radix_sort_pairs(nkeys, nvals, nleafent, nsh + gbits, s);
            segment_offsets_hi32(nkeys, nleafent, leaf_off, ng, s, nsh);
        }
        // merge consecutive near leaves into ranges
        int* head = dalloc<int>(nleafent + 2);
        int* hscan = dalloc<int>(nleafent + 2);
        if (nleafent) {
            k_near_heads<<<ceil_div(nleafent, kTB), kTB, 0, s>>>(nkeys, nvals, nleafent, nsh, t.node_count, head);
            WNNC_LAUNCH_CHECK();
        }
        // sentinel head[n] = 1 so that the last entry closes its range
        k_set_i32<<<1, 1, 0, s>>>(head + nleafent, 1);
        WNNC_LAUNCH_CHECK();
        exclusive_scan_i32(head, hscan, nleafent + 1, s);
        nr0 = read_int(hscan + nleafent, s);   // heads among the real entries
        rng0 = dalloc<int2>(nr0);
        if (nleafent) {
            k_near_ranges<<<ceil_div(nleafent, kTB), kTB, 0, s>>>(nkeys, nvals, nleafent, nsh, t.node_count,
                                                                 hscan, rng0);
            WNNC_LAUNCH_CHECK();
        }
        // range offsets per group = number of heads before the group's first leaf entry
        k_gather_i32<<<ceil_div(ng + 1, kTB), kTB, 0, s>>>(hscan, leaf_off, ng + 1, near_off0);
        WNNC_LAUNCH_CHECK();
        wait_before_free(s);
        pool_free(fpool); pool_free(chunks); pool_free(nkeys); pool_free(nvals); pool_free(head); pool_free(hscan);
        pool_free(leaf_off); pool_free(err); pool_free(unsorted); pool_free(counts); pool_free(gcount);
        pool_free(nchunks); pool_free(ncount);
    }
    // cut ranges to at most kMaxRange points
    {
        int* cnt = dalloc<int>(nr0 + 1);
        int* off = dalloc<int>(nr0 + 2);
        if (nr0) {
            k_cap_count<<<ceil_div(nr0, kTB), kTB, 0, s>>>(rng0, nr0, cnt);
            WNNC_LAUNCH_CHECK();
        }
        exclusive_scan_i32(cnt, off, nr0, s);
        ts.near_ranges = read_int(off + nr0, s);
        ts.near_rng = dalloc<int2>(ts.near_ranges);
        if (nr0) {
            k_cap_write<<<ceil_div(nr0, kTB), kTB, 0, s>>>(rng0, nr0, off, ts.near_rng);
            WNNC_LAUNCH_CHECK();
        }
        ts.near_off = dalloc<int>(ng + 1);
        k_gather_i32<<<ceil_div(ng + 1, kTB), kTB, 0, s>>>(off, near_off0, ng + 1, ts.near_off);
        WNNC_LAUNCH_CHECK();
        wait_before_free(s);
        pool_free(cnt); pool_free(off); pool_free(rng0); pool_free(near_off0);
    }
    if (K) {
        wait_before_free(s);
        pool_free(cl_lo); pool_free(cl_hi); pool_free(cl_e);
    }
    unsigned long long* pc = dalloc<unsigned long long>(6);
    WNNC_CUDA(cudaMemsetAsync(pc, 0, 6 * sizeof(unsigned long long), s));
    k_pair_counts<<<ceil_div(ng, kTB), kTB, 0, s>>>(ng, ts.goff, ts.far_off, ts.far_lsplit, ts.far_csplit, K,
                                                    ts.near_off, ts.near_rng, pc);
    WNNC_LAUNCH_CHECK();
    WorkBuild wb;
    work_count(wb, 0, ng, ts.near_off, ts.near_rng, ts.far_off, ts.far_lsplit, true, s);
    unsigned long long* hc = reinterpret_cast<unsigned long long*>(pinned_scratch());
    int* wt = reinterpret_cast<int*>(hc + 6);
    WNNC_CUDA(cudaMemcpyAsync(hc, pc, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    WNNC_CUDA(cudaMemcpyAsync(wt, wb.tot, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    WNNC_CUDA(cudaStreamSynchronize(s));
    pool_free(pc);
    ts.far_pairs = (int64_t)hc[0];
    ts.near_pairs = (int64_t)hc[1];
    ts.local_entries = (int64_t)hc[2];
    ts.local_pairs = (int64_t)hc[3];
    ts.cluster_entries = (int64_t)hc[4];
    ts.cluster_pairs = (int64_t)hc[5];
    work_fill(ts.work, wb, wt, s);
}

void free_target_set(TargetSet& ts) {
    dfree(ts.perm); dfree(ts.pos); dfree(ts.corig); dfree(ts.gorig); dfree(ts.goff); dfree(ts.glo);
    dfree(ts.ghi); dfree(ts.gbl); dfree(ts.gbh); dfree(ts.far_off); dfree(ts.far_id); dfree(ts.near_off); dfree(ts.near_rng);
    dfree(ts.far_lsplit); dfree(ts.gctr); dfree(ts.far_csplit); dfree(ts.cctr); dfree(ts.cexp);
    free_work(ts.work);
}

static void grow_nodes(Tree& t, int& cap, int need) {
    if (need <= cap) return;
    int ncap = std::max(need, 2 * cap);
    auto grow = [&](int*& p) {
        int* q = dalloc<int>(ncap);
        WNNC_CUDA(cudaMemcpyAsync(q, p, sizeof(int) * cap, cudaMemcpyDeviceToDevice, alloc_stream()));
        pool_free(p);
        p = q;
    };
    grow(t.node_start); grow(t.node_count); grow(t.node_parent);
    grow(t.node_child0); grow(t.node_nchild); grow(t.node_depth);
    cap = ncap;
}

// Transposed far lists (node -> the far entries that name it), on stream s.
static void build_tfar(Tree& t, cudaStream_t s) {
    const TargetSet& S = t.self;
    const int ng = S.ngroups;
    t.tfar_off = dalloc<int>(t.nnodes + 1);
    const int64_t ne = S.far_entries;
    if (S.far_lsplit && ne >= (int64_t(1) << 30)) fail(WNNC_ECAPACITY, "too many far entries for local expansions");
    t.tfar_ent = dalloc<int>(std::max<int64_t>(ne, 1));
    if (ne == 0) {
        WNNC_CUDA(cudaMemsetAsync(t.tfar_off, 0, sizeof(int) * (t.nnodes + 1), s));
        return;
    }
    uint64_t* k = dalloc<uint64_t>(ne);
    k_tfar_keys<<<ceil_div((int64_t)ng * 32, kTB), kTB, 0, s>>>(S.far_off, S.far_id, ng, S.far_lsplit, S.far_csplit,
                                                               S.cluster_k, t.nnodes, k);
    WNNC_LAUNCH_CHECK();
    // entry order already ascending: the node bits and, with local
    // expansions, the class bits (each node's list by class, so that the
    // warps of the node gather mostly take one kind of entry at a time)
    radix_sort_pairs(k, nullptr, ne, 32 + bits_for(t.nnodes + 1), s, S.far_lsplit ? 30 : 32);
    k_tfar_finish<<<ceil_div(ne, kTB), kTB, 0, s>>>(k, ne, t.nnodes, t.tfar_ent, t.tfar_off);
    WNNC_LAUNCH_CHECK();
    wait_before_free(s);
    pool_free(k);
}

void build_tree(Tree& t, const float* pts, cudaStream_t s) {
    const int64_t n = t.n;
    const wnnc_tree_params& P = t.params;
    // --- normalisation and Morton order ---
    const int nparts = (int)std::min<int64_t>(1024, ceil_div(n, kTB));
    double* part = dalloc<double>(6 * nparts);
    double* cs = dalloc<double>(4);
    k_bbox_partial<<<nparts, kTB, 0, s>>>(pts, n, part);
    WNNC_LAUNCH_CHECK();
    k_bbox_final<<<1, 1024, 0, s>>>(part, nparts, cs);
    WNNC_LAUNCH_CHECK();
    double* hcs = reinterpret_cast<double*>(pinned_scratch());
    WNNC_CUDA(cudaMemcpyAsync(hcs, cs, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    double* xn = dalloc<double>(3 * n);
    uint32_t* idx = dalloc<uint32_t>(n);
    t.keys = dalloc<uint64_t>(n);
    k_normalize_keys<<<ceil_div(n, kTB), kTB, 0, s>>>(pts, n, cs, xn, t.keys, idx);
    WNNC_LAUNCH_CHECK();
    WNNC_CUDA(cudaStreamSynchronize(s));
    if (!(hcs[3] > 0.0) || !std::isfinite(hcs[3]))
        fail(WNNC_EINVAL, "point coordinates must be finite");
    for (int k = 0; k < 3; ++k) t.center[k] = hcs[k];
    t.scale = hcs[3];
    radix_sort_pairs(t.keys, idx, n, kKeyBits, s);
    t.xs = dalloc<double>(3 * n);
    int64_t* perm_tmp = dalloc<int64_t>(n);
    k_gather_sorted<<<ceil_div(n, kTB), kTB, 0, s>>>(xn, idx, n, t.xs, perm_tmp);
    WNNC_LAUNCH_CHECK();

    // --- octree, breadth-first by level ---
    int cap = (int)std::min<int64_t>(INT32_MAX / 2, 2 * n + 64);
    t.node_start = dalloc<int>(cap); t.node_count = dalloc<int>(cap); t.node_parent = dalloc<int>(cap);
    t.node_child0 = dalloc<int>(cap); t.node_nchild = dalloc<int>(cap); t.node_depth = dalloc<int>(cap);
    std::vector<int> level_off = {0, 1};
    int total_nodes = 1;
    int* nkids = dalloc<int>(n + 1);
    int* bnd = dalloc<int>(8 * (size_t)(n + 1));   // child range ends; a level holds at most n nodes
    bool built = false;
    {
        // one cooperative launch, if the device takes one and the nodes fit
        int dev = 0, coop = 0, sms = 0, per_sm = 0;
        WNNC_CUDA(cudaGetDevice(&dev));
        WNNC_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        WNNC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        WNNC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_octree, kOctThreads, 0));
        if (coop && per_sm > 0) {
            const int G = std::min(per_sm, 2) * sms;
            int* ctl = dalloc<int>(kOctMaxLevels + 8 + G);   // lvl, barrier, status, block totals
            WNNC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(int) * (kOctMaxLevels + 8 + G), s));
            OctArgs A;
            A.keys = t.keys;
            A.n = (int)n;
            A.leaf_size = P.leaf_size;
            A.max_depth = P.max_depth;
            A.cap = cap;
            A.start = t.node_start;
            A.count = t.node_count;
            A.parent = t.node_parent;
            A.child0 = t.node_child0;
            A.nchild = t.node_nchild;
            A.depth = t.node_depth;
            A.bnd = bnd;
            A.nkids = nkids;
            A.lvl = ctl;
            A.bar = reinterpret_cast<GridBar*>(ctl + kOctMaxLevels);
            A.status = ctl + kOctMaxLevels + 4;
            A.block_tot = ctl + kOctMaxLevels + 8;
            void* args[] = {&A};
            const cudaError_t le =
                cudaLaunchCooperativeKernel((const void*)k_octree, dim3(G), dim3(kOctThreads), args, 0, s);
            if (le == cudaErrorCooperativeLaunchTooLarge) {
                // fewer SMs than the device reports (a partitioned device): by launches
                (void)cudaGetLastError();
            } else {
                WNNC_CUDA(le);
                WNNC_LAUNCH_CHECK();
                int* h = reinterpret_cast<int*>(pinned_scratch());
                WNNC_CUDA(cudaMemcpyAsync(h, ctl, sizeof(int) * (kOctMaxLevels + 8), cudaMemcpyDeviceToHost, s));
                WNNC_CUDA(cudaStreamSynchronize(s));
                const int* hl = h;
                const GridBar* hb = reinterpret_cast<const GridBar*>(h + kOctMaxLevels);
                const int* hs = h + kOctMaxLevels + 4;
                if (hb->err) {
                    pool_free(ctl);
                    fail(WNNC_ETIMEOUT, "a grid barrier of the octree build gave up");
                }
                if (!hs[1]) {
                    built = true;
                    total_nodes = hs[0];
                    for (int L = 1; L < kOctMaxLevels && hl[L] > 0; ++L)
                        level_off.push_back(level_off.back() + hl[L]);
                }
            }
            pool_free(ctl);
        }
    }
    if (!built) {
        // level by level, one launch each, growing the node arrays as needed
        {
            int h0 = 0, hn = (int)n, hp = -1;
            WNNC_CUDA(cudaMemcpyAsync(t.node_start, &h0, sizeof(int), cudaMemcpyHostToDevice, s));
            WNNC_CUDA(cudaMemcpyAsync(t.node_count, &hn, sizeof(int), cudaMemcpyHostToDevice, s));
            WNNC_CUDA(cudaMemcpyAsync(t.node_parent, &hp, sizeof(int), cudaMemcpyHostToDevice, s));
            WNNC_CUDA(cudaMemcpyAsync(t.node_depth, &h0, sizeof(int), cudaMemcpyHostToDevice, s));
        }
        int* koff = dalloc<int>(n + 2);
        int base = 0, m = 1, depth = 0;
        while (m > 0) {
            k_split_count<<<ceil_div((int64_t)8 * m, kTB), kTB, 0, s>>>(t.keys, t.node_start, t.node_count, base, m,
                                                                       depth, P.leaf_size, P.max_depth, nkids, bnd);
            WNNC_LAUNCH_CHECK();
            exclusive_scan_i32(nkids, koff, m, s);
            int nnext = read_int(koff + m, s);
            grow_nodes(t, cap, total_nodes + nnext);
            k_split_write<<<ceil_div(m, kTB), kTB, 0, s>>>(t.node_start, t.node_count, t.node_parent,
                                                          t.node_child0, t.node_nchild, t.node_depth, base, m, depth,
                                                          total_nodes, koff, nkids, bnd);
            WNNC_LAUNCH_CHECK();
            base = total_nodes;
            total_nodes += nnext;
            m = nnext;
            if (m > 0) {
                level_off.push_back(total_nodes);
                ++depth;
            }
        }
        pool_free(koff);
    }
    pool_free(nkids);
    pool_free(bnd);
    t.nnodes = total_nodes;
    t.nlevels = (int)level_off.size() - 1;
    t.depth_reached = t.nlevels - 1;
    t.level_off = new int[level_off.size()];
    std::copy(level_off.begin(), level_off.end(), t.level_off);

    // --- boxes and centroids, from the leaves up ---
    t.node_lo = dalloc<double>(3 * (size_t)t.nnodes);
    t.node_hi = dalloc<double>(3 * (size_t)t.nnodes);
    double* sum = dalloc<double>(3 * (size_t)t.nnodes);
    {
        int* arrive = dalloc<int>(t.nnodes);
        WNNC_CUDA(cudaMemsetAsync(arrive, 0, sizeof(int) * (size_t)t.nnodes, s));
        k_node_boxes<<<ceil_div(t.nnodes, kTB), kTB, 0, s>>>(t.xs, t.node_start, t.node_count, t.node_child0,
                                                            t.node_nchild, t.node_parent, t.nnodes, t.node_lo,
                                                            t.node_hi, sum, arrive);
        WNNC_LAUNCH_CHECK();
        pool_free(arrive);
    }
    t.node_lof = dalloc<float4>(t.nnodes);
    t.node_hif = dalloc<float4>(t.nnodes);
    k_node_fbox<<<ceil_div(t.nnodes, kTB), kTB, 0, s>>>(t.node_lo, t.node_hi, t.nnodes, t.node_lof, t.node_hif);
    WNNC_LAUNCH_CHECK();
    t.node_cell = dalloc<float4>(t.nnodes);
    t.node_cent = dalloc<float4>(t.nnodes);
    t.leaf_of = dalloc<int>(n);
    k_node_cells<<<ceil_div(t.nnodes, kTB), kTB, 0, s>>>(t.keys, t.node_start, t.node_count, t.node_depth,
                                                        t.node_nchild, sum, t.nnodes, t.node_cell,
                                                        t.node_cent, t.leaf_of);
    WNNC_LAUNCH_CHECK();
    wait_before_free(s);
    pool_free(sum);
    // the classes of the moment sums: nodes summed over their points by one
    // thread (<= kMomSmall points) or one warp (up to kMomDirect points, and
    // leaves of any size: a leaf at the depth limit may hold more); the inner
    // nodes above that ("top") are summed from their "front", the summed nodes
    // whose parent is a top node, which partition a top node's points in
    // Morton order.  Lists by flags and prefix sums (ascending node id); the
    // front sorted by first point.
    {
        const int nn = t.nnodes;
        int* fl = dalloc<int>(4 * ((size_t)nn + 1));   // flags, then offsets: mid, top, front, leaf
        k_mom_flags<<<ceil_div(nn, kTB), kTB, 0, s>>>(t.node_nchild, t.node_count, t.node_parent, nn, fl);
        WNNC_LAUNCH_CHECK();
        // in place; entry nn of each array receives the total
        for (int c = 0; c < 4; ++c) exclusive_scan_i32(fl + c * ((int64_t)nn + 1), fl + c * ((int64_t)nn + 1), nn, s);
        int* tot = dalloc<int>(4);
        k_mom_totals<<<1, 32, 0, s>>>(fl, nn, tot);
        WNNC_LAUNCH_CHECK();
        int h[4];
        int* hp = reinterpret_cast<int*>(pinned_scratch());
        WNNC_CUDA(cudaMemcpyAsync(hp, tot, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        WNNC_CUDA(cudaStreamSynchronize(s));
        std::copy(hp, hp + 4, h);
        t.nmom_mid = h[0];
        t.nmom_top = h[1];
        t.nleaves = h[3];
        const int nfront = h[2];
        t.mom_mid = dalloc<int>(h[0]);
        t.mom_top = dalloc<int>(h[1]);
        t.mom_top_rng = dalloc<int2>(h[1]);
        t.mom_front = dalloc<int>(nfront);
        uint64_t* fkeys = dalloc<uint64_t>(nfront);
        k_mom_lists<<<ceil_div(nn, kTB), kTB, 0, s>>>(fl, nn, t.node_start, t.mom_mid, t.mom_top, fkeys);
        WNNC_LAUNCH_CHECK();
        radix_sort_pairs(fkeys, nullptr, nfront, 32 + bits_for(n), s, 32);   // node ids already ascending
        if (nfront > 0) {
            k_low32<<<ceil_div(nfront, kTB), kTB, 0, s>>>(fkeys, nfront, t.mom_front);
            WNNC_LAUNCH_CHECK();
        }
        if (h[1] > 0) {
            k_mom_top_ranges<<<ceil_div(h[1], kTB), kTB, 0, s>>>(t.mom_top, h[1], t.node_start, t.node_count, fkeys,
                                                                  nfront, t.mom_top_rng);
            WNNC_LAUNCH_CHECK();
        }
        wait_before_free(s);
        pool_free(fl);
        pool_free(tot);
        pool_free(fkeys);
    }

    // --- the points as targets: same Morton order as the sources; the
    // transposed far lists, which only the adjoint reads, are built on the
    // second stream once the far lists are final, beside the rest ---
    if (!t.aux) WNNC_CUDA(cudaStreamCreateWithFlags(&t.aux, cudaStreamNonBlocking));
    cudaEvent_t ev_far = nullptr, ev_tfar = nullptr;
    WNNC_CUDA(cudaEventCreateWithFlags(&ev_far, cudaEventDisableTiming));
    WNNC_CUDA(cudaEventCreateWithFlags(&ev_tfar, cudaEventDisableTiming));
    build_target_set(t, t.self, xn, n, true, s, perm_tmp, [&] {
        WNNC_CUDA(cudaEventRecord(ev_far, s));
        WNNC_CUDA(cudaStreamWaitEvent(t.aux, ev_far, 0));
        AllocStream as(t.aux);
        build_tfar(t, t.aux);
        WNNC_CUDA(cudaEventRecord(ev_tfar, t.aux));
    });
    pool_free(xn);
    pool_free(idx);
    pool_free(perm_tmp);
    pool_free(part);
    pool_free(cs);

    // --- transposed lists and work lists for the adjoint ---
    const TargetSet& S = t.self;
    const int ng = S.ngroups;
    const int nach = ceil_div(t.n, kAdjChunk);
    t.nach = nach;
    {
        int64_t nr = S.near_ranges;
        // near slots: lengths of the ranges, scanned (ranges are group-major)
        int* len = dalloc<int>(nr + 1);
        t.rng_slot = dalloc<int>(nr + 2);
        if (nr) {
            k_range_len<<<ceil_div(nr, kTB), kTB, 0, s>>>(S.near_rng, nr, len);
            WNNC_LAUNCH_CHECK();
        }
        exclusive_scan_i32(len, t.rng_slot, nr, s);
        int* cnt = dalloc<int>(nr + 1);
        int* coff = dalloc<int>(nr + 2);
        if (nr) {
            k_tnear_count<<<ceil_div(nr, kTB), kTB, 0, s>>>(S.near_rng, nr, cnt);
            WNNC_LAUNCH_CHECK();
        }
        exclusive_scan_i32(cnt, coff, nr, s);
        // both totals with one read-back
        int* hp = reinterpret_cast<int*>(pinned_scratch());
        WNNC_CUDA(cudaMemcpyAsync(hp, t.rng_slot + nr, sizeof(int), cudaMemcpyDeviceToHost, s));
        WNNC_CUDA(cudaMemcpyAsync(hp + 1, coff + nr, sizeof(int), cudaMemcpyDeviceToHost, s));
        WNNC_CUDA(cudaStreamSynchronize(s));
        t.near_slots = hp[0];
        const int ne = hp[1];
        pool_free(len);
        uint64_t* k = dalloc<uint64_t>(ne);
        uint32_t* msk = dalloc<uint32_t>(ne);
        int* slt = dalloc<int>(ne);
        uint32_t* idx = dalloc<uint32_t>(ne);
        if (nr) {
            k_tnear_fill<<<ceil_div(nr, kTB), kTB, 0, s>>>(S.near_rng, nr, S.near_off, ng, coff, t.rng_slot, k,
                                                          msk, slt, idx);
            WNNC_LAUNCH_CHECK();
        }
        radix_sort_pairs(k, idx, ne, 32 + bits_for(nach), s, 32);   // groups already ascending
        int* head = dalloc<int>(ne + 1);
        int* hscan = dalloc<int>(ne + 2);
        if (ne) {
            k_key_heads<<<ceil_div(ne, kTB), kTB, 0, s>>>(k, ne, head);
            WNNC_LAUNCH_CHECK();
        }
        exclusive_scan_i32(head, hscan, ne, s);
        int nu = read_int(hscan + ne, s);
        t.tnear_entries = nu;
        t.tnear_ent = dalloc<int2>(nu);
        uint64_t* uk = dalloc<uint64_t>(nu);
        if (ne) {
            k_tnear_merge<<<ceil_div(ne, kTB), kTB, 0, s>>>(k, idx, msk, slt, ne, hscan, t.tnear_ent, uk);
            WNNC_LAUNCH_CHECK();
        }
        t.tnear_off = dalloc<int>(nach + 1);
        segment_offsets_hi32(uk, nu, t.tnear_off, nach, s);
        wait_before_free(s);
        pool_free(cnt); pool_free(coff); pool_free(k); pool_free(msk); pool_free(slt); pool_free(idx);
        pool_free(head); pool_free(hscan); pool_free(uk);
    }
    // the adjoint's three work lists, sized by one read-back
    {
        WorkBuild wb[3];
        work_count(wb[0], 2, ng, nullptr, nullptr, S.far_off, S.far_lsplit, false, s);
        work_count(wb[1], 0, ng, S.near_off, S.near_rng, nullptr, nullptr, false, s);
        work_count(wb[2], 1, nach, t.tnear_off, nullptr, nullptr, nullptr, true, s);
        int* ht = reinterpret_cast<int*>(pinned_scratch());
        for (int k = 0; k < 3; ++k)
            WNNC_CUDA(cudaMemcpyAsync(ht + 3 * k, wb[k].tot, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
        WNNC_CUDA(cudaStreamSynchronize(s));
        int wt[3][3];
        std::copy(ht, ht + 9, &wt[0][0]);
        work_fill(t.adj_far_work, wb[0], wt[0], s);
        work_fill(t.adj_pair_work, wb[1], wt[1], s);
        work_fill(t.adj_near_work, wb[2], wt[2], s);
    }
    WNNC_CUDA(cudaStreamWaitEvent(s, ev_tfar, 0));
    WNNC_CUDA(cudaEventDestroy(ev_far));
    WNNC_CUDA(cudaEventDestroy(ev_tfar));
}

void free_tree(Tree& t) {
    if (t.aux) cudaStreamDestroy(t.aux);
    if (t.ev_fork) cudaEventDestroy(t.ev_fork);
    if (t.ev_join) cudaEventDestroy(t.ev_join);
    t.aux = nullptr;
    t.ev_fork = t.ev_join = nullptr;
    dfree(t.keys); dfree(t.xs);
    dfree(t.node_start); dfree(t.node_count); dfree(t.node_parent); dfree(t.node_child0);
    dfree(t.node_nchild); dfree(t.node_depth); dfree(t.node_lo); dfree(t.node_hi); dfree(t.node_lof); dfree(t.node_hif);
    dfree(t.node_cell); dfree(t.node_cent); dfree(t.leaf_of);
    delete[] t.level_off;
    t.level_off = nullptr;
    free_target_set(t.self);
    dfree(t.tfar_off); dfree(t.tfar_ent); dfree(t.tnear_off); dfree(t.tnear_ent); dfree(t.rng_slot);
    free_work(t.adj_pair_work);
    free_work(t.adj_far_work);
    free_work(t.adj_near_work);
    dfree(t.mu_a); dfree(t.mu_b); dfree(t.r_s); dfree(t.g_mu); dfree(t.g_r); dfree(t.s_s); dfree(t.area_s); dfree(t.mom);
    dfree(t.mom_r); dfree(t.mom_x); dfree(t.dmom); dfree(t.mom_mid); dfree(t.mom_top); dfree(t.mom_top_rng); dfree(t.mom_front); dfree(t.node_rep); dfree(t.contrib);
    dfree(t.near_contrib); dfree(t.vnode); dfree(t.red_ticket);
    dfree(t.mom_dip); dfree(t.mom_dip_r); dfree(t.dip_corr); dfree(t.contrib_h0); dfree(t.contrib_h1);
    dfree(t.node_abs); dfree(t.local_rec); dfree(t.gadj);
    dfree(t.gather_raw);
    dfree(t.cadj);
    dfree(t.hnode0); dfree(t.hnode1);
    dfree(t.partials); dfree(t.red); dfree(t.part_acc); dfree(t.scalars); dfree(t.err_flag);
}

}  // namespace wnnc
