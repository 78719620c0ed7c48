// operators.cu -- node moments and the treecode sums of A, G and A^T.
//
// Pair terms (d = x_source - x_target, r = |d|, every term zero when r < w):
//   A  : gradPhi(x_t - x_s) . mu_s = (d . mu_s) / (4 pi r^3)             (Thm. 1, Eq. 5)
//   G  : -HPhi(x_t - x_s) mu_s = mu_s/(4 pi r^3) - 3 d (d.mu_s)/(4 pi r^5) (Eq. 9, Eq. 10)
//   A^T: s_s gradPhi(x_s - x_t) = -s_s d / (4 pi r^3)                    (Sec. 4.5)
// A far node B acts as one source at its representative x_B carrying
// nu_B = sum of its points' attributes (Eq. 13, Eq. 14).
//
// Layout: one warp per work item (a slice of one target group's lists, see
// WorkList), one target per lane.  Sources (a range of points, or a batch of
// far nodes) are staged 32 at a time in shared memory, shifted into the
// group's frame (dyadic origins, exact shifts), and every lane sums over them
// with rsqrt and FMA chains.  The 1/(4 pi) factor is applied once.  Groups cut
// into several items write partial sums to scratch slots; a finalize pass adds
// them in a fixed order (results do not depend on scheduling).
//
// Cut-off test per batch: when every staged source of a batch lies farther
// from the group's box than the cut-off radius (with a margin far above the
// rounding of the test), no pair of the batch can be cut, and the batch runs
// an inner loop without the compare/select; its terms are bit-identical to
// those of the general loop.
#include <algorithm>
#include <cmath>
#include <cuda_bf16.h>
#include <cfloat>
#include <type_traits>
#include <utility>

#include "common.cuh"

namespace wnnc {

namespace {

constexpr int kTB = 256;
constexpr int kGatherWarps = 4;
// Inner-loop unroll depth and minimum resident blocks per SM of the pair
// kernels (tuning knobs; the defaults are the measured best on B300).
#ifndef WNNC_UNROLL
#define WNNC_UNROLL 16
#endif
// The treecode gather runs with at least 6 resident blocks per SM and the
// two adjoint pair kernels with at least 7 (the register caps that measured
// fastest; a few bytes spill in the gather); the other kernels take the
// registers they need.
#ifndef WNNC_GATHER_MINB
#define WNNC_GATHER_MINB 6
#endif
#ifndef WNNC_ADJ_MINB
#define WNNC_ADJ_MINB 7
#endif
#define WNNC_GATHER_BOUNDS __launch_bounds__(32 * kGatherWarps)
#define WNNC_CAPPED_BOUNDS __launch_bounds__(32 * kGatherWarps, WNNC_GATHER_MINB)
#define WNNC_ADJ_BOUNDS __launch_bounds__(32 * kGatherWarps, WNNC_ADJ_MINB)
constexpr int kUnroll = WNNC_UNROLL;
// targets per lane of the treecode gather (1 or 2)
#ifndef WNNC_GATHER_TPL
#define WNNC_GATHER_TPL 2
#endif
constexpr int kGatherTPL = WNNC_GATHER_TPL;

// ---------------------------------------------------------------------------
// Node moments in two launches, with no dependency chain through the whole
// tree:
//   1. one thread per node of at most kMomSmall points sums its point range;
//   2. one warp per node of up to kMomDirect points (or a leaf of any size)
//      sums its range (lane-strided, then a fixed xor reduction); classes 1
//      and 2 share a launch;
//   3. one block per larger inner node (the top levels) adds the sums of the
//      class 1 and 2 nodes that partition its points.
//   mom[b]  = (sum nu, sum |nu|)        (nu = mu: 3 components; nu = s: 1)
//   momx[b] = sum |nu| (x - cell_b)     (only for the |nu|-weighted representative)
//   rep[b]  = momx[b] / sum |nu|, or the point centroid when sum |nu| = 0
// ---------------------------------------------------------------------------
// Sums run in Acc = float, or double with moments_fp64 (the double sums of
// every node are then kept in dmom, 8 per node, for the top levels).
// Point term of the moments: nu (3 or 1 components), |nu|, |nu| (x - cell).
template <bool SCALAR, bool WEIGHTED, class Acc>
__device__ __forceinline__ void mom_point(int j, const float4& cb, const float4* spos, const float4* scorig,
                                          const float4* nu_vec, const float* nu_s, Acc (&m)[7]) {
    float v0, v1 = 0.f, v2 = 0.f, a;
    if (SCALAR) {
        v0 = nu_s[j];
        a = fabsf(v0);
    } else {
        const float4 v = nu_vec[j];
        v0 = v.x; v1 = v.y; v2 = v.z;
        a = sqrtf(v0 * v0 + v1 * v1 + v2 * v2);
    }
    m[0] += v0; m[1] += v1; m[2] += v2; m[3] += a;
    if (WEIGHTED) {
        const float4 p = spos[j], go = scorig[j >> 5];   // the point in its chunk frame
        m[4] += (Acc)a * (Acc)((go.x - cb.x) + p.x);
        m[5] += (Acc)a * (Acc)((go.y - cb.y) + p.y);
        m[6] += (Acc)a * (Acc)((go.z - cb.z) + p.z);
    }
}

template <bool WEIGHTED, class Acc>
__device__ __forceinline__ void mom_store(int b, const float4* ncent, float4* mom, float4* momx, float4* rep,
                                          double* dmom, const Acc (&m)[7]) {
    mom[b] = make_float4((float)m[0], (float)m[1], (float)m[2], (float)m[3]);
    if (WEIGHTED) {
        momx[b] = make_float4((float)m[4], (float)m[5], (float)m[6], 0.f);
        rep[b] = m[3] > 0 ? make_float4((float)(m[4] / m[3]), (float)(m[5] / m[3]), (float)(m[6] / m[3]), 0.f)
                          : ncent[b];
    }
    if (dmom)
        for (int k = 0; k < 7; ++k) dmom[8 * (int64_t)b + k] = (double)m[k];
}

template <bool SCALAR, bool WEIGHTED, class Acc>
__device__ __forceinline__ void mom_small(int b, int nnodes, const int* nstart, const int* ncount,
                                          const float4* ncell, const float4* ncent, const float4* spos,
                                          const float4* scorig, const float4* nu_vec, const float* nu_s,
                                          float4* mom, float4* momx, float4* rep, double* dmom) {
    if (b >= nnodes) return;
    const int cnt = ncount[b];
    if (cnt > kMomSmall) return;
    const int j0 = nstart[b];
    const float4 cb = ncell[b];
    Acc m[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
    for (int j = j0; j < j0 + cnt; ++j) mom_point<SCALAR, WEIGHTED, Acc>(j, cb, spos, scorig, nu_vec, nu_s, m);
    mom_store<WEIGHTED, Acc>(b, ncent, mom, momx, rep, dmom, m);
}

template <bool SCALAR, bool WEIGHTED, class Acc>
__device__ __forceinline__ void mom_direct(int k, int lane, int nmid, const int* mid, const int* nstart,
                                           const int* ncount, const float4* ncell, const float4* ncent,
                                           const float4* spos, const float4* scorig, const float4* nu_vec,
                                           const float* nu_s, float4* mom, float4* momx, float4* rep,
                                           double* dmom) {
    if (k >= nmid) return;
    const int b = mid[k];
    const int cnt = ncount[b];
    const int j0 = nstart[b];
    const float4 cb = ncell[b];
    Acc m[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
    for (int j = j0 + lane; j < j0 + cnt; j += 32)
        mom_point<SCALAR, WEIGHTED, Acc>(j, cb, spos, scorig, nu_vec, nu_s, m);
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        if (!WEIGHTED && c >= 4) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m[c] += __shfl_xor_sync(0xffffffffu, m[c], o);
    }
    if (lane == 0) mom_store<WEIGHTED, Acc>(b, ncent, mom, momx, rep, dmom, m);
}

// Classes 1 and 2 in one launch: blocks [0, grid_m) take the warp class
// (warp per node of the mid list), the rest the thread class.
template <bool SCALAR, bool WEIGHTED, class Acc>
__global__ void k_mom_sums(int nnodes, int nmid, int grid_m, const int* mid, const int* nstart,
                           const int* ncount, const float4* ncell, const float4* ncent, const float4* spos,
                           const float4* scorig, const float4* nu_vec, const float* nu_s, float4* mom,
                           float4* momx, float4* rep, double* dmom) {
    if ((int)blockIdx.x < grid_m) {
        const int k = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
        mom_direct<SCALAR, WEIGHTED, Acc>(k, threadIdx.x & 31, nmid, mid, nstart, ncount, ncell, ncent, spos,
                                          scorig, nu_vec, nu_s, mom, momx, rep, dmom);
    } else {
        const int b = (int)((blockIdx.x - grid_m) * blockDim.x + threadIdx.x);
        mom_small<SCALAR, WEIGHTED, Acc>(b, nnodes, nstart, ncount, ncell, ncent, spos, scorig, nu_vec, nu_s,
                                         mom, momx, rep, dmom);
    }
}

// Class 3: one block per top node (an inner node of more than kMomDirect
// points) adds the moments of its front, the summed nodes that partition its
// points (ordered by first point): thread k takes front nodes k, k + 256,
// ..., then a fixed xor reduction per warp and the warps' sums in order.  No
// top node waits for another, so the top levels cost one short launch.
constexpr int kMomTopThreads = 256;
template <bool WEIGHTED, class Acc>
__global__ void __launch_bounds__(kMomTopThreads) k_mom_top(const int* top, const int2* top_rng, const int* front,
                                                            const float4* ncell, const float4* ncent,
                                                            float4* mom, float4* momx, float4* rep, double* dmom) {
    __shared__ Acc red[kMomTopThreads / 32][7];
    const int b = top[blockIdx.x];
    const int2 fr = top_rng[blockIdx.x];
    const float4 cp = ncell[b];
    Acc m[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int q = fr.x + (int)threadIdx.x; q < fr.y; q += kMomTopThreads) {
        const int c = front[q];
        Acc cm[7];
        if (dmom) {
            for (int k = 0; k < 7; ++k) cm[k] = (Acc)dmom[8 * (int64_t)c + k];
        } else {
            const float4 mm = mom[c];
            cm[0] = mm.x; cm[1] = mm.y; cm[2] = mm.z; cm[3] = mm.w;
            if (WEIGHTED) {
                const float4 xx = momx[c];
                cm[4] = xx.x; cm[5] = xx.y; cm[6] = xx.z;
            }
        }
        for (int k = 0; k < 4; ++k) m[k] += cm[k];
        if (WEIGHTED) {
            // re-centre the front node's weighted offsets on this node's cell
            const float4 cc = ncell[c];
            m[4] += cm[4] + cm[3] * (Acc)(cc.x - cp.x);
            m[5] += cm[5] + cm[3] * (Acc)(cc.y - cp.y);
            m[6] += cm[6] + cm[3] * (Acc)(cc.z - cp.z);
        }
    }
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        if (!WEIGHTED && k >= 4) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m[k] += __shfl_xor_sync(0xffffffffu, m[k], o);
        if (lane == 0) red[wl][k] = m[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Acc t[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < kMomTopThreads / 32; ++w)
            for (int k = 0; k < (WEIGHTED ? 7 : 4); ++k) t[k] += red[w][k];
        mom_store<WEIGHTED, Acc>(b, ncent, mom, momx, rep, dmom, t);
    }
}

// ---------------------------------------------------------------------------
// Gather kernel (one warp per work item)
// ---------------------------------------------------------------------------
enum Epi : int {
    kEpiStoreW = 0,      // out[perm[i]] = F
    kEpiStoreGrad,       // out[perm[i]] = grad F (caller units) = -G * scale
    kEpiStoreATpaper,    // out[perm[i]] = A^T s (caller units) = acc * scale^2
    kEpiResidual,        // s_s[i] = 1/2 - F; partial |s|^2
    kEpiNormSq,          // partial |F|^2
    kEpiRescale,         // mu_out[i] = Ghat |mu_i| / |Ghat| (or sigma_i / |Ghat|)
    kEpiStoreR,          // mu_out[i] = acc / (4 pi) (sorted, normalised); partial |.|^2
    kEpiResidualAG,      // kOpAG: s_s[i] = 1/2 - F, partial |s|^2; g_out[i] = G / (4 pi)
    kEpiNormSqAG,        // kOpAG: partial |F|^2; g_out[i] = G / (4 pi)
};

struct GatherArgs {
    // work
    const Item* items;
    int nitems;
    const int4* splits;
    unsigned* split_cnt;
    int nsplit;
    float4* part_acc;
    // targets
    int ngroups;
    const int* goff;
    const float4* tpos;
    const float4* tcorig;
    const float4* tgorig;
    const int64_t* tperm;
    const int* far_id;
    const int2* near_rng;
    // sources
    const float4* spos;
    const float4* scorig;
    const float4* sval;       // mu (x,y,z) per sorted source point
    const float* sval_s;      // s per sorted source point (A^T, paper mode)
    const float4* ncell;
    const float4* nrep;
    const float4* nmom;
    float w2;
    float fast2;              // squared batch-test radius (cut-off radius plus margin)
    int near_bf16;            // round near-field coordinates to bfloat16
    const float4* tgbl;       // target group boxes in their own frames
    const float4* tgbh;
    float scale;              // output unit conversion factor
    // epilogue buffers
    float* out;
    float* s_out;
    double* partial;
    const float4* mu_cur;     // rescale: the field before the WNNC update
    const float* area;        // rescale mode 1
    float4* mu_out;
    float4* g_out;            // kOpAG: G of the field (sorted, normalised)
    int rescale_mode;
    // per-target walk (criterion 1)
    int walk;                 // 1: k_walk instead of the list gather
    float copen;              // c = 1/theta (infinite for theta = 0)
    const int* nchild0;       // first child of each node
    const int* nnchild;       // number of children (0 for leaves)
    const int* nstart;        // first sorted point of each node
    const int* ncount;        // points of each node
    int* err_flag;            // device error flags (a walk stack overflow sets kErrCapacity)
    const float4* dip_corr;   // per sorted target, far terms added in the epilogue (G x,y,z, A): the
                              // first-order terms (far_order 1) or the local expansions (local_theta > 0)
    const int* far_off;       // far list offsets per group
    const int* lsplit;        // local_theta > 0: first expanded far entry of each group
    const float4* gctr;       //   the expansion centre in the group's frame and the group's radius
    const float4* lrec;       //   per node (centroid, M_x), (M_y, M_z, 0, 0) of this call's field
    float4* raw;              // set: items of groups not cut store their sums here (G x,y,z, A)
                              // instead of running the epilogue (k_gather_finalize_all does)
    const int* gsplit;        //   per group its record in splits, or -1
    const int* csplit;        // local_cluster > 0: first entry expanded about the group's cluster
    int cluster_k;            //   groups per cluster
    int nclusters;
    const float4* cctr;       //   cluster frame origins
    const float4* cexp;       //   expansion centre in the cluster's frame and the cluster's radius
};

// Accumulators: (x, y, z) holds the A / A^T sum, or for G the sum of
// mu / r^3; (u, v, q) holds, for G only, the sum of (d.mu) d / r^5, so that
// G = (x, y, z) - 3 (u, v, q); s holds A's sum when both run together.
struct Acc3 {
    float x = 0.f, y = 0.f, z = 0.f;
    float u = 0.f, v = 0.f, q = 0.f;
    float s = 0.f;            // A's sum when A and G run together (kOpAG)
};

// One pair term.  CUT: apply the cut-off r^2 >= w2 (otherwise the caller has
// shown that every pair of the batch passes it).
template <int OP, bool CUT>
__device__ __forceinline__ void interact(const float4& t, const float4& sp, const float4& sv, float w2,
                                         Acc3& a) {
    float dx = sp.x - t.x, dy = sp.y - t.y, dz = sp.z - t.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float ir = rsqrtf(r2);
    if (CUT) ir = (r2 >= w2) ? ir : 0.f;
    if (OP == kOpA) {
        float ir3 = ir * ir * ir;
        float dm = fmaf(dx, sv.x, fmaf(dy, sv.y, dz * sv.z));
        a.x = fmaf(dm, ir3, a.x);
    } else if (OP == kOpG || OP == kOpAG) {
        float ir2 = ir * ir;
        float ir3 = ir2 * ir;
        float dm = fmaf(dx, sv.x, fmaf(dy, sv.y, dz * sv.z));
        float k5 = (dm * ir2) * ir3;
        if (OP == kOpAG) a.s = fmaf(dm, ir3, a.s);
        a.x = fmaf(sv.x, ir3, a.x);
        a.y = fmaf(sv.y, ir3, a.y);
        a.z = fmaf(sv.z, ir3, a.z);
        a.u = fmaf(dx, k5, a.u);
        a.v = fmaf(dy, k5, a.v);
        a.q = fmaf(dz, k5, a.q);
    } else {   // paper-mode A^T: -s d / r^3
        float q = -sv.x * (ir * ir * ir);
        a.x = fmaf(q, dx, a.x);
        a.y = fmaf(q, dy, a.y);
        a.z = fmaf(q, dz, a.z);
    }
}

// Two targets' accumulators of the fused A and G sums, packed in float2
// halves (.x: first target, .y: second), for the paired FP32 instructions of
// sm_100 and later (two lanes of FP32 work per issued instruction).
struct Acc2 {
    float2 x = {0.f, 0.f}, y = {0.f, 0.f}, z = {0.f, 0.f};
    float2 u = {0.f, 0.f}, v = {0.f, 0.f}, q = {0.f, 0.f};
    float2 s = {0.f, 0.f};
};

// The pair term of interact<OP, CUT> for two targets at once: (ntx, nty,
// ntz) are the targets' negated coordinates.  The same operations in the same
// order as the scalar form, so each half is bit-identical to it.
template <int OP, bool CUT>
__device__ __forceinline__ void interact2(const float2& ntx, const float2& nty, const float2& ntz,
                                          const float4& sp, const float4& sv, float w2, Acc2& a) {
    const float2 dx = __fadd2_rn(make_float2(sp.x, sp.x), ntx);
    const float2 dy = __fadd2_rn(make_float2(sp.y, sp.y), nty);
    const float2 dz = __fadd2_rn(make_float2(sp.z, sp.z), ntz);
    float2 r2 = __fmul2_rn(dz, dz);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dx, dx, r2);
    float2 ir = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    if (CUT) {
        ir.x = (r2.x >= w2) ? ir.x : 0.f;
        ir.y = (r2.y >= w2) ? ir.y : 0.f;
    }
    const float2 vx = make_float2(sv.x, sv.x);
    if (OP == kOpA) {
        const float2 ir3 = __fmul2_rn(__fmul2_rn(ir, ir), ir);
        const float2 vy = make_float2(sv.y, sv.y), vz = make_float2(sv.z, sv.z);
        float2 dm = __fmul2_rn(dz, vz);
        dm = __ffma2_rn(dy, vy, dm);
        dm = __ffma2_rn(dx, vx, dm);
        a.x = __ffma2_rn(dm, ir3, a.x);
    } else if (OP == kOpG || OP == kOpAG) {
        const float2 ir2 = __fmul2_rn(ir, ir);
        const float2 ir3 = __fmul2_rn(ir2, ir);
        const float2 vy = make_float2(sv.y, sv.y), vz = make_float2(sv.z, sv.z);
        float2 dm = __fmul2_rn(dz, vz);
        dm = __ffma2_rn(dy, vy, dm);
        dm = __ffma2_rn(dx, vx, dm);
        const float2 k5 = __fmul2_rn(__fmul2_rn(dm, ir2), ir3);
        if (OP == kOpAG) a.s = __ffma2_rn(dm, ir3, a.s);
        a.x = __ffma2_rn(vx, ir3, a.x);
        a.y = __ffma2_rn(vy, ir3, a.y);
        a.z = __ffma2_rn(vz, ir3, a.z);
        a.u = __ffma2_rn(dx, k5, a.u);
        a.v = __ffma2_rn(dy, k5, a.v);
        a.q = __ffma2_rn(dz, k5, a.q);
    } else {   // paper-mode A^T: -s d / r^3
        const float2 q = __fmul2_rn(make_float2(-sv.x, -sv.x), __fmul2_rn(__fmul2_rn(ir, ir), ir));
        a.x = __ffma2_rn(q, dx, a.x);
        a.y = __ffma2_rn(q, dy, a.y);
        a.z = __ffma2_rn(q, dz, a.z);
    }
}

// Shift a point stored in chunk frame `c` into the frame with origin `o`
// (both origins are multiples of 2^-12, so the shift is exact).
__device__ __forceinline__ float4 shift(const float4& c, const float4& o, const float4& p) {
    return make_float4((c.x - o.x) + p.x, (c.y - o.y) + p.y, (c.z - o.z) + p.z, 0.f);
}

// A point rounded to bfloat16 per coordinate (the near-field precision study).
__device__ __forceinline__ float4 bf16_point(const float4& p) {
    return make_float4(__bfloat162float(__float2bfloat16_rn(p.x)), __bfloat162float(__float2bfloat16_rn(p.y)),
                       __bfloat162float(__float2bfloat16_rn(p.z)), p.w);
}

// Squared distance from p to the box [lo, hi] (zero inside).
__device__ __forceinline__ float box_gap2(const float4& lo, const float4& hi, const float4& p) {
    const float ex = fmaxf(fmaxf(lo.x - p.x, p.x - hi.x), 0.f);
    const float ey = fmaxf(fmaxf(lo.y - p.y, p.y - hi.y), 0.f);
    const float ez = fmaxf(fmaxf(lo.z - p.z, p.z - hi.z), 0.f);
    return fmaf(ex, ex, fmaf(ey, ey, ez * ez));
}

// G's two partial sums combined: (x, y, z) - 3 (u, v, q).
template <int OP>
__device__ __forceinline__ Acc3 combine(Acc3 a) {
    if (OP == kOpG || OP == kOpAG) {
        a.x = fmaf(-3.f, a.u, a.x);
        a.y = fmaf(-3.f, a.v, a.y);
        a.z = fmaf(-3.f, a.q, a.z);
    }
    return a;
}

// Epilogue of one group (all 32 lanes call it; lane < size holds target i).
template <int EPI>
__device__ __forceinline__ void gather_epilogue(const GatherArgs& A, int g, int64_t i, bool valid,
                                                Acc3 acc, int lane) {
    double part = 0.0;
    // far_order 1: the first-order far terms of the target, summed over its
    // group's far list by k_far_dip (same units as the sums here)
    if (A.dip_corr && valid) {
        const float4 c = A.dip_corr[i];
        if (EPI == kEpiStoreW || EPI == kEpiResidual || EPI == kEpiNormSq) {
            acc.x += c.w;
        } else if (EPI == kEpiStoreGrad || EPI == kEpiRescale) {
            acc.x += c.x; acc.y += c.y; acc.z += c.z;
        } else if (EPI == kEpiResidualAG || EPI == kEpiNormSqAG) {
            acc.s += c.w;
            acc.x += c.x; acc.y += c.y; acc.z += c.z;
        }
    }
    if (EPI == kEpiStoreW) {
        if (valid) A.out[A.tperm[i]] = acc.x * kInv4Pi;
    } else if (EPI == kEpiStoreGrad || EPI == kEpiStoreATpaper) {
        if (valid) {
            const float f = (EPI == kEpiStoreGrad ? -kInv4Pi : kInv4Pi) * A.scale;
            const int64_t o3 = 3 * A.tperm[i];
            A.out[o3] = acc.x * f;
            A.out[o3 + 1] = acc.y * f;
            A.out[o3 + 2] = acc.z * f;
        }
    } else if (EPI == kEpiResidual) {
        if (valid) {
            const float sres = 0.5f - acc.x * kInv4Pi;
            A.s_out[i] = sres;
            part = (double)sres * (double)sres;
        }
    } else if (EPI == kEpiNormSq) {
        if (valid) {
            const float v = acc.x * kInv4Pi;
            part = (double)v * (double)v;
        }
    } else if (EPI == kEpiRescale) {
        if (valid) {
            const float gx = acc.x * kInv4Pi, gy = acc.y * kInv4Pi, gz = acc.z * kInv4Pi;
            const float4 mc = A.mu_cur[i];
            const float hn = sqrtf(gx * gx + gy * gy + gz * gz);
            float4 res = mc;
            if (hn > 0.f) {
                const float len = A.rescale_mode == 1 ? A.area[i] : sqrtf(mc.x * mc.x + mc.y * mc.y + mc.z * mc.z);
                const float f = len / hn;
                res = make_float4(gx * f, gy * f, gz * f, 0.f);
            }
            A.mu_out[i] = res;
        }
    } else if (EPI == kEpiStoreR) {
        if (valid) {
            const float4 v = make_float4(acc.x * kInv4Pi, acc.y * kInv4Pi, acc.z * kInv4Pi, 0.f);
            A.mu_out[i] = v;
            part = (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z;
        }
    } else if (EPI == kEpiResidualAG || EPI == kEpiNormSqAG) {
        if (valid) {
            const float f = acc.s * kInv4Pi;
            if (EPI == kEpiResidualAG) {
                const float sres = 0.5f - f;
                A.s_out[i] = sres;
                part = (double)sres * (double)sres;
            } else {
                part = (double)f * (double)f;
            }
            A.g_out[i] = make_float4(acc.x * kInv4Pi, acc.y * kInv4Pi, acc.z * kInv4Pi, 0.f);
        }
    }
    if (EPI == kEpiResidual || EPI == kEpiNormSq || EPI == kEpiStoreR || EPI == kEpiResidualAG ||
        EPI == kEpiNormSqAG) {
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o2);
        if (lane == 0) A.partial[g] = part;
    }
}

// A group cut into several work items: each item stores its part (one
// float4 per lane), and the item that finishes last adds all parts in order
// (part 0 first) and runs the group's epilogue.  Returns true in the warp of
// that item.  Each lane fences its store before lane 0 counts the part in; the
// last item resets the counter for the next launch.
__device__ __forceinline__ bool last_part(unsigned* cnt, int split, int nparts, int lane) {
    __threadfence();
    __syncwarp();
    unsigned tk = 0;
    if (lane == 0) tk = atomicAdd(cnt + split, 1u);
    tk = __shfl_sync(0xffffffffu, tk, 0);
    const bool last = tk == (unsigned)nparts - 1u;
    if (last && lane == 0) cnt[split] = 0u;
    return last;
}

// One warp per work item (a target group's near ranges and far entries).
// Sources are staged 32 at a time in shared memory, and the loads of the
// next batch are issued before the current batch is summed, so that their
// latency overlaps the arithmetic.
//   * Near sources: the item's ranges (about ten points on average) form one
//     stream cut into full batches of 32.  Lanes read 32 ranges at once; a
//     lane finds the range of its stream position by a binary search over the
//     ranges' prefix sums (shuffles).
//   * Far entries: the node ids of batch k + 2 and the node data of batch
//     k + 1 are read while batch k is summed.
// TPL targets per lane: with TPL = 2, lanes h*16 + k (h = 0, 1) hold targets
// k and k + 16 of the group and take the staged sources of index h, h + 2,
// ...; each source load then serves two pair terms, and the two halves' sums
// are added once per item.  NB: the near-field bfloat16 study (a template
// parameter, so that the default kernel carries no trace of it).
template <int OP, int EPI, bool NB, int TPL>
__global__ void WNNC_CAPPED_BOUNDS k_gather(GatherArgs A) {
    static_assert(TPL == 1 || TPL == 2, "one or two targets per lane");
    constexpr int kLanesPerStream = 32 / TPL;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ float4 sp_all[kGatherWarps][32];
    __shared__ float4 sv_all[kGatherWarps][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x * kGatherWarps + wl;
    if (it >= A.nitems) return;
    float4* sp = sp_all[wl];
    float4* sv = sv_all[wl];
    const Item item = A.items[it];
    const int g = item.g;
    const int i0 = A.goff[g];
    const int gsize = A.goff[g + 1] - i0;
    const float4 o = A.tgorig[g];
    const int h = lane / kLanesPerStream;      // source stream of this lane
    const int tl = lane % kLanesPerStream;
    float4 t[TPL], tn[TPL];                    // tn: the target as the near field sees it
    Acc3 acc[TPL];
#pragma unroll
    for (int u = 0; u < TPL; ++u) {
        const int k = tl + u * kLanesPerStream;
        const int64_t i = (int64_t)i0 + k;
        t[u] = k < gsize ? shift(A.tcorig[i >> 5], o, A.tpos[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
        tn[u] = NB ? bf16_point(t[u]) : t[u];
    }
    const float4 blo = A.tgbl[g], bhi = A.tgbh[g];
    // two targets per lane: paired FP32 instructions
    constexpr bool kPack = TPL == 2;
    Acc2 acc2;
    const float2 ntx = make_float2(-t[0].x, -t[TPL - 1].x), nty = make_float2(-t[0].y, -t[TPL - 1].y),
                 ntz = make_float2(-t[0].z, -t[TPL - 1].z);
    const float2 nnx = make_float2(-tn[0].x, -tn[TPL - 1].x), nny = make_float2(-tn[0].y, -tn[TPL - 1].y),
                 nnz = make_float2(-tn[0].z, -tn[TPL - 1].z);

    // the sums of one staged batch of cnt sources against this lane's targets
    auto sum_batch = [&](int cnt, bool clear, bool near) {
        if (kPack) {
            const float2 &ax = near ? nnx : ntx, &ay = near ? nny : nty, &az = near ? nnz : ntz;
            if (cnt == 32) {
                // a full batch (almost all of them): a compile-time trip count, no bounds guards
                if (clear) {
#pragma unroll
                    for (int j = 0; j < 32 / TPL; ++j)
                        interact2<OP, false>(ax, ay, az, sp[h + TPL * j], sv[h + TPL * j], A.w2, acc2);
                } else {
#pragma unroll
                    for (int j = 0; j < 32 / TPL; ++j)
                        interact2<OP, true>(ax, ay, az, sp[h + TPL * j], sv[h + TPL * j], A.w2, acc2);
                }
                return;
            }
            if (clear) {
#pragma unroll kUnroll
                for (int k = h; k < cnt; k += TPL) interact2<OP, false>(ax, ay, az, sp[k], sv[k], A.w2, acc2);
            } else {
#pragma unroll kUnroll
                for (int k = h; k < cnt; k += TPL) interact2<OP, true>(ax, ay, az, sp[k], sv[k], A.w2, acc2);
            }
            return;
        }
        if (clear) {
#pragma unroll kUnroll
            for (int k = h; k < cnt; k += TPL) {
                const float4 p = sp[k], v = sv[k];
#pragma unroll
                for (int u = 0; u < TPL; ++u) interact<OP, false>(near ? tn[u] : t[u], p, v, A.w2, acc[u]);
            }
        } else {
#pragma unroll kUnroll
            for (int k = h; k < cnt; k += TPL) {
                const float4 p = sp[k], v = sv[k];
#pragma unroll
                for (int u = 0; u < TPL; ++u) interact<OP, true>(near ? tn[u] : t[u], p, v, A.w2, acc[u]);
            }
        }
    };
    // lane < cnt: stage the source held in registers (frame origin c, point p,
    // value v); returns whether every staged source clears the cut-off radius
    auto stage = [&](int cnt, const float4& c, const float4& pp, const float4& v, bool near) {
        bool clear = true;
        if (lane < cnt) {
            const float4 p = shift(c, o, pp);
            clear = box_gap2(blo, bhi, p) >= A.fast2;
            sp[lane] = (NB && near) ? bf16_point(p) : p;
            sv[lane] = v;
        }
        clear = __all_sync(kFull, clear);
        __syncwarp();
        return clear;
    };

    float4 my_c = make_float4(0.f, 0.f, 0.f, 0.f), my_p = my_c, my_v = my_c;

    // ---- near field ----
    {
        int qn = item.q0;                 // first range not yet in a window
        int wx = 0, wpre = 0;             // this lane's range in the window: start, stream offset
        int wn = 0, wtot = 0, cur = 0;    // ranges in the window, their points, stream position
        auto next_near = [&]() {
            int cnt = 0;
            while (cnt < 32) {
                if (cur == wtot) {
                    if (qn >= item.q1) break;
                    wn = min(32, item.q1 - qn);
                    int2 r = make_int2(0, 0);
                    if (lane < wn) r = A.near_rng[qn + lane];
                    const int len = r.y - r.x;
                    int inc = len;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int u = __shfl_up_sync(kFull, inc, d);
                        if (lane >= d) inc += u;
                    }
                    wx = r.x;
                    wpre = inc - len;
                    wtot = __shfl_sync(kFull, inc, 31);
                    qn += wn;
                    cur = 0;
                    continue;
                }
                const int take = min(32 - cnt, wtot - cur);
                const int x = cur + lane - cnt;           // stream position of this lane's slot
                int k = 0;                                // last range with wpre <= x
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int c = k + st;
                    const int pc = __shfl_sync(kFull, wpre, c & 31);
                    if (c < wn && pc <= x) k = c;
                }
                const int rx = __shfl_sync(kFull, wx, k), pk = __shfl_sync(kFull, wpre, k);
                if (lane >= cnt && lane < cnt + take) {
                    const int j = rx + (x - pk);
                    my_p = A.spos[j];
                    my_c = A.scorig[j >> 5];
                    if (OP == kOpATpaper) my_v = make_float4(A.sval_s[j], 0.f, 0.f, 0.f);
                    else my_v = A.sval[j];
                }
                cnt += take;
                cur += take;
            }
            return cnt;
        };
        int cnt = next_near();
        while (cnt > 0) {
            const bool clear = stage(cnt, my_c, my_p, my_v, true);
            const int cnt_next = next_near();
            sum_batch(cnt, clear, true);
            __syncwarp();
            cnt = cnt_next;
        }
    }

    // ---- far field: node representatives ----
    if (item.f0 < item.f1) {
        int cnt = min(32, item.f1 - item.f0);
        if (lane < cnt) {
            const int b = A.far_id[item.f0 + lane];
            my_p = A.nrep[b];
            my_c = A.ncell[b];
            my_v = A.nmom[b];
        }
        int b_next = 0;                   // node ids one batch ahead of the data
        if (lane < min(32, item.f1 - item.f0 - 32)) b_next = A.far_id[item.f0 + 32 + lane];
        for (int base = item.f0; base < item.f1; base += 32) {
            const bool clear = stage(cnt, my_c, my_p, my_v, false);
            const int cnt_next = min(32, item.f1 - base - 32);   // <= 0 after the last batch
            if (lane < cnt_next) {
                my_p = A.nrep[b_next];
                my_c = A.ncell[b_next];
                my_v = A.nmom[b_next];
            }
            if (lane < min(32, item.f1 - base - 64)) b_next = A.far_id[base + 64 + lane];
            sum_batch(cnt, clear, false);
            __syncwarp();
            cnt = cnt_next;
        }
    }

    if (kPack) {
#pragma unroll
        for (int u = 0; u < TPL; ++u) {
            acc[u].x = u == 0 ? acc2.x.x : acc2.x.y;
            acc[u].y = u == 0 ? acc2.y.x : acc2.y.y;
            acc[u].z = u == 0 ? acc2.z.x : acc2.z.y;
            acc[u].u = u == 0 ? acc2.u.x : acc2.u.y;
            acc[u].v = u == 0 ? acc2.v.x : acc2.v.y;
            acc[u].q = u == 0 ? acc2.q.x : acc2.q.y;
            acc[u].s = u == 0 ? acc2.s.x : acc2.s.y;
        }
    }
    Acc3 mine = acc[0];
    if (TPL == 2) {
        // add the other source stream's sums; lane l then keeps target l
#pragma unroll
        for (int u = 0; u < TPL; ++u) {
            acc[u].x += __shfl_xor_sync(kFull, acc[u].x, 16);
            acc[u].y += __shfl_xor_sync(kFull, acc[u].y, 16);
            acc[u].z += __shfl_xor_sync(kFull, acc[u].z, 16);
            acc[u].u += __shfl_xor_sync(kFull, acc[u].u, 16);
            acc[u].v += __shfl_xor_sync(kFull, acc[u].v, 16);
            acc[u].q += __shfl_xor_sync(kFull, acc[u].q, 16);
            acc[u].s += __shfl_xor_sync(kFull, acc[u].s, 16);
        }
        mine = h == 0 ? acc[0] : acc[TPL - 1];
    }
    mine = combine<OP>(mine);
    const int64_t i = (int64_t)i0 + lane;
    const bool valid = lane < gsize;
    if (item.pslot >= 0) {
        A.part_acc[(int64_t)item.pslot * 32 + lane] = make_float4(mine.x, mine.y, mine.z, mine.s);
    } else if (A.raw) {
        if (valid) A.raw[i] = make_float4(mine.x, mine.y, mine.z, mine.s);
    } else {
        gather_epilogue<EPI>(A, g, i, valid, mine, lane);
    }
}

// Groups cut into several items: add the parts in order, then the epilogue.
// (A separate launch: finishing a group inside the gather by its last item
// cost the gather more under its register cap than the launch it saves.)
template <int EPI>
__global__ void k_gather_finalize(GatherArgs A) {
    const int sidx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sidx >= A.nsplit) return;
    const int4 sp = A.splits[sidx];
    const int g = sp.x;
    Acc3 acc;
    for (int p = 0; p < sp.z; ++p) {
        const float4 v = A.part_acc[(int64_t)(sp.y + p) * 32 + lane];
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.s += v.w;
    }
    const int i0 = A.goff[g];
    gather_epilogue<EPI>(A, g, (int64_t)i0 + lane, lane < A.goff[g + 1] - i0, acc, lane);
}

// ---------------------------------------------------------------------------
// Far entries expanded about the target group's centre (local_theta > 0).
// One warp per target group (kLocalWarps groups per block); the lanes take
// the group's expanded entries [lsplit[g], far_off[g + 1]) two at a time
// (entries base + lane and base + 32 + lane), the next two nodes' 32-byte
// records (centroid and moment, one sector) read while these are summed.
// With E = x_B - c_g (group frame) and M the node's moment, in the units of
// the gather's sums (4 pi times the operator), each entry adds the value of
// A, the value of G and the Jacobian of G at c_g:
//   a = (E.M)/r^3,  g = M/r^3 - 3 (E.M) E/r^5,
//   J = 3 (M E^T + E M^T + (E.M) I)/r^5 - 15 (E.M) E E^T/r^7,
// so that a target at c_g + d gets A = a - d.g and G = g + J d (G = -grad A,
// first-order Taylor expansion of both about c_g).  When both entries of a
// lane pass, their terms run in the two halves of paired FP32 instructions.
// An entry whose pairs may straddle the cut-off (|E| - rho_g < w) is queued
// and summed pair by pair with the cut-off instead (from the node's exact
// cell-relative data), every lane taking one target.  Each target's result
// goes to corr (G x, y, z, A), which the gather's epilogue adds.
// ---------------------------------------------------------------------------
constexpr int kLocalWarps = 4;

// Node centroids in normalised coordinates (cell centre + offset, rounded to
// float): the expansions need them to about 1e-7 only, far from the group.
__global__ void k_node_abs(int nn, const float4* ncell, const float4* ncent, float4* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nn) return;
    const float4 c = ncell[b], d = ncent[b];
    out[b] = make_float4(c.x + d.x, c.y + d.y, c.z + d.z, 0.f);
}

// Per node one 32-byte record of the centroid and this call's moment.
__global__ void k_local_pack(int nn, const float4* nabs, const float4* mom, float4* rec) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nn) return;
    const float4 x = nabs[b], m = mom[b];
    rec[2 * b] = make_float4(x.x, x.y, x.z, m.x);
    rec[2 * b + 1] = make_float4(m.y, m.z, 0.f, 0.f);
}

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// The expansion accumulators of one lane: two halves per coefficient (added
// at the end), (a, g_x, g_y, g_z, J_xx, J_yy, J_zz, J_xy, J_xz, J_yz).
struct LocalAcc {
    float2 c[10];
};

// One or two entries' terms (halves .x, .y; a half with keep = 0 adds nothing).
template <bool kG>
__device__ __forceinline__ void local_terms(const float2& ex, const float2& ey, const float2& ez, const float2& ir,
                                            const float2& mx, const float2& my, const float2& mz, LocalAcc& L) {
    const float2 ir2 = __fmul2_rn(ir, ir), ir3 = __fmul2_rn(ir2, ir), ir5 = __fmul2_rn(ir3, ir2);
    float2 em = __fmul2_rn(ez, mz);
    em = __ffma2_rn(ey, my, em);
    em = __ffma2_rn(ex, mx, em);
    const float2 emr5 = __fmul2_rn(em, ir5);
    const float2 k3n = __fmul2_rn(emr5, f2(-3.f));                  // -3 (E.M)/r^5
    L.c[0] = __ffma2_rn(em, ir3, L.c[0]);
    L.c[1] = __ffma2_rn(k3n, ex, __ffma2_rn(mx, ir3, L.c[1]));
    L.c[2] = __ffma2_rn(k3n, ey, __ffma2_rn(my, ir3, L.c[2]));
    L.c[3] = __ffma2_rn(k3n, ez, __ffma2_rn(mz, ir3, L.c[3]));
    if (kG) {
        const float2 t3 = __fmul2_rn(ir5, f2(3.f));
        const float2 t15n = __fmul2_rn(__fmul2_rn(emr5, ir2), f2(-15.f));   // -15 (E.M)/r^7
        const float2 vx = __fmul2_rn(t15n, ex), vy = __fmul2_rn(t15n, ey), vz = __fmul2_rn(t15n, ez);
        L.c[4] = __ffma2_rn(vx, ex, __ffma2_rn(t3, __ffma2_rn(__fadd2_rn(mx, mx), ex, em), L.c[4]));
        L.c[5] = __ffma2_rn(vy, ey, __ffma2_rn(t3, __ffma2_rn(__fadd2_rn(my, my), ey, em), L.c[5]));
        L.c[6] = __ffma2_rn(vz, ez, __ffma2_rn(t3, __ffma2_rn(__fadd2_rn(mz, mz), ez, em), L.c[6]));
        L.c[7] = __ffma2_rn(vx, ey, __ffma2_rn(t3, __ffma2_rn(mx, ey, __fmul2_rn(my, ex)), L.c[7]));
        L.c[8] = __ffma2_rn(vx, ez, __ffma2_rn(t3, __ffma2_rn(mx, ez, __fmul2_rn(mz, ex)), L.c[8]));
        L.c[9] = __ffma2_rn(vy, ez, __ffma2_rn(t3, __ffma2_rn(my, ez, __fmul2_rn(mz, ey)), L.c[9]));
    }
}

template <int OP>
__global__ void __launch_bounds__(32 * kLocalWarps) k_local_ag(GatherArgs A, float4* corr) {
    constexpr bool kG = OP == kOpG || OP == kOpAG;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ int qb_all[kLocalWarps][32];                // queued entries' nodes
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * kLocalWarps + wl;
    if (g >= A.ngroups) return;
    int* qb = qb_all[wl];
    const int i0 = A.goff[g], gsize = A.goff[g + 1] - i0;
    const float4 o = A.tgorig[g];
    const float4 cg = A.gctr[g];
    const int64_t it = (int64_t)i0 + lane;
    const float4 tl = lane < gsize ? shift(A.tcorig[it >> 5], o, A.tpos[it]) : make_float4(0.f, 0.f, 0.f, 0.f);
    const int w0 = A.lsplit[g], w1 = A.csplit ? A.csplit[g] : A.far_off[g + 1];
    LocalAcc L;
#pragma unroll
    for (int q = 0; q < 10; ++q) L.c[q] = make_float2(0.f, 0.f);
    float4 fs = make_float4(0.f, 0.f, 0.f, 0.f);           // this lane's target: queued pair sums (G, A)
    int nq = 0;                                             // entries queued
    // the queued entries' pair terms at this lane's target, with the cut-off
    auto flush = [&]() {
        for (int k = 0; k < nq; ++k) {
            const int b = qb[k];
            const float4 p = shift(A.ncell[b], o, A.nrep[b]), m = A.nmom[b];
            const float dx = p.x - tl.x, dy = p.y - tl.y, dz = p.z - tl.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ir = r2 >= A.w2 ? rsqrtf(r2) : 0.f;
            const float ir2 = ir * ir, ir3 = ir2 * ir;
            const float dm = fmaf(dx, m.x, fmaf(dy, m.y, dz * m.z));
            const float k5 = 3.f * (dm * ir2) * ir3;
            fs.w = fmaf(dm, ir3, fs.w);
            fs.x += fmaf(m.x, ir3, -k5 * dx);
            fs.y += fmaf(m.y, ir3, -k5 * dy);
            fs.z += fmaf(m.z, ir3, -k5 * dz);
        }
        __syncwarp();
        nq = 0;
    };
    auto queue = [&](bool fall, int b) {
        const unsigned fm = __ballot_sync(kFull, fall);
        if (!fm) return;
        const int nf = __popc(fm);
        if (nq + nf > 32) flush();
        if (fall) qb[nq + __popc(fm & ((1u << lane) - 1u))] = b;
        nq += nf;
        __syncwarp();
    };
    // node records one step ahead, node ids two steps ahead
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
    int ia = 0, ib = 0, na = 0, nb = 0;
    if (w0 + lane < w1) { ia = A.far_id[w0 + lane]; a0 = A.lrec[2 * ia]; a1 = A.lrec[2 * ia + 1]; }
    if (w0 + 32 + lane < w1) { ib = A.far_id[w0 + 32 + lane]; b0 = A.lrec[2 * ib]; b1 = A.lrec[2 * ib + 1]; }
    if (w0 + 64 + lane < w1) na = A.far_id[w0 + 64 + lane];
    if (w0 + 96 + lane < w1) nb = A.far_id[w0 + 96 + lane];
    for (int base = w0; base < w1; base += 64) {
        const int ea = base + lane, eb = ea + 32;
        const bool va = ea < w1, vb = eb < w1;
        const float2 ex = __fadd2_rn(make_float2(a0.x, b0.x), f2(-(o.x + cg.x)));
        const float2 ey = __fadd2_rn(make_float2(a0.y, b0.y), f2(-(o.y + cg.y)));
        const float2 ez = __fadd2_rn(make_float2(a0.z, b0.z), f2(-(o.z + cg.z)));
        const float2 mx = make_float2(a0.w, b0.w), my = make_float2(a1.x, b1.x), mz = make_float2(a1.y, b1.y);
        const int ca = ia, cb = ib;
        if (ea + 64 < w1) { ia = na; a0 = A.lrec[2 * ia]; a1 = A.lrec[2 * ia + 1]; }
        if (eb + 64 < w1) { ib = nb; b0 = A.lrec[2 * ib]; b1 = A.lrec[2 * ib + 1]; }
        if (ea + 128 < w1) na = A.far_id[ea + 128];
        if (eb + 128 < w1) nb = A.far_id[eb + 128];
        float2 r2 = __fmul2_rn(ez, ez);
        r2 = __ffma2_rn(ey, ey, r2);
        r2 = __ffma2_rn(ex, ex, r2);
        float2 ir = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 bound = __ffma2_rn(r2, ir, f2(-cg.w));     // |E| - rho_g
        const bool oka = va && bound.x > 0.f && bound.x * bound.x >= A.w2;
        const bool okb = vb && bound.y > 0.f && bound.y * bound.y >= A.w2;
        // a half that is invalid or queued adds nothing (1/r = 0 zeroes each of its terms)
        ir = make_float2(oka ? ir.x : 0.f, okb ? ir.y : 0.f);
        local_terms<kG>(ex, ey, ez, ir, mx, my, mz, L);
        queue(va && !oka, ca);
        queue(vb && !okb, cb);
    }
    if (nq) flush();
    float k[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        k[q] = L.c[q].x + L.c[q].y;
        if (q < 4 || kG) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) k[q] += __shfl_xor_sync(kFull, k[q], d);
        }
    }
    const float dx = tl.x - cg.x, dy = tl.y - cg.y, dz = tl.z - cg.z;
    float4 f = fs;
    f.w += k[0] - fmaf(dx, k[1], fmaf(dy, k[2], dz * k[3]));
    if (kG) {
        f.x += k[1] + fmaf(k[4], dx, fmaf(k[7], dy, k[8] * dz));
        f.y += k[2] + fmaf(k[7], dx, fmaf(k[5], dy, k[9] * dz));
        f.z += k[3] + fmaf(k[8], dx, fmaf(k[9], dy, k[6] * dz));
    }
    if (lane < gsize) corr[i0 + lane] = f;
}

// The second level (local_cluster = K): one warp per cluster of K consecutive
// groups, over the entries expanded about the cluster's centre (the first
// member's part from csplit on; every member lists the same nodes).  The same
// terms as k_local_ag about the cluster's centre c_C, evaluated at each of the
// cluster's up to 32 K targets (lane l takes targets l, l + 32, ...) and added
// to corr; an entry whose pairs may straddle the cut-off (|E| - rho_C < w) is
// queued and summed pair by pair at every target of the cluster.
template <int OP>
__global__ void __launch_bounds__(32 * kLocalWarps) k_local_cl(GatherArgs A, float4* corr) {
    constexpr bool kG = OP == kOpG || OP == kOpAG;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ float4 tq_all[kLocalWarps][32 * kMaxCluster];   // targets in the cluster's frame
    __shared__ float4 fs_all[kLocalWarps][32 * kMaxCluster];   // queued entries' pair sums (G, A)
    __shared__ int qb_all[kLocalWarps][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = blockIdx.x * kLocalWarps + wl;
    if (C >= A.nclusters) return;
    const int K = A.cluster_k;
    const int g0 = C * K, g1 = min(g0 + K, A.ngroups);
    const int i0 = A.goff[g0], nt = A.goff[g1] - i0;
    const float4 o = A.cctr[C];
    const float4 cg = A.cexp[C];
    float4* tq = tq_all[wl];
    float4* fsum = fs_all[wl];
    int* qb = qb_all[wl];
    for (int k = lane; k < nt; k += 32) {
        const int64_t i = (int64_t)i0 + k;
        tq[k] = shift(A.tcorig[i >> 5], o, A.tpos[i]);
        fsum[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    const int w0 = A.csplit[g0], w1 = A.far_off[g0 + 1];
    LocalAcc L;
#pragma unroll
    for (int q = 0; q < 10; ++q) L.c[q] = make_float2(0.f, 0.f);
    int nq = 0;
    auto flush = [&]() {
        for (int k = lane; k < nt; k += 32) {
            const float4 tl = tq[k];
            float4 fs = fsum[k];
            for (int j = 0; j < nq; ++j) {
                const int b = qb[j];
                const float4 p = shift(A.ncell[b], o, A.nrep[b]), m = A.nmom[b];
                const float dx = p.x - tl.x, dy = p.y - tl.y, dz = p.z - tl.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float ir = r2 >= A.w2 ? rsqrtf(r2) : 0.f;
                const float ir2 = ir * ir, ir3 = ir2 * ir;
                const float dm = fmaf(dx, m.x, fmaf(dy, m.y, dz * m.z));
                const float k5 = 3.f * (dm * ir2) * ir3;
                fs.w = fmaf(dm, ir3, fs.w);
                fs.x += fmaf(m.x, ir3, -k5 * dx);
                fs.y += fmaf(m.y, ir3, -k5 * dy);
                fs.z += fmaf(m.z, ir3, -k5 * dz);
            }
            fsum[k] = fs;
        }
        __syncwarp();
        nq = 0;
    };
    auto queue = [&](bool fall, int b) {
        const unsigned fm = __ballot_sync(kFull, fall);
        if (!fm) return;
        const int nf = __popc(fm);
        if (nq + nf > 32) flush();
        if (fall) qb[nq + __popc(fm & ((1u << lane) - 1u))] = b;
        nq += nf;
        __syncwarp();
    };
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
    int ia = 0, ib = 0, na = 0, nb = 0;
    if (w0 + lane < w1) { ia = A.far_id[w0 + lane]; a0 = A.lrec[2 * ia]; a1 = A.lrec[2 * ia + 1]; }
    if (w0 + 32 + lane < w1) { ib = A.far_id[w0 + 32 + lane]; b0 = A.lrec[2 * ib]; b1 = A.lrec[2 * ib + 1]; }
    if (w0 + 64 + lane < w1) na = A.far_id[w0 + 64 + lane];
    if (w0 + 96 + lane < w1) nb = A.far_id[w0 + 96 + lane];
    for (int base = w0; base < w1; base += 64) {
        const int ea = base + lane, eb = ea + 32;
        const bool va = ea < w1, vb = eb < w1;
        const float2 ex = __fadd2_rn(make_float2(a0.x, b0.x), f2(-(o.x + cg.x)));
        const float2 ey = __fadd2_rn(make_float2(a0.y, b0.y), f2(-(o.y + cg.y)));
        const float2 ez = __fadd2_rn(make_float2(a0.z, b0.z), f2(-(o.z + cg.z)));
        const float2 mx = make_float2(a0.w, b0.w), my = make_float2(a1.x, b1.x), mz = make_float2(a1.y, b1.y);
        const int ca = ia, cb = ib;
        if (ea + 64 < w1) { ia = na; a0 = A.lrec[2 * ia]; a1 = A.lrec[2 * ia + 1]; }
        if (eb + 64 < w1) { ib = nb; b0 = A.lrec[2 * ib]; b1 = A.lrec[2 * ib + 1]; }
        if (ea + 128 < w1) na = A.far_id[ea + 128];
        if (eb + 128 < w1) nb = A.far_id[eb + 128];
        float2 r2 = __fmul2_rn(ez, ez);
        r2 = __ffma2_rn(ey, ey, r2);
        r2 = __ffma2_rn(ex, ex, r2);
        float2 ir = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 bound = __ffma2_rn(r2, ir, f2(-cg.w));     // |E| - rho_C
        const bool oka = va && bound.x > 0.f && bound.x * bound.x >= A.w2;
        const bool okb = vb && bound.y > 0.f && bound.y * bound.y >= A.w2;
        ir = make_float2(oka ? ir.x : 0.f, okb ? ir.y : 0.f);
        local_terms<kG>(ex, ey, ez, ir, mx, my, mz, L);
        queue(va && !oka, ca);
        queue(vb && !okb, cb);
    }
    if (nq) flush();
    float k[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        k[q] = L.c[q].x + L.c[q].y;
        if (q < 4 || kG) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) k[q] += __shfl_xor_sync(kFull, k[q], d);
        }
    }
    for (int j = lane; j < nt; j += 32) {
        const float4 tl = tq[j];
        const float dx = tl.x - cg.x, dy = tl.y - cg.y, dz = tl.z - cg.z;
        float4 f = fsum[j];
        f.w += k[0] - fmaf(dx, k[1], fmaf(dy, k[2], dz * k[3]));
        if (kG) {
            f.x += k[1] + fmaf(k[4], dx, fmaf(k[7], dy, k[8] * dz));
            f.y += k[2] + fmaf(k[7], dx, fmaf(k[5], dy, k[9] * dz));
            f.z += k[3] + fmaf(k[8], dx, fmaf(k[9], dy, k[6] * dz));
        }
        const float4 c = corr[i0 + j];
        corr[i0 + j] = make_float4(c.x + f.x, c.y + f.y, c.z + f.z, c.w + f.w);
    }
}

// Every group's epilogue after a gather that left its sums in A.raw (groups
// not cut) or in the part slots (cut groups, added in order): warp per group.
template <int EPI>
__global__ void k_gather_finalize_all(GatherArgs A) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= A.ngroups) return;
    const int i0 = A.goff[g];
    const bool valid = lane < A.goff[g + 1] - i0;
    Acc3 acc;
    const int sp = A.gsplit[g];
    if (sp >= 0) {
        const int4 r = A.splits[sp];
        for (int p = 0; p < r.z; ++p) {
            const float4 v = A.part_acc[(int64_t)(r.y + p) * 32 + lane];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.s += v.w;
        }
    } else if (valid) {
        const float4 v = A.raw[i0 + lane];
        acc.x = v.x;
        acc.y = v.y;
        acc.z = v.z;
        acc.s = v.w;
    }
    gather_epilogue<EPI>(A, g, (int64_t)i0 + lane, valid, acc, lane);
}

// ---------------------------------------------------------------------------
// The paper's treecode, Alg. 4 per target (tree parameter criterion = 1).
// One warp per target group, one target per lane, in the group's frame.
// Each lane walks the octree from the root on its own stack: node B is far
// for target x_i iff |x_i - x_B| > c width(B) (c = 1/theta, x_B the node's
// representative of this call, Eq. 13), and then contributes one term with
// nu_B (Eq. 14); else its children are visited; else (a leaf) its points
// are summed.  Every term takes the cut-off of Sec. 4.4.  The sums and the
// epilogues are the gather's.  With depth D <= 15 the stack holds at most
// 1 + 7 D entries; a push that would not fit sets the capacity flag and the
// lane drops that node (the result is then reported as an error, not used).
// ---------------------------------------------------------------------------
constexpr int kWalkStack = 128;

template <int OP, int EPI>
__global__ void __launch_bounds__(32 * kGatherWarps) k_walk(GatherArgs A) {
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * kGatherWarps + wl;
    if (g >= A.ngroups) return;
    const int i0 = A.goff[g], cnt = A.goff[g + 1] - i0;
    const int64_t i = (int64_t)i0 + lane;
    const bool valid = lane < cnt;
    const float4 o = A.tgorig[g];
    Acc3 acc;
    if (valid) {
        const float4 t = shift(A.tcorig[i >> 5], o, A.tpos[i]);
        int stk[kWalkStack];
        int sp = 0;
        stk[sp++] = 0;
        while (sp > 0) {
            const int b = stk[--sp];
            const float4 cell = A.ncell[b];
            const float4 rp = shift(cell, o, A.nrep[b]);
            const float dx = rp.x - t.x, dy = rp.y - t.y, dz = rp.z - t.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float cw = A.copen * cell.w;
            if (r2 > cw * cw) {
                const float4 nv = A.nmom[b];
                interact<OP, true>(t, rp, nv, A.w2, acc);
                continue;
            }
            const int nc = A.nnchild[b];
            if (nc > 0) {
                if (sp + nc > kWalkStack) {
                    atomicOr(A.err_flag, kErrCapacity);
                    continue;
                }
                const int c0 = A.nchild0[b];
                for (int q = nc - 1; q >= 0; --q) stk[sp++] = c0 + q;
                continue;
            }
            const int j0 = A.nstart[b], j1 = j0 + A.ncount[b];
            for (int j = j0; j < j1; ++j) {
                const float4 sp4 = shift(A.scorig[j >> 5], o, A.spos[j]);
                const float4 sv = OP == kOpATpaper ? make_float4(A.sval_s[j], 0.f, 0.f, 0.f) : A.sval[j];
                interact<OP, true>(t, sp4, sv, A.w2, acc);
            }
        }
    }
    gather_epilogue<EPI>(A, g, i, valid, combine<OP>(acc), lane);
}

// ---------------------------------------------------------------------------
// Exact adjoint of the rep_mode-1 tree operator A.
//   far:  contrib[e] = sum_{i in g} s_i (x_B - x_i) / r^3 for far entry e = (g, B)
//   node: vnode[B]   = sum of contrib over B's entries (ascending group)
//   near: per source chunk, gather over (target group, lane mask) entries, then
//         add the far sums of every node containing the point (walk to the root).
// ---------------------------------------------------------------------------
struct AdjArgs {
    const Item* items;
    int nitems;
    const int4* splits;
    unsigned* split_cnt;
    int nsplit;
    float4* part_acc;
    int64_t n;
    const int* goff;
    const float4* pos;
    const float4* corig;
    const float4* gorig;
    const float* sv;
    const int* far_id;
    const float4* ncell;
    const float4* ncent;
    float4* contrib;
    const int2* tnear_ent;
    const int2* near_rng;
    const int* rng_slot;
    float4* near_contrib;
    const int* leaf_of;
    const int* nparent;
    const float4* vnode;
    float w2;
    float fast2;              // squared batch-test radius (cut-off radius plus margin)
    const float4* gbl;        // group boxes in their own frames
    const float4* gbh;
    float scale;
    const int64_t* perm;
    float* out;
    float4* r_out;
    double* partial;
    const float4* hnode0;     // far_order 1: per node sum of s HPhi, (xx, yy, zz, -)
    const float4* hnode1;     //   and (xy, xz, yz, -)
    float4* contrib_h0;       // the same per far entry (k_adj_far_dip)
    float4* contrib_h1;
    const int* far_off;       // far list offsets per group
    const int* lsplit;        // local_theta > 0: first expanded far entry of each group
    const float4* gctr;       //   the expansion centre in the group's frame and the group's radius
    const float4* nabs;       //   per node the centroid in normalised coordinates
    int ngroups;
    int nnodes;
    const int* tfar_off;      // transposed far lists (node -> entries)
    const int* tfar_ent;      //   with local_theta > 0: class << 30 | id (0 the entry, 1 a group, 2 a cluster)
    float4* gadj;             //   per group (c_g, rho_g), (D, S), normalised coordinates
    float4* cadj;             //   local_cluster > 0: per cluster (c_C, rho_C), (D, S)
    int cluster_k;
    int nclusters;
    const float4* cctr;       //   cluster frame origins
    const float4* cexp;       //   expansion centre in the cluster's frame and the cluster's radius
};

// Adjoint terms s_i gradPhi(x_i - x) = s_i (x - x_i) / r^3 at x = p from a
// target (x_i, s_i), two at once with paired FP32 instructions: one point
// against two targets, or two points against one target ((tx, ty, tz) the
// negated target coordinates, tw the s).  In each half: d = p - x_i,
// r^2 = d.x^2 + (d.y^2 + d.z^2) by fma, ir = rsqrt(r^2) (0 where the cut-off
// drops the pair, CUT as in interact()), q = s_i ((ir ir) ir).  Returns q and
// d through the references; the caller accumulates q d.
template <bool CUT>
__device__ __forceinline__ void adj_term2(const float2& px, const float2& py, const float2& pz, const float2& tx,
                                          const float2& ty, const float2& tz, const float2& tw, float w2,
                                          float2& dx, float2& dy, float2& dz, float2& q) {
    dx = __fadd2_rn(px, tx);
    dy = __fadd2_rn(py, ty);
    dz = __fadd2_rn(pz, tz);
    float2 r2 = __fmul2_rn(dz, dz);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dx, dx, r2);
    float2 ir = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    if (CUT) {
        ir.x = (r2.x >= w2) ? ir.x : 0.f;
        ir.y = (r2.y >= w2) ? ir.y : 0.f;
    }
    q = __fmul2_rn(tw, __fmul2_rn(__fmul2_rn(ir, ir), ir));
}

// Far part, one warp per work item (a slice of one group's far entries):
// each lane takes two entries (nodes) of a batch of 64 and sums over the
// group's targets, staged once in shared memory, so that each target load
// serves two pair terms.  The node ids of batch k + 2 and the node centroids
// of batch k + 1 are read while batch k is summed.
__global__ void WNNC_ADJ_BOUNDS k_adj_far(AdjArgs A) {
    __shared__ float4 tp_all[kGatherWarps][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x * kGatherWarps + wl;
    if (it >= A.nitems) return;
    float4* tp = tp_all[wl];
    const Item item = A.items[it];
    const int g = item.g;
    const int i0 = A.goff[g], cnt_t = A.goff[g + 1] - i0;
    const int64_t i = (int64_t)i0 + lane;
    const float4 o = A.gorig[g];
    float4 p = lane < cnt_t ? shift(A.corig[i >> 5], o, A.pos[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    p.w = lane < cnt_t ? A.sv[i] : 0.f;
    tp[lane] = make_float4(-p.x, -p.y, -p.z, p.w);   // negated: the paired terms add them
    const float4 blo = A.gbl[g], bhi = A.gbh[g];
    __syncwarp();
    // this lane's entries of a batch at `base`: base + lane and base + 32 + lane
    float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), m0 = c0, c1 = c0, m1 = c0;   // cell origins, centroids
    int b0 = 0, b1 = 0;
    {
        const int e0 = item.f0 + lane, e1 = e0 + 32;
        if (e0 < item.f1) { const int b = A.far_id[e0]; c0 = A.ncell[b]; m0 = A.ncent[b]; }
        if (e1 < item.f1) { const int b = A.far_id[e1]; c1 = A.ncell[b]; m1 = A.ncent[b]; }
        if (e0 + 64 < item.f1) b0 = A.far_id[e0 + 64];
        if (e1 + 64 < item.f1) b1 = A.far_id[e1 + 64];
    }
    for (int base = item.f0; base < item.f1; base += 64) {
        const int e0 = base + lane, e1 = e0 + 32;
        const bool v0 = e0 < item.f1, v1 = e1 < item.f1;
        const float4 bp0 = shift(c0, o, m0), bp1 = shift(c1, o, m1);
        bool clear = (!v0 || box_gap2(blo, bhi, bp0) >= A.fast2) && (!v1 || box_gap2(blo, bhi, bp1) >= A.fast2);
        clear = __all_sync(0xffffffffu, clear);
        // next batch's centroids (ids read one batch earlier), then the ids after it
        if (e0 + 64 < item.f1) { c0 = A.ncell[b0]; m0 = A.ncent[b0]; }
        if (e1 + 64 < item.f1) { c1 = A.ncell[b1]; m1 = A.ncent[b1]; }
        if (e0 + 128 < item.f1) b0 = A.far_id[e0 + 128];
        if (e1 + 128 < item.f1) b1 = A.far_id[e1 + 128];
        // the two entries' sums in the halves of float2 (paired FP32 instructions)
        const float2 px = make_float2(bp0.x, bp1.x), py = make_float2(bp0.y, bp1.y), pz = make_float2(bp0.z, bp1.z);
        float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
        auto term = [&](const float4& tk, auto cut_tag) {
            constexpr bool CUT = decltype(cut_tag)::value;
            float2 dx, dy, dz, q;
            adj_term2<CUT>(px, py, pz, make_float2(tk.x, tk.x), make_float2(tk.y, tk.y), make_float2(tk.z, tk.z),
                           make_float2(tk.w, tk.w), A.w2, dx, dy, dz, q);
            ax = __ffma2_rn(q, dx, ax);
            ay = __ffma2_rn(q, dy, ay);
            az = __ffma2_rn(q, dz, az);
        };
        if (cnt_t == 32) {
            // a full group: a compile-time trip count, no bounds guards
            if (clear) {
#pragma unroll
                for (int k = 0; k < 32; ++k) term(tp[k], std::false_type{});
            } else {
#pragma unroll
                for (int k = 0; k < 32; ++k) term(tp[k], std::true_type{});
            }
        } else if (clear) {
#pragma unroll kUnroll
            for (int k = 0; k < cnt_t; ++k) term(tp[k], std::false_type{});
        } else {
#pragma unroll kUnroll
            for (int k = 0; k < cnt_t; ++k) term(tp[k], std::true_type{});
        }
        if (v0) A.contrib[e0] = make_float4(ax.x, ay.x, az.x, 0.f);
        if (v1) A.contrib[e1] = make_float4(ax.y, ay.y, az.y, 0.f);
    }
}

// Expanded far entries of the adjoint (local_theta > 0), the transpose of
// k_local_ag's expansion: with E = x_B - c_g, S = sum_i s_i and
// D = sum_i s_i (x_i - c_g) over group g, entry (g, B) adds to node B
//   S E/r^3 + (3 E (E.D) - r^2 D)/r^5
// (first order in x_i - c_g of sum_i s_i (x_B - x_i)/|x_B - x_i|^3), unless
// its pairs may straddle the cut-off (|E| - rho_g < w): then its pairs.
// k_local_records writes each group's (c_g, rho_g), (D, S) (and each
// cluster's); the node gather evaluates the expanded entries as it meets them.
__device__ __forceinline__ void local_group_record(const AdjArgs& A, int g, int lane) {
    const int i0 = A.goff[g], cnt_t = A.goff[g + 1] - i0;
    const float4 o = A.gorig[g];
    const float4 cg = A.gctr[g];
    const int64_t i = (int64_t)i0 + lane;
    const float4 p = lane < cnt_t ? shift(A.corig[i >> 5], o, A.pos[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float sv = lane < cnt_t ? A.sv[i] : 0.f;
    float sS = sv, sx = sv * (p.x - cg.x), sy = sv * (p.y - cg.y), sz = sv * (p.z - cg.z);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        sS += __shfl_xor_sync(0xffffffffu, sS, d);
        sx += __shfl_xor_sync(0xffffffffu, sx, d);
        sy += __shfl_xor_sync(0xffffffffu, sy, d);
        sz += __shfl_xor_sync(0xffffffffu, sz, d);
    }
    if (lane == 0) {
        A.gadj[2 * g] = make_float4(o.x + cg.x, o.y + cg.y, o.z + cg.z, cg.w);
        A.gadj[2 * g + 1] = make_float4(sx, sy, sz, sS);
    }
}

// The same records per cluster of the second level (warp per cluster, its
// up to 32 K targets in the cluster's frame).
__device__ __forceinline__ void local_cluster_record(const AdjArgs& A, int C, int lane) {
    const int g0 = C * A.cluster_k, g1 = min(g0 + A.cluster_k, A.ngroups);
    const float4 o = A.cctr[C];
    const float4 cg = A.cexp[C];
    float sS = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
    for (int i = A.goff[g0] + lane; i < A.goff[g1]; i += 32) {
        const float4 p = shift(A.corig[i >> 5], o, A.pos[i]);
        const float sv = A.sv[i];
        sS += sv;
        sx += sv * (p.x - cg.x);
        sy += sv * (p.y - cg.y);
        sz += sv * (p.z - cg.z);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        sS += __shfl_xor_sync(0xffffffffu, sS, d);
        sx += __shfl_xor_sync(0xffffffffu, sx, d);
        sy += __shfl_xor_sync(0xffffffffu, sy, d);
        sz += __shfl_xor_sync(0xffffffffu, sz, d);
    }
    if (lane == 0) {
        A.cadj[2 * C] = make_float4(o.x + cg.x, o.y + cg.y, o.z + cg.z, cg.w);
        A.cadj[2 * C + 1] = make_float4(sx, sy, sz, sS);
    }
}

// Both record sets in one launch: warps [0, ngroups) take the groups, the
// next nclusters warps the clusters.
__global__ void k_local_records(AdjArgs A) {
    const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w < A.ngroups) local_group_record(A, w, lane);
    else if (w < A.ngroups + A.nclusters) local_cluster_record(A, w - A.ngroups, lane);
}

// The pairs of one expanded entry whose pairs may straddle the cut-off: node
// b against the targets i0 .. i1 - 1, in the frame with origin o, from the
// exact cell-relative data.
__device__ __noinline__ float4 local_entry_pairs(const AdjArgs& A, int i0, int i1, const float4& o, int b) {
    const float4 xb = shift(A.ncell[b], o, A.ncent[b]);
    float cx = 0.f, cy = 0.f, cz = 0.f;
    for (int i = i0; i < i1; ++i) {
        const float4 x = shift(A.corig[i >> 5], o, A.pos[i]);
        const float dx = xb.x - x.x, dy = xb.y - x.y, dz = xb.z - x.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float ir = r2 >= A.w2 ? rsqrtf(r2) : 0.f;
        const float q = A.sv[i] * (ir * ir * ir);
        cx = fmaf(q, dx, cx);
        cy = fmaf(q, dy, cy);
        cz = fmaf(q, dz, cz);
    }
    return make_float4(cx, cy, cz, 0.f);
}

// The node gather with expanded entries: one warp per node, lanes over the
// node's whole transposed list (U reads in flight per lane, then the sums:
// 4 for the longer lists of one expansion level, 1 with clusters, whose
// shorter lists gain more from the extra resident warps of the smaller
// register count: 130 us per launch at 2, 115 at 1, 164 at 3).  Each list item carries its class in bits 30-31: an entry
// summed pair by pair (its contrib), one expanded about a group (the group;
// its record gadj) or one expanded about a cluster (the cluster; cadj); a
// node's list holds its items by class.
constexpr int kNodeGathers = 16;

// The transposed term of one expanded entry from its group's or cluster's
// record (c, rho), (D, S) at the node centroid xb: S E/r^3 + (3 E (E.D) - r^2 D)/r^5,
// E = xb - c, or, when |E| - rho < w, the entry's pairs (targets i0 .. i1 - 1,
// frame origin o).
__device__ __forceinline__ void adj_local_term(const AdjArgs& A, const float4& xb, const float4& c0,
                                               const float4& c1, int b, int i0, int i1, const float4& o,
                                               float& ax, float& ay, float& az);

template <int U>
__global__ void k_adj_node_local(AdjArgs A, float4* vnode) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= A.nnodes) return;
    const int q0 = A.tfar_off[b], q1 = A.tfar_off[b + 1];
    float ax = 0.f, ay = 0.f, az = 0.f;
    const float4 xb = A.nabs[b];
    for (int q = q0 + lane; q < q1; q += 32 * U) {
        int v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = q + 32 * u < q1 ? A.tfar_ent[q + 32 * u] : -1;
        float4 c0[U], c1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            c0[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            c1[u] = c0[u];
            if (v[u] == -1) continue;   // class 2 sets the sign bit
            const int cls = (unsigned)v[u] >> 30, id = v[u] & 0x3fffffff;
            if (cls == 0) {
                c0[u] = A.contrib[id];
            } else {
                const float4* rec = cls == 1 ? A.gadj : A.cadj;
                c0[u] = rec[2 * id];
                c1[u] = rec[2 * id + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (v[u] == -1) continue;   // class 2 sets the sign bit
            const int cls = (unsigned)v[u] >> 30, id = v[u] & 0x3fffffff;
            if (cls == 0) {
                ax += c0[u].x;
                ay += c0[u].y;
                az += c0[u].z;
            } else if (cls == 1) {
                adj_local_term(A, xb, c0[u], c1[u], b, A.goff[id], A.goff[id + 1], A.gorig[id], ax, ay, az);
            } else {
                const int g0 = id * A.cluster_k, g1 = min(g0 + A.cluster_k, A.ngroups);
                adj_local_term(A, xb, c0[u], c1[u], b, A.goff[g0], A.goff[g1], A.cctr[id], ax, ay, az);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if (lane == 0) vnode[b] = make_float4(ax, ay, az, 0.f);
}

__device__ __forceinline__ void adj_local_term(const AdjArgs& A, const float4& xb, const float4& c0,
                                               const float4& c1, int b, int i0, int i1, const float4& o,
                                               float& ax, float& ay, float& az) {
    const float ex = xb.x - c0.x, ey = xb.y - c0.y, ez = xb.z - c0.z;
    const float r2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    const float ir = rsqrtf(r2);
    const float bound = fmaf(r2, ir, -c0.w);
    if (bound > 0.f && bound * bound >= A.w2) {
        const float ir3 = ir * ir * ir, ir5 = ir3 * ir * ir;
        const float ed3 = 3.f * fmaf(ex, c1.x, fmaf(ey, c1.y, ez * c1.z));
        const float sr = c1.w * ir3;
        ax += fmaf(sr, ex, fmaf(ed3, ex, -r2 * c1.x) * ir5);
        ay += fmaf(sr, ey, fmaf(ed3, ey, -r2 * c1.y) * ir5);
        az += fmaf(sr, ez, fmaf(ed3, ez, -r2 * c1.z) * ir5);
    } else {
        const float4 cc = local_entry_pairs(A, i0, i1, o, b);
        ax += cc.x;
        ay += cc.y;
        az += cc.z;
    }
}

// One warp per node; lanes take the node's entries (consecutive slots of the
// node-major list) 32 x kNodeGathers at a time, kNodeGathers independent
// gathers per lane in flight, then reduce.  The kernel is bound by the latency
// of the gathers.
__global__ void k_adj_node(int nnodes, const int* tfar_off, const int* tfar_ent, const float4* contrib,
                           float4* vnode) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nnodes) return;
    float ax = 0.f, ay = 0.f, az = 0.f;
    const int q1 = tfar_off[b + 1];
    for (int q = tfar_off[b] + lane; q < q1; q += 32 * kNodeGathers) {
        int e[kNodeGathers];
#pragma unroll
        for (int u = 0; u < kNodeGathers; ++u) e[u] = q + 32 * u < q1 ? tfar_ent[q + 32 * u] : -1;
        float4 c[kNodeGathers];
#pragma unroll
        for (int u = 0; u < kNodeGathers; ++u) c[u] = e[u] >= 0 ? contrib[e[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kNodeGathers; ++u) { ax += c[u].x; ay += c[u].y; az += c[u].z; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if (lane == 0) vnode[b] = make_float4(ax, ay, az, 0.f);
}

// Epilogue of one source chunk: far part (walk to the root), 1/(4 pi), store.
template <int EPI>
__device__ __forceinline__ void adj_epilogue(const AdjArgs& A, int gs, int64_t j, bool valid, float ax,
                                             float ay, float az, int lane) {
    double part = 0.0;
    if (valid) {
        for (int a = A.leaf_of[j]; a >= 0; a = A.nparent[a]) {
            const float4 v = A.vnode[a];
            ax += v.x; ay += v.y; az += v.z;
            if (A.hnode0) {
                // far_order 1: - H_a (x_j - x_a), x_a the node's point centroid
                const float4 p = shift(A.corig[j >> 5], A.ncell[a], A.pos[j]);
                const float4 c = A.ncent[a];
                const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
                const float4 h0 = A.hnode0[a], h1 = A.hnode1[a];   // (xx, yy, zz), (xy, xz, yz)
                ax -= fmaf(h0.x, dx, fmaf(h1.x, dy, h1.y * dz));
                ay -= fmaf(h1.x, dx, fmaf(h0.y, dy, h1.z * dz));
                az -= fmaf(h1.y, dx, fmaf(h1.z, dy, h0.z * dz));
            }
        }
        ax *= kInv4Pi; ay *= kInv4Pi; az *= kInv4Pi;
        if (EPI == kEpiStoreATpaper) {
            const int64_t o3 = 3 * A.perm[j];
            A.out[o3] = ax * A.scale;
            A.out[o3 + 1] = ay * A.scale;
            A.out[o3 + 2] = az * A.scale;
        } else {
            A.r_out[j] = make_float4(ax, ay, az, 0.f);
            part = (double)ax * ax + (double)ay * ay + (double)az * az;
        }
    }
    if (EPI != kEpiStoreATpaper) {
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o2);
        if (lane == 0) A.partial[gs] = part;
    }
}

// ---------------------------------------------------------------------------
// First-order far field (tree parameter far_order = 1; rep_mode 1).  With
// d = x_B - x_i (node centroid minus target, as in the pair terms), r = |d|,
// and the node moment S = sum_j sym((x_j - x_B) nu_j^T), the first-order
// Taylor terms of the kernels about x_B add to a far node's term, in the
// units of the sums (times 4 pi):
//   A:   tr S / r^3 - 3 (d.S d) / r^5
//   G:   -(6 S d + 3 tr S d) / r^5 + 15 (d.S d) d / r^7
// and the exact transpose adds, for every point j of a node B, -H_B (x_j - x_B)
// with H_B = sum over the node's far entries of s_i (3 d d^T - r^2 I) / r^5.
// Pairs take the cut-off decision of the node's monopole term (the same r^2,
// computed in the same order).
// ---------------------------------------------------------------------------
// S of every node that is not a top node, by the size classes of the
// monopole moments: one thread per node of at most kMomSmall points, one warp
// per node of the mid list (up to kMomDirect points, or a leaf of any size);
// blocks [0, grid_m) take the warp class.  Stored as (Sxx, Syy, Szz, Sxy),
// (Sxz, Syz, tr S, 0) at out[2b], out[2b + 1].
__device__ __forceinline__ void dip_point(int j, const float4& cb, const float4& cc, const float4* spos,
                                          const float4* scorig, const float4* nu, float (&m)[6]) {
    const float4 p = shift(scorig[j >> 5], cb, spos[j]);   // the point relative to the cell centre
    const float dx = p.x - cc.x, dy = p.y - cc.y, dz = p.z - cc.z;
    const float4 v = nu[j];
    m[0] = fmaf(dx, v.x, m[0]);
    m[1] = fmaf(dy, v.y, m[1]);
    m[2] = fmaf(dz, v.z, m[2]);
    m[3] = fmaf(0.5f, fmaf(dx, v.y, dy * v.x), m[3]);
    m[4] = fmaf(0.5f, fmaf(dx, v.z, dz * v.x), m[4]);
    m[5] = fmaf(0.5f, fmaf(dy, v.z, dz * v.y), m[5]);
}

__device__ __forceinline__ void dip_store(int b, const float (&m)[6], float4* out) {
    out[2 * (int64_t)b] = make_float4(m[0], m[1], m[2], m[3]);
    out[2 * (int64_t)b + 1] = make_float4(m[4], m[5], m[0] + m[1] + m[2], 0.f);
}

__global__ void k_mom_dipole(int nnodes, int nmid, int grid_m, const int* mid, const int* nstart, const int* ncount,
                             const float4* ncell, const float4* ncent, const float4* spos, const float4* scorig,
                             const float4* nu, float4* out) {
    float m[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if ((int)blockIdx.x < grid_m) {
        const int k = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
        const int lane = threadIdx.x & 31;
        if (k >= nmid) return;
        const int b = mid[k];
        const float4 cb = ncell[b], cc = ncent[b];
        const int j0 = nstart[b], cnt = ncount[b];
        for (int j = j0 + lane; j < j0 + cnt; j += 32) dip_point(j, cb, cc, spos, scorig, nu, m);
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m[c] += __shfl_xor_sync(0xffffffffu, m[c], o);
        if (lane == 0) dip_store(b, m, out);
        return;
    }
    const int b = (int)((blockIdx.x - grid_m) * blockDim.x + threadIdx.x);
    if (b >= nnodes) return;
    const int cnt = ncount[b];
    if (cnt > kMomSmall) return;                          // warp class or top node
    const float4 cb = ncell[b], cc = ncent[b];
    const int j0 = nstart[b];
    for (int j = j0; j < j0 + cnt; ++j) dip_point(j, cb, cc, spos, scorig, nu, m);
    dip_store(b, m, out);
}

// S of the top nodes from their fronts (the non-top nodes under a top node
// that partition its points), moved to the top node's centroid:
//   S_top = sum_f S_f + sym((x_f - x_top) nu_f^T),  nu_f the front node's sum.
// One warp per top node, lanes over the front, then a fixed xor reduction.
__global__ void k_mom_dipole_top(int ntop, const int* top, const int2* top_rng, const int* front,
                                 const float4* ncell, const float4* ncent, const float4* mom, float4* out) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= ntop) return;
    const int b = top[k];
    const int2 rg = top_rng[k];
    const float4 cb = ncell[b], cc = ncent[b];
    float m[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int q = rg.x + lane; q < rg.y; q += 32) {
        const int f = front[q];
        const float4 cf = ncell[f], ef = ncent[f], v = mom[f];
        const float dx = ((cf.x - cb.x) + ef.x) - cc.x;   // centroid of f minus that of b
        const float dy = ((cf.y - cb.y) + ef.y) - cc.y;
        const float dz = ((cf.z - cb.z) + ef.z) - cc.z;
        const float4 s0 = out[2 * (int64_t)f], s1 = out[2 * (int64_t)f + 1];
        m[0] += fmaf(dx, v.x, s0.x);
        m[1] += fmaf(dy, v.y, s0.y);
        m[2] += fmaf(dz, v.z, s0.z);
        m[3] += fmaf(0.5f, fmaf(dx, v.y, dy * v.x), s0.w);
        m[4] += fmaf(0.5f, fmaf(dx, v.z, dz * v.x), s1.x);
        m[5] += fmaf(0.5f, fmaf(dy, v.z, dz * v.y), s1.y);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m[c] += __shfl_xor_sync(0xffffffffu, m[c], o);
    if (lane == 0) {
        out[2 * (int64_t)b] = make_float4(m[0], m[1], m[2], m[3]);
        out[2 * (int64_t)b + 1] = make_float4(m[4], m[5], m[0] + m[1] + m[2], 0.f);
    }
}

// The first-order far terms of every target: one warp per work item of the
// gather (a slice of one target group's far entries; the items are cut and
// ordered heaviest first, so the groups with the longest lists do not set the
// kernel's time), one target per lane; the item's far nodes (centroid in the
// group's frame, S) staged 32 at a time in shared memory.  OP kOpA: A's term
// in .w; kOpG: G's in .xyz; kOpAG: both.  A group cut into several items
// writes one part per item into `parts` (every lane), and
// k_far_dip_finalize adds the parts in order.
template <int OP>
__global__ void __launch_bounds__(32 * kGatherWarps) k_far_dip(GatherArgs A, const float4* mdip, float4* corr,
                                                               float4* parts) {
    __shared__ float4 sp_all[kGatherWarps][32], s0_all[kGatherWarps][32], s1_all[kGatherWarps][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x * kGatherWarps + wl;
    if (it >= A.nitems) return;
    float4* sp = sp_all[wl];
    float4* s0 = s0_all[wl];
    float4* s1 = s1_all[wl];
    const Item item = A.items[it];
    const int g = item.g;
    const int i0 = A.goff[g], cnt_t = A.goff[g + 1] - i0;
    const int64_t i = (int64_t)i0 + lane;
    const bool valid = lane < cnt_t;
    const float4 o = A.tgorig[g];
    const float4 t = valid ? shift(A.tcorig[i >> 5], o, A.tpos[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    float cx = 0.f, cy = 0.f, cz = 0.f, ca = 0.f;
    for (int base = item.f0; base < item.f1; base += 32) {
        const int cnt = min(32, item.f1 - base);
        if (lane < cnt) {
            const int b = A.far_id[base + lane];
            sp[lane] = shift(A.ncell[b], o, A.nrep[b]);
            s0[lane] = mdip[2 * (int64_t)b];
            s1[lane] = mdip[2 * (int64_t)b + 1];
        }
        __syncwarp();
        if (valid) {
#pragma unroll 4
            for (int k = 0; k < cnt; ++k) {
                const float4 p = sp[k];
                const float dx = p.x - t.x, dy = p.y - t.y, dz = p.z - t.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (!(r2 >= A.w2)) continue;
                const float ir = rsqrtf(r2);
                const float ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
                const float4 a0 = s0[k], a1 = s1[k];
                const float sdx = fmaf(a0.x, dx, fmaf(a0.w, dy, a1.x * dz));
                const float sdy = fmaf(a0.w, dx, fmaf(a0.y, dy, a1.y * dz));
                const float sdz = fmaf(a1.x, dx, fmaf(a1.y, dy, a0.z * dz));
                const float dsd = fmaf(dx, sdx, fmaf(dy, sdy, dz * sdz));
                const float tr = a1.z;
                if (OP == kOpA || OP == kOpAG) ca += fmaf(tr, ir3, -3.f * dsd * ir5);
                if (OP == kOpG || OP == kOpAG) {
                    const float f15 = 15.f * dsd * (ir5 * ir2);
                    cx += fmaf(f15, dx, -fmaf(6.f, sdx, 3.f * tr * dx) * ir5);
                    cy += fmaf(f15, dy, -fmaf(6.f, sdy, 3.f * tr * dy) * ir5);
                    cz += fmaf(f15, dz, -fmaf(6.f, sdz, 3.f * tr * dz) * ir5);
                }
            }
        }
        __syncwarp();
    }
    if (item.pslot < 0) {
        if (valid) corr[i] = make_float4(cx, cy, cz, ca);
    } else {
        parts[(int64_t)item.pslot * 32 + lane] = make_float4(cx, cy, cz, ca);
    }
}

// Groups cut into several items: the parts of k_far_dip added in order.
__global__ void k_far_dip_finalize(GatherArgs A, const float4* parts, float4* corr) {
    const int sidx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sidx >= A.nsplit) return;
    const int4 sp = A.splits[sidx];
    const int g = sp.x;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int p = 0; p < sp.z; ++p) {
        const float4 v = parts[(int64_t)(sp.y + p) * 32 + lane];
        acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    const int i0 = A.goff[g];
    if (lane < A.goff[g + 1] - i0) corr[(int64_t)i0 + lane] = acc;
}

// far_order 1: the far adjoint with the transpose of the first-order terms.
// k_adj_far's layout (one warp per work item, the group's targets staged once,
// two entries per lane in the halves of float2, paired FP32 instructions),
// summing per entry both V = sum s_i d / r^3 and H = sum s_i (3 d d^T - r^2 I) / r^5
// (d = x_B - x_i), with the same cut-off decisions as k_adj_far.
__global__ void __launch_bounds__(32 * kGatherWarps) k_adj_far_dip(AdjArgs A) {
    __shared__ float4 tp_all[kGatherWarps][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x * kGatherWarps + wl;
    if (it >= A.nitems) return;
    float4* tp = tp_all[wl];
    const Item item = A.items[it];
    const int g = item.g;
    const int i0 = A.goff[g], cnt_t = A.goff[g + 1] - i0;
    const int64_t i = (int64_t)i0 + lane;
    const float4 o = A.gorig[g];
    float4 p = lane < cnt_t ? shift(A.corig[i >> 5], o, A.pos[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    p.w = lane < cnt_t ? A.sv[i] : 0.f;
    tp[lane] = make_float4(-p.x, -p.y, -p.z, p.w);   // negated: the paired terms add them
    __syncwarp();
    for (int base = item.f0; base < item.f1; base += 64) {
        const int e0 = base + lane, e1 = e0 + 32;
        const bool v0 = e0 < item.f1, v1 = e1 < item.f1;
        float4 bp0 = make_float4(0.f, 0.f, 0.f, 0.f), bp1 = bp0;
        if (v0) { const int b = A.far_id[e0]; bp0 = shift(A.ncell[b], o, A.ncent[b]); }
        if (v1) { const int b = A.far_id[e1]; bp1 = shift(A.ncell[b], o, A.ncent[b]); }
        const float2 px = make_float2(bp0.x, bp1.x), py = make_float2(bp0.y, bp1.y), pz = make_float2(bp0.z, bp1.z);
        float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
        float2 hxx = ax, hyy = ax, hzz = ax, hxy = ax, hxz = ax, hyz = ax;
#pragma unroll 4
        for (int k = 0; k < cnt_t; ++k) {
            const float4 tk = tp[k];
            // the pair of adj_term2 (same operations and order, so the same cut-off decisions)
            const float2 dx = __fadd2_rn(px, make_float2(tk.x, tk.x));
            const float2 dy = __fadd2_rn(py, make_float2(tk.y, tk.y));
            const float2 dz = __fadd2_rn(pz, make_float2(tk.z, tk.z));
            float2 r2 = __fmul2_rn(dz, dz);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dx, dx, r2);
            float2 ir = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
            ir.x = (r2.x >= A.w2) ? ir.x : 0.f;
            ir.y = (r2.y >= A.w2) ? ir.y : 0.f;
            const float2 ir2 = __fmul2_rn(ir, ir);
            const float2 q = __fmul2_rn(make_float2(tk.w, tk.w), __fmul2_rn(ir2, ir));   // s / r^3
            ax = __ffma2_rn(q, dx, ax);
            ay = __ffma2_rn(q, dy, ay);
            az = __ffma2_rn(q, dz, az);
            // s (3 d d^T - r^2 I) / r^5 = (3 q / r^2) d d^T - q I
            const float2 q3 = __fmul2_rn(__fmul2_rn(make_float2(3.f, 3.f), q), ir2);
            const float2 nq = __fmul2_rn(make_float2(-1.f, -1.f), q);
            const float2 q3x = __fmul2_rn(q3, dx), q3y = __fmul2_rn(q3, dy);
            hxx = __ffma2_rn(q3x, dx, __fadd2_rn(hxx, nq));
            hyy = __ffma2_rn(q3y, dy, __fadd2_rn(hyy, nq));
            hzz = __ffma2_rn(__fmul2_rn(q3, dz), dz, __fadd2_rn(hzz, nq));
            hxy = __ffma2_rn(q3x, dy, hxy);
            hxz = __ffma2_rn(q3x, dz, hxz);
            hyz = __ffma2_rn(q3y, dz, hyz);
        }
        if (v0) {
            A.contrib[e0] = make_float4(ax.x, ay.x, az.x, 0.f);
            A.contrib_h0[e0] = make_float4(hxx.x, hyy.x, hzz.x, 0.f);
            A.contrib_h1[e0] = make_float4(hxy.x, hxz.x, hyz.x, 0.f);
        }
        if (v1) {
            A.contrib[e1] = make_float4(ax.y, ay.y, az.y, 0.f);
            A.contrib_h0[e1] = make_float4(hxx.y, hyy.y, hzz.y, 0.f);
            A.contrib_h1[e1] = make_float4(hxy.y, hxz.y, hyz.y, 0.f);
        }
    }
}

// far_order 1: the node gather of k_adj_node for the three per-entry sums
// (V, and H in two parts) at once, sharing the entry-id reads.
__global__ void k_adj_node3(int nnodes, const int* tfar_off, const int* tfar_ent, const float4* c0,
                            const float4* c1, const float4* c2, float4* v0, float4* v1, float4* v2) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nnodes) return;
    float a[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int q1 = tfar_off[b + 1];
    for (int q = tfar_off[b] + lane; q < q1; q += 32 * 4) {
        int e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) e[u] = q + 32 * u < q1 ? tfar_ent[q + 32 * u] : -1;
        float4 x[4], y[4], z[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            x[u] = e[u] >= 0 ? c0[e[u]] : zero;
            y[u] = e[u] >= 0 ? c1[e[u]] : zero;
            z[u] = e[u] >= 0 ? c2[e[u]] : zero;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[0] += x[u].x; a[1] += x[u].y; a[2] += x[u].z;
            a[3] += y[u].x; a[4] += y[u].y; a[5] += y[u].z;
            a[6] += z[u].x; a[7] += z[u].y; a[8] += z[u].z;
        }
    }
#pragma unroll
    for (int c = 0; c < 9; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a[c] += __shfl_xor_sync(0xffffffffu, a[c], o);
    if (lane == 0) {
        v0[b] = make_float4(a[0], a[1], a[2], 0.f);
        v1[b] = make_float4(a[3], a[4], a[5], 0.f);
        v2[b] = make_float4(a[6], a[7], a[8], 0.f);
    }
}

// x += a y over all four components (the first-order moments of mu + alpha r).
__global__ void k_axpy4(float4* x, const float4* y, const double* scalars, int64_t n) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float a = (float)scalars[3];
    const float4 u = x[k], v = y[k];
    x[k] = make_float4(fmaf(a, v.x, u.x), fmaf(a, v.y, u.y), fmaf(a, v.z, u.z), fmaf(a, v.w, u.w));
}

// Near part, first kernel: the pair sums of each (group, source) near slot.
// One warp per work item (a slice of one target group's near ranges).  The
// group's targets (negated point, s_i) are staged once in shared memory;
// each lane takes two sources of a batch of 64 from the item's near stream
// (stream positions base + lane and base + 32 + lane: the ranges
// concatenated, as in the gather) and sums, for each, the terms of all the
// group's targets in target order, with paired FP32 instructions (one staged
// target against the lane's two sources).  A source's sum lands whole in its
// lane and goes to its near slot; the next batch's sources are read while the
// current batch is summed.  The second kernel adds each point's slots in a
// fixed order.
__global__ void WNNC_ADJ_BOUNDS k_adj_near_pairs(AdjArgs A) {
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ float4 tp_all[kGatherWarps][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x * kGatherWarps + wl;
    if (it >= A.nitems) return;
    const Item item = A.items[it];
    if (item.q0 >= item.q1) return;
    float4* tp = tp_all[wl];
    const int g = item.g;
    const int i0 = A.goff[g], cnt_t = A.goff[g + 1] - i0;
    const float4 o = A.gorig[g];
    {
        const int64_t i = (int64_t)i0 + lane;
        float4 p = lane < cnt_t ? shift(A.corig[i >> 5], o, A.pos[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
        p.w = lane < cnt_t ? A.sv[i] : 0.f;
        tp[lane] = make_float4(-p.x, -p.y, -p.z, p.w);   // negated: the paired terms add them
    }
    const float4 blo = A.gbl[g], bhi = A.gbh[g];
    __syncwarp();

    int qn = item.q0;                 // first range not yet in a window
    int wx = 0, wpre = 0, wslot = 0;  // this lane's range in the window: start, stream offset, slot
    int wn = 0, wtot = 0, cur = 0;    // ranges in the window, their points, stream position
    // the next (up to) 32 sources of the stream into lanes 0..cnt-1: point
    // dp in chunk frame dc, near slot ds; returns cnt (< 32 only at the end)
    auto next_near = [&](float4& dp, float4& dc, int& ds) {
        int cnt = 0;
        while (cnt < 32) {
            if (cur == wtot) {
                if (qn >= item.q1) break;
                wn = min(32, item.q1 - qn);
                int2 r = make_int2(0, 0);
                int rs = 0;
                if (lane < wn) {
                    r = A.near_rng[qn + lane];
                    rs = A.rng_slot[qn + lane];
                }
                const int len = r.y - r.x;
                int inc = len;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int u = __shfl_up_sync(kFull, inc, d);
                    if (lane >= d) inc += u;
                }
                wx = r.x;
                wpre = inc - len;
                wslot = rs;
                wtot = __shfl_sync(kFull, inc, 31);
                qn += wn;
                cur = 0;
                continue;
            }
            const int take = min(32 - cnt, wtot - cur);
            const int x = cur + lane - cnt;
            int k = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int c = k + st;
                const int pc = __shfl_sync(kFull, wpre, c & 31);
                if (c < wn && pc <= x) k = c;
            }
            const int rx = __shfl_sync(kFull, wx, k), pk = __shfl_sync(kFull, wpre, k);
            const int rs = __shfl_sync(kFull, wslot, k);
            if (lane >= cnt && lane < cnt + take) {
                const int j = rx + (x - pk);
                dp = A.pos[j];
                dc = A.corig[j >> 5];
                ds = rs + (x - pk);
            }
            cnt += take;
            cur += take;
        }
        return cnt;
    };

    float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), c0 = p0, p1 = p0, c1 = p0;
    int s0 = 0, s1 = 0;
    int n0 = next_near(p0, c0, s0);
    int n1 = n0 == 32 ? next_near(p1, c1, s1) : 0;
    while (n0 > 0) {
        const bool v0 = lane < n0, v1 = lane < n1;
        const float4 bp0 = shift(c0, o, p0), bp1 = shift(c1, o, p1);
        const int slot0 = s0, slot1 = s1;
        bool clear = (!v0 || box_gap2(blo, bhi, bp0) >= A.fast2) && (!v1 || box_gap2(blo, bhi, bp1) >= A.fast2);
        clear = __all_sync(kFull, clear);
        // the next batch's sources, read while this batch is summed
        int m0 = 0, m1 = 0;
        if (n1 == 32) {
            m0 = next_near(p0, c0, s0);
            if (m0 == 32) m1 = next_near(p1, c1, s1);
        }
        // the two sources' sums in the halves of float2
        const float2 px = make_float2(bp0.x, bp1.x), py = make_float2(bp0.y, bp1.y), pz = make_float2(bp0.z, bp1.z);
        float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
        auto term = [&](const float4& tk, auto cut_tag) {
            constexpr bool CUT = decltype(cut_tag)::value;
            float2 dx, dy, dz, q;
            adj_term2<CUT>(px, py, pz, make_float2(tk.x, tk.x), make_float2(tk.y, tk.y), make_float2(tk.z, tk.z),
                           make_float2(tk.w, tk.w), A.w2, dx, dy, dz, q);
            ax = __ffma2_rn(q, dx, ax);
            ay = __ffma2_rn(q, dy, ay);
            az = __ffma2_rn(q, dz, az);
        };
        if (cnt_t == 32) {
            // a full group: a compile-time trip count, no bounds guards
            if (clear) {
#pragma unroll
                for (int k = 0; k < 32; ++k) term(tp[k], std::false_type{});
            } else {
#pragma unroll
                for (int k = 0; k < 32; ++k) term(tp[k], std::true_type{});
            }
        } else if (clear) {
#pragma unroll kUnroll
            for (int k = 0; k < cnt_t; ++k) term(tp[k], std::false_type{});
        } else {
#pragma unroll kUnroll
            for (int k = 0; k < cnt_t; ++k) term(tp[k], std::true_type{});
        }
        if (v0) A.near_contrib[slot0] = make_float4(ax.x, ay.x, az.x, 0.f);
        if (v1) A.near_contrib[slot1] = make_float4(ax.y, ay.y, az.y, 0.f);
        n0 = m0;
        n1 = m1;
    }
}

// Near part, second kernel, one warp per work item: a slice of the
// transposed entries of source chunk C (kAdjChunk = 8 consecutive sorted
// points).  Lane l handles source point 8C + (l & 7) and every fourth entry
// (offset l >> 3): if the entry's mask holds the point, it adds the point's
// near slot of that entry (the entry's slot plus the number of mask bits
// below the point).  A lane reads kAdjNearReads entries, then their slots,
// before it adds them in entry order.  The four partial sums of a point are
// added at the end (fixed order), into lanes 0..7, followed by the far part
// and the output.
constexpr int kAdjNearReads = 8;

template <int EPI>
__global__ void WNNC_GATHER_BOUNDS k_adj_near(AdjArgs A) {
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x * kGatherWarps + wl;
    if (it >= A.nitems) return;
    const Item item = A.items[it];
    const int sc = item.g;                       // source chunk (outputs)
    const int sl = lane & (kAdjChunk - 1), tq = lane / kAdjChunk;
    const int64_t j = (int64_t)sc * kAdjChunk + sl;
    const bool valid = j < A.n;
    const unsigned below = (1u << sl) - 1u;
    float ax = 0.f, ay = 0.f, az = 0.f;
    constexpr int kStep = 32 / kAdjChunk;
    for (int q = item.q0 + tq; q < item.q1; q += kStep * kAdjNearReads) {
        int2 ent[kAdjNearReads];
#pragma unroll
        for (int u = 0; u < kAdjNearReads; ++u)
            ent[u] = q + kStep * u < item.q1 ? A.tnear_ent[q + kStep * u] : make_int2(0, 0);
        float4 c[kAdjNearReads];
#pragma unroll
        for (int u = 0; u < kAdjNearReads; ++u) {
            const unsigned mask = (unsigned)ent[u].y;
            c[u] = ((mask >> sl) & 1u) ? A.near_contrib[ent[u].x + __popc(mask & below)]
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kAdjNearReads; ++u) {
            if (((unsigned)ent[u].y >> sl) & 1u) {
                ax += c[u].x;
                ay += c[u].y;
                az += c[u].z;
            }
        }
    }
#pragma unroll
    for (int o2 = kAdjChunk; o2 < 32; o2 <<= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o2);
        ay += __shfl_xor_sync(0xffffffffu, ay, o2);
        az += __shfl_xor_sync(0xffffffffu, az, o2);
    }
    if (item.pslot < 0) {
        adj_epilogue<EPI>(A, sc, j, valid && lane < kAdjChunk, ax, ay, az, lane);
    } else {
        A.part_acc[(int64_t)item.pslot * 32 + lane] = make_float4(ax, ay, az, 0.f);
        const int4 sp = A.splits[item.split];
        if (last_part(A.split_cnt, item.split, sp.z, lane)) {
            float sx = 0.f, sy = 0.f, sz = 0.f;
            for (int p = 0; p < sp.z; ++p) {
                const float4 v = __ldcg(A.part_acc + (int64_t)(sp.y + p) * 32 + lane);
                sx += v.x; sy += v.y; sz += v.z;
            }
            adj_epilogue<EPI>(A, sc, j, valid && lane < kAdjChunk, sx, sy, sz, lane);
        }
    }
}

// ---------------------------------------------------------------------------
// Permutations / small kernels
// ---------------------------------------------------------------------------
__global__ void k_perm_in_vec(const float* in, const int64_t* perm, int64_t n, float f, float4* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = 3 * perm[i];
    out[i] = make_float4(in[j] * f, in[j + 1] * f, in[j + 2] * f, 0.f);
}
__global__ void k_perm_in_scalar(const float* in, const int64_t* perm, int64_t n, float f, float* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[perm[i]] * f;
}
__global__ void k_perm_out_vec(const float4* in, const int64_t* perm, int64_t n, float f, float* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = 3 * perm[i];
    const float4 v = in[i];
    out[j] = v.x * f;
    out[j + 1] = v.y * f;
    out[j + 2] = v.z * f;
}
__global__ void k_normalize_queries(const float* q, int64_t m, double cx, double cy, double cz,
                                    double s, double* qn, int* bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    if (!isfinite(q[3 * i]) || !isfinite(q[3 * i + 1]) || !isfinite(q[3 * i + 2])) *bad = 1;
    qn[3 * i] = __dmul_rn(__dsub_rn((double)q[3 * i], cx), s);
    qn[3 * i + 1] = __dmul_rn(__dsub_rn((double)q[3 * i + 1], cy), s);
    qn[3 * i + 2] = __dmul_rn(__dsub_rn((double)q[3 * i + 2], cz), s);
}

// Deterministic reduction of the per-group partials and the step length of
// Alg. 2: alpha = |r|^2 / |A r|^2 (0 if |A r| = 0).  Also records the stats.
// First stage of the reduction of the three partial-sum arrays: block b adds
// the b-th of kRedBlocks fixed slices of each array (FP64 runs at a small
// fraction of the FP32 rate, so one block alone is slow for 10^4-10^5
// partials).  The order depends only on the sizes.
constexpr int kRedBlocks = 256;
// The three sums of the step length (E = |s|^2, |r|^2, |A r|^2) from the
// per-group partials: each of kRedBlocks blocks sums a fixed slice, and the
// block that finishes last adds the kRedBlocks block sums in index order
// (the same tree as a separate one-block pass) and sets
// alpha = |r|^2 / |A r|^2 (0 if |A r| = 0; a non-finite alpha sets the error
// flag).  The ticket counts finished blocks and is reset by the last one.
__global__ void k_reduce3(const double* a0, int n0, const double* a1, int n1, const double* a2, int n2,
                          double* out, double* scalars, float* stats, float w, int* err, unsigned* ticket) {
    __shared__ double sh[3][kTB];
    __shared__ bool last;
    const double* arr[3] = {a0, a1, a2};
    const int n[3] = {n0, n1, n2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int per = (n[c] + kRedBlocks - 1) / kRedBlocks;
        const int lo = blockIdx.x * per, hi = min(n[c], lo + per);
        double s = 0.0;
        for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) s += arr[c][k];
        sh[c][threadIdx.x] = s;
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; ++c) out[c * kRedBlocks + blockIdx.x] = sh[c][0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == kRedBlocks - 1;
    }
    __syncthreads();
    if (!last) return;
    // second stage (one block, kTB = kRedBlocks threads: one block sum each)
    static_assert(kTB == kRedBlocks, "one block sum per thread");
#pragma unroll
    for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = __ldcg(out + c * kRedBlocks + threadIdx.x);
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double E = sh[0][0], R = sh[1][0], Q = sh[2][0];
        double alpha = Q > 0.0 ? R / Q : 0.0;
        if (!isfinite(alpha)) {
            atomicOr(err, kErrNonFinite);
            alpha = 0.0;
        }
        scalars[0] = E;
        scalars[1] = R;
        scalars[2] = Q;
        scalars[3] = alpha;
        if (stats) {
            stats[0] = w;
            stats[1] = (float)E;
            stats[2] = (float)alpha;
            stats[3] = (float)R;
        }
        *ticket = 0u;
    }
}

__global__ void k_axpy(const float4* mu, const float4* r, const double* scalars, int64_t n, float4* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = (float)scalars[3];
    const float4 m = mu[i], d = r[i];
    out[i] = make_float4(fmaf(a, d.x, m.x), fmaf(a, d.y, m.y), fmaf(a, d.z, m.z), 0.f);
}

// Moments of mu + alpha r from those of mu and r (point-centroid
// representatives: the moments are linear in nu; the .w sums are not used).
__global__ void k_node_axpy(float4* mom, const float4* mom_r, const double* scalars, int nnodes) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nnodes) return;
    const float a = (float)scalars[3];
    const float4 m = mom[b], d = mom_r[b];
    mom[b] = make_float4(fmaf(a, d.x, m.x), fmaf(a, d.y, m.y), fmaf(a, d.z, m.z), m.w + fabsf(a) * d.w);
}

// WNNC update of the fused iteration: mu' = mu + alpha r, G(mu') = G(mu) +
// alpha G(r) (G is linear with point-centroid representatives), then the
// rescale of Alg. 3 (or Eq. 19 with fixed areas); mu' is kept where G = 0.
__global__ void k_wnnc_update(const float4* mu, const float4* r, const float4* gmu, const float4* gr,
                              const double* scalars, const float* area, int rescale_mode, int64_t n,
                              float4* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = (float)scalars[3];
    const float4 m = mu[i], d = r[i], g0 = gmu[i], g1 = gr[i];
    const float4 mp = make_float4(fmaf(a, d.x, m.x), fmaf(a, d.y, m.y), fmaf(a, d.z, m.z), 0.f);
    const float gx = fmaf(a, g1.x, g0.x), gy = fmaf(a, g1.y, g0.y), gz = fmaf(a, g1.z, g0.z);
    const float hn = sqrtf(gx * gx + gy * gy + gz * gz);
    float4 res = mp;
    if (hn > 0.f) {
        const float len = rescale_mode == 1 ? area[i] : sqrtf(mp.x * mp.x + mp.y * mp.y + mp.z * mp.z);
        const float f = len / hn;
        res = make_float4(gx * f, gy * f, gz * f, 0.f);
    }
    out[i] = res;
}

__global__ void k_stats_nograd(float* stats, float w) {
    stats[0] = w;
    stats[1] = 0.f;
    stats[2] = 0.f;
    stats[3] = 0.f;
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
// Squared cut-off: w^2, floored at (2^-20)^2 so that coincident pairs (the
// self term, repeated samples) never count, also when w = 0 (Alg. 1).
inline float cutoff2(float w) { return fmaxf(w * w, 0x1p-40f); }

// Squared radius of the per-batch cut-off test: a source farther than
// sqrt(cutoff2) * 1.001 + 4e-6 from a group's box is farther than the cut-off
// from every target of the group, also after the FP32 rounding of the box, of
// the frame shifts and of r^2 (all below 1e-6 in normalised units).
inline float fast_radius2(float w) {
    const double r = std::sqrt((double)cutoff2(w)) * 1.001 + 4e-6;
    return (float)(r * r * (1.0 + 1e-6));
}

GatherArgs base_args(const Tree& t, const TargetSet& ts, float w, float4* part_acc) {
    GatherArgs a{};
    a.items = ts.work.items;
    a.nitems = ts.work.nitems;
    a.splits = ts.work.splits;
    a.split_cnt = ts.work.split_cnt;
    a.nsplit = ts.work.nsplit;
    a.part_acc = part_acc;
    a.ngroups = ts.ngroups;
    a.goff = ts.goff;
    a.tpos = ts.pos;
    a.tcorig = ts.corig;
    a.tgorig = ts.gorig;
    a.tperm = ts.perm;
    a.far_id = ts.far_id;
    a.near_rng = ts.near_rng;
    a.spos = t.self.pos;
    a.scorig = t.self.corig;
    a.ncell = t.node_cell;
    a.nrep = t.params.rep_mode == 0 ? t.node_rep : t.node_cent;
    a.nmom = t.mom;
    a.w2 = cutoff2(w);
    a.fast2 = fast_radius2(w);
    a.near_bf16 = t.params.near_bf16;
    a.tgbl = ts.gbl;
    a.tgbh = ts.gbh;
    a.walk = t.params.criterion == 1;
    a.copen = t.params.theta > 0.f ? 1.f / t.params.theta : INFINITY;
    a.nchild0 = t.node_child0;
    a.nnchild = t.node_nchild;
    a.nstart = t.node_start;
    a.ncount = t.node_count;
    a.err_flag = t.err_flag;
    a.far_off = ts.far_off;
    a.lsplit = ts.far_lsplit;
    a.gctr = ts.gctr;
    a.csplit = ts.far_csplit;
    a.cluster_k = ts.cluster_k;
    a.nclusters = ts.nclusters;
    a.cctr = ts.cctr;
    a.cexp = ts.cexp;
    return a;
}

template <int OP, int EPI>
void launch_gather(Tree& t, const GatherArgs& a, cudaStream_t s) {
    if (a.nitems == 0) return;
    ProfScope ps(&t.prof,
                 OP == kOpAG ? WNNC_PROF_AG
                             : (OP == kOpG ? WNNC_PROF_G : (OP == kOpA ? WNNC_PROF_A : WNNC_PROF_ADJ_NEAR)),
                 s);
    if (a.walk) {
        k_walk<OP, EPI><<<ceil_div(a.ngroups, kGatherWarps), 32 * kGatherWarps, 0, s>>>(a);
        WNNC_LAUNCH_CHECK();
        return;
    }
    // the bfloat16 near-field study applies to the sums of A and G only
    if ((OP == kOpA || OP == kOpG || OP == kOpAG) && a.near_bf16)
        k_gather<OP, EPI, true, kGatherTPL><<<ceil_div(a.nitems, kGatherWarps), 32 * kGatherWarps, 0, s>>>(a);
    else
        k_gather<OP, EPI, false, kGatherTPL><<<ceil_div(a.nitems, kGatherWarps), 32 * kGatherWarps, 0, s>>>(a);
    WNNC_LAUNCH_CHECK();
    if (a.nsplit > 0) {
        k_gather_finalize<EPI><<<ceil_div((int64_t)a.nsplit * 32, kTB), kTB, 0, s>>>(a);
        WNNC_LAUNCH_CHECK();
    }
}

AdjArgs adj_args(const Tree& t, float w) {
    const TargetSet& S = t.self;
    AdjArgs a{};
    a.part_acc = t.part_acc;
    a.n = t.n;
    a.goff = S.goff;
    a.pos = S.pos;
    a.corig = S.corig;
    a.gorig = S.gorig;
    a.far_id = S.far_id;
    a.ncell = t.node_cell;
    a.ncent = t.node_cent;
    a.contrib = t.contrib;
    a.tnear_ent = t.tnear_ent;
    a.near_rng = S.near_rng;
    a.rng_slot = t.rng_slot;
    a.near_contrib = t.near_contrib;
    a.leaf_of = t.leaf_of;
    a.nparent = t.node_parent;
    a.vnode = t.vnode;
    a.w2 = cutoff2(w);
    a.fast2 = fast_radius2(w);
    a.gbl = S.gbl;
    a.gbh = S.gbh;
    a.far_off = S.far_off;
    a.lsplit = S.far_lsplit;
    a.gctr = S.gctr;
    a.nabs = t.node_abs;
    a.ngroups = S.ngroups;
    a.nnodes = t.nnodes;
    a.tfar_off = t.tfar_off;
    a.tfar_ent = t.tfar_ent;
    a.gadj = t.gadj;
    a.cadj = t.cadj;
    a.cluster_k = S.cluster_k;
    a.nclusters = S.nclusters;
    a.cctr = S.cctr;
    a.cexp = S.cexp;
    return a;
}

}  // namespace

// ---------------------------------------------------------------------------
// Profiler
// ---------------------------------------------------------------------------
cudaEvent_t Profiler::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    WNNC_CUDA(cudaEventCreate(&e));
    return e;
}

void Profiler::collect() {
    for (auto& r : recs) {
        WNNC_CUDA(cudaEventSynchronize(r.b));
        float ms_ = 0.f;
        WNNC_CUDA(cudaEventElapsedTime(&ms_, r.a, r.b));
        launches[r.cls] += 1;
        ms[r.cls] += ms_;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    recs.clear();
}

void Profiler::reset() {
    collect();
    for (int k = 0; k < WNNC_PROF_CLASSES; ++k) {
        launches[k] = 0;
        ms[k] = 0.0;
    }
}

Profiler::~Profiler() {
    for (auto& r : recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
}

ProfScope::ProfScope(Profiler* p_, int cls_, cudaStream_t s_) : p(p_), cls(cls_), s(s_) {
    if (p && p->on && ((p->mask >> cls) & 1u)) {
        a = p->get();
        b = p->get();
        cudaEventRecord(a, s);
    }
}

ProfScope::~ProfScope() {
    if (a) {
        cudaEventRecord(b, s);
        p->recs.push_back({cls, a, b});
    }
}

// Moments of nu over all nodes into `out` (and the dynamic representatives
// in rep_mode 0).
void moments(Tree& t, const float4* nu_vec, const float* nu_s, int rep_mode, float4* out, cudaStream_t s) {
    ProfScope ps(&t.prof, WNNC_PROF_MOMENTS, s);
    const bool w = rep_mode == 0;
    const int grid_s = ceil_div(t.nnodes, kTB), grid_m = ceil_div((int64_t)t.nmom_mid * 32, kTB);
    const bool fp64 = t.params.moments_fp64 != 0;
#define WNNC_MOM_SUMS(SC, WE, ACC, DM)                                                                    \
    do {                                                                                                  \
        k_mom_sums<SC, WE, ACC><<<grid_m + grid_s, kTB, 0, s>>>(                                          \
            t.nnodes, t.nmom_mid, grid_m, t.mom_mid, t.node_start, t.node_count, t.node_cell, t.node_cent,  \
            t.self.pos, t.self.corig, nu_vec, nu_s, out, t.mom_x, t.node_rep, DM);                        \
        WNNC_LAUNCH_CHECK();                                                                              \
        if (t.nmom_top > 0) {                                                                             \
            k_mom_top<WE, ACC><<<t.nmom_top, kMomTopThreads, 0, s>>>(t.mom_top, t.mom_top_rng, t.mom_front, \
                                                                     t.node_cell, t.node_cent, out, t.mom_x, \
                                                                     t.node_rep, DM);                     \
            WNNC_LAUNCH_CHECK();                                                                          \
        }                                                                                                 \
    } while (0)
#define WNNC_MOM_PREC(SC, WE)                                      \
    do {                                                           \
        if (fp64) WNNC_MOM_SUMS(SC, WE, double, t.dmom);           \
        else WNNC_MOM_SUMS(SC, WE, float, (double*)nullptr);       \
    } while (0)
    if (nu_s) {
        if (w) WNNC_MOM_PREC(true, true); else WNNC_MOM_PREC(true, false);
    } else {
        if (w) WNNC_MOM_PREC(false, true); else WNNC_MOM_PREC(false, false);
    }
#undef WNNC_MOM_PREC
#undef WNNC_MOM_SUMS
}

static void perm_in_vec(Tree& t, const float* in, float f, float4* out, cudaStream_t s) {
    ProfScope ps(&t.prof, WNNC_PROF_SMALL, s);
    k_perm_in_vec<<<ceil_div(t.n, kTB), kTB, 0, s>>>(in, t.self.perm, t.n, f, out);
    WNNC_LAUNCH_CHECK();
}

// far_order 1: the first-order moments S of the sorted field nu into mdip
// (mom: the field's monopole moments, already computed).
static void dipole_moments(Tree& t, const float4* nu, const float4* mom, float4* mdip, cudaStream_t s) {
    ProfScope ps(&t.prof, WNNC_PROF_MOMENTS, s);
    const int grid_s = ceil_div(t.nnodes, kTB), grid_m = ceil_div((int64_t)t.nmom_mid * 32, kTB);
    k_mom_dipole<<<grid_m + grid_s, kTB, 0, s>>>(t.nnodes, t.nmom_mid, grid_m, t.mom_mid, t.node_start,
                                                  t.node_count, t.node_cell, t.node_cent, t.self.pos, t.self.corig,
                                                  nu, mdip);
    WNNC_LAUNCH_CHECK();
    if (t.nmom_top > 0) {
        k_mom_dipole_top<<<ceil_div((int64_t)t.nmom_top * 32, kTB), kTB, 0, s>>>(
            t.nmom_top, t.mom_top, t.mom_top_rng, t.mom_front, t.node_cell, t.node_cent, mom, mdip);
        WNNC_LAUNCH_CHECK();
    }
}

// far_order 1: the first-order far terms of the targets of ts (moments mdip)
// into corr, and the gather arguments a told to add them.
template <int OP>
static void far_dipole(Tree& t, const TargetSet& ts, const float4* mdip, GatherArgs& a, float4* corr,
                       float4* parts, cudaStream_t s) {
    ProfScope ps(&t.prof, OP == kOpAG ? WNNC_PROF_AG : (OP == kOpG ? WNNC_PROF_G : WNNC_PROF_A), s);
    if (a.nitems > 0) {
        k_far_dip<OP><<<ceil_div(a.nitems, kGatherWarps), 32 * kGatherWarps, 0, s>>>(a, mdip, corr, parts);
        WNNC_LAUNCH_CHECK();
        if (a.nsplit > 0) {
            k_far_dip_finalize<<<ceil_div((int64_t)a.nsplit * 32, kTB), kTB, 0, s>>>(a, parts, corr);
            WNNC_LAUNCH_CHECK();
        }
    }
    a.dip_corr = corr;
}


// Far terms of the entries expanded about each target group's centre
// (local_theta > 0), stored per target in corr and added by the gather's
// epilogue; a's moments must be those of the field summed.  The nodes'
// centroids and this field's moments are packed first into one 32-byte
// record per node.
template <int OP>
static void local_far(Tree& t, const TargetSet& ts, GatherArgs& a, float4* corr, cudaStream_t s) {
    if (!ts.far_lsplit || ts.ngroups == 0) return;
    ProfScope ps(&t.prof, WNNC_PROF_LOCAL, s);
    k_local_pack<<<ceil_div(t.nnodes, kTB), kTB, 0, s>>>(t.nnodes, t.node_abs, a.nmom, t.local_rec);
    WNNC_LAUNCH_CHECK();
    a.lrec = t.local_rec;
    k_local_ag<OP><<<ceil_div(ts.ngroups, kLocalWarps), 32 * kLocalWarps, 0, s>>>(a, corr);
    WNNC_LAUNCH_CHECK();
    if (ts.far_csplit) {
        k_local_cl<OP><<<ceil_div(ts.nclusters, kLocalWarps), 32 * kLocalWarps, 0, s>>>(a, corr);
        WNNC_LAUNCH_CHECK();
    }
    a.dip_corr = corr;
}

void local_setup(Tree& t, cudaStream_t s) {
    if (t.nnodes == 0) return;
    k_node_abs<<<ceil_div(t.nnodes, kTB), kTB, 0, s>>>(t.nnodes, t.node_cell, t.node_cent, t.node_abs);
    WNNC_LAUNCH_CHECK();
}

// The gather of one field with its expanded far entries.  On the points as
// targets, with a second stream: the expanded entries (latency-bound) run on
// it while the gather (FP32-bound) sums the pairs on s and leaves its sums in
// gather_raw; after the join, one pass per group adds both and runs the
// epilogue.  Otherwise the expanded entries first, then the gather.
template <int OP, int EPI>
static void gather_with_local(Tree& t, const TargetSet& ts, GatherArgs& a, cudaStream_t s) {
    if (!ts.far_lsplit) {
        launch_gather<OP, EPI>(t, a, s);
        return;
    }
    if (!t.aux || &ts != &t.self || !ts.work.gsplit || a.walk || a.near_bf16) {
        local_far<OP>(t, ts, a, t.dip_corr, s);
        launch_gather<OP, EPI>(t, a, s);
        return;
    }
    WNNC_CUDA(cudaEventRecord(t.ev_fork, s));
    WNNC_CUDA(cudaStreamWaitEvent(t.aux, t.ev_fork, 0));
    local_far<OP>(t, ts, a, t.dip_corr, t.aux);
    WNNC_CUDA(cudaEventRecord(t.ev_join, t.aux));
    a.raw = t.gather_raw;
    a.gsplit = ts.work.gsplit;
    {
        ProfScope ps(&t.prof,
                     OP == kOpAG ? WNNC_PROF_AG : (OP == kOpG ? WNNC_PROF_G : WNNC_PROF_A), s);
        if (a.nitems > 0) {
            k_gather<OP, EPI, false, kGatherTPL><<<ceil_div(a.nitems, kGatherWarps), 32 * kGatherWarps, 0, s>>>(a);
            WNNC_LAUNCH_CHECK();
        }
    }
    WNNC_CUDA(cudaStreamWaitEvent(s, t.ev_join, 0));
    ProfScope ps(&t.prof, WNNC_PROF_SMALL, s);
    k_gather_finalize_all<EPI><<<ceil_div((int64_t)ts.ngroups * 32, kTB), kTB, 0, s>>>(a);
    WNNC_LAUNCH_CHECK();
}

void eval_w(Tree& t, const float* mu, float w, float* out, cudaStream_t s) {
    const float s2 = (float)(t.scale * t.scale);
    perm_in_vec(t, mu, s2, t.mu_a, s);
    moments(t, t.mu_a, nullptr, t.params.rep_mode, t.mom, s);
    GatherArgs a = base_args(t, t.self, w, t.part_acc);
    if (t.params.far_order == 1) {
        dipole_moments(t, t.mu_a, t.mom, t.mom_dip, s);
        far_dipole<kOpA>(t, t.self, t.mom_dip, a, t.dip_corr, t.part_acc, s);
    }
    a.sval = t.mu_a;
    a.out = out;
    gather_with_local<kOpA, kEpiStoreW>(t, t.self, a, s);
}

void eval_grad(Tree& t, const float* mu, float w, float* out, cudaStream_t s) {
    const float s2 = (float)(t.scale * t.scale);
    perm_in_vec(t, mu, s2, t.mu_a, s);
    moments(t, t.mu_a, nullptr, t.params.rep_mode, t.mom, s);
    GatherArgs a = base_args(t, t.self, w, t.part_acc);
    if (t.params.far_order == 1) {
        dipole_moments(t, t.mu_a, t.mom, t.mom_dip, s);
        far_dipole<kOpG>(t, t.self, t.mom_dip, a, t.dip_corr, t.part_acc, s);
    }
    a.sval = t.mu_a;
    a.out = out;
    a.scale = (float)t.scale;
    gather_with_local<kOpG, kEpiStoreGrad>(t, t.self, a, s);
}

// r_sorted <- A^T(s_sorted) in normalised units (exact transpose, rep_mode 1),
// or stores to out (caller units) when out != nullptr.
static void adjoint_exact(Tree& t, const float* s_sorted, float w, float* out, float4* r_sorted,
                          double* partial, cudaStream_t s) {
    AdjArgs a = adj_args(t, w);
    a.sv = s_sorted;
    // the near pair sums need only s: on the second stream, overlapping the far path
    const bool fork = t.adj_pair_work.nitems > 0 && t.aux;
    if (fork) {
        WNNC_CUDA(cudaEventRecord(t.ev_fork, s));
        WNNC_CUDA(cudaStreamWaitEvent(t.aux, t.ev_fork, 0));
        ProfScope ps(&t.prof, WNNC_PROF_ADJ_NEAR, t.aux);
        AdjArgs pr = a;
        pr.items = t.adj_pair_work.items;
        pr.nitems = t.adj_pair_work.nitems;
        k_adj_near_pairs<<<ceil_div(pr.nitems, kGatherWarps), 32 * kGatherWarps, 0, t.aux>>>(pr);
        WNNC_LAUNCH_CHECK();
        WNNC_CUDA(cudaEventRecord(t.ev_join, t.aux));
    }
    if (t.self.far_entries > 0) {
        const bool dip = t.params.far_order == 1;
        {
            ProfScope ps(&t.prof, WNNC_PROF_ADJ_FAR, s);
            AdjArgs f = a;
            f.items = t.adj_far_work.items;
            f.nitems = t.adj_far_work.nitems;
            if (dip) {
                // with the transpose of the first-order far terms (s HPhi per entry)
                f.contrib_h0 = t.contrib_h0;
                f.contrib_h1 = t.contrib_h1;
                k_adj_far_dip<<<ceil_div(f.nitems, kGatherWarps), 32 * kGatherWarps, 0, s>>>(f);
            } else {
                k_adj_far<<<ceil_div(f.nitems, kGatherWarps), 32 * kGatherWarps, 0, s>>>(f);
            }
            WNNC_LAUNCH_CHECK();
        }
        if (a.lsplit) {
            // each group's and cluster's record for its expanded entries
            ProfScope ps(&t.prof, WNNC_PROF_LOCAL, s);
            const int64_t nrec = (int64_t)t.self.ngroups + (a.cadj ? t.self.nclusters : 0);
            k_local_records<<<ceil_div(nrec * 32, kTB), kTB, 0, s>>>(a);
            WNNC_LAUNCH_CHECK();
        }
        ProfScope ps(&t.prof, WNNC_PROF_ADJ_NODE, s);
        if (a.lsplit && a.cadj) {
            k_adj_node_local<1><<<ceil_div((int64_t)t.nnodes * 32, kTB), kTB, 0, s>>>(a, t.vnode);
        } else if (a.lsplit) {
            k_adj_node_local<4><<<ceil_div((int64_t)t.nnodes * 32, kTB), kTB, 0, s>>>(a, t.vnode);
        } else if (dip) {
            // the node sums of V and H, pushed down in the near kernel's epilogue
            k_adj_node3<<<ceil_div((int64_t)t.nnodes * 32, kTB), kTB, 0, s>>>(
                t.nnodes, t.tfar_off, t.tfar_ent, t.contrib, t.contrib_h0, t.contrib_h1, t.vnode, t.hnode0, t.hnode1);
            a.hnode0 = t.hnode0;
            a.hnode1 = t.hnode1;
        } else {
            k_adj_node<<<ceil_div((int64_t)t.nnodes * 32, kTB), kTB, 0, s>>>(t.nnodes, t.tfar_off, t.tfar_ent,
                                                                             t.contrib, t.vnode);
        }
        WNNC_LAUNCH_CHECK();
    } else {
        WNNC_CUDA(cudaMemsetAsync(t.vnode, 0, sizeof(float4) * t.nnodes, s));
    }
    if (fork) {
        WNNC_CUDA(cudaStreamWaitEvent(s, t.ev_join, 0));
    } else if (t.adj_pair_work.nitems > 0) {
        ProfScope ps(&t.prof, WNNC_PROF_ADJ_NEAR, s);
        AdjArgs pr = a;
        pr.items = t.adj_pair_work.items;
        pr.nitems = t.adj_pair_work.nitems;
        k_adj_near_pairs<<<ceil_div(pr.nitems, kGatherWarps), 32 * kGatherWarps, 0, s>>>(pr);
        WNNC_LAUNCH_CHECK();
    }
    a.items = t.adj_near_work.items;
    a.nitems = t.adj_near_work.nitems;
    a.splits = t.adj_near_work.splits;
    a.split_cnt = t.adj_near_work.split_cnt;
    a.nsplit = t.adj_near_work.nsplit;
    a.perm = t.self.perm;
    a.out = out;
    a.r_out = r_sorted;
    a.partial = partial;
    a.scale = out ? (float)(t.scale * t.scale) : 1.f;
    ProfScope ps(&t.prof, WNNC_PROF_ADJ_NEAR, s);
    const int grid = ceil_div(a.nitems, kGatherWarps);
    if (out) k_adj_near<kEpiStoreATpaper><<<grid, 32 * kGatherWarps, 0, s>>>(a);
    else k_adj_near<kEpiNormSq><<<grid, 32 * kGatherWarps, 0, s>>>(a);
    WNNC_LAUNCH_CHECK();
}

void eval_adjoint(Tree& t, const float* sv, float w, float* out, cudaStream_t s) {
    {
        ProfScope ps(&t.prof, WNNC_PROF_SMALL, s);
        k_perm_in_scalar<<<ceil_div(t.n, kTB), kTB, 0, s>>>(sv, t.self.perm, t.n, 1.f, t.s_s);
        WNNC_LAUNCH_CHECK();
    }
    if (t.params.rep_mode == 1) {
        adjoint_exact(t, t.s_s, w, out, nullptr, nullptr, s);
    } else {
        moments(t, nullptr, t.s_s, 0, t.mom, s);
        GatherArgs a = base_args(t, t.self, w, t.part_acc);
        a.sval_s = t.s_s;
        a.out = out;
        a.scale = (float)(t.scale * t.scale);
        launch_gather<kOpATpaper, kEpiStoreATpaper>(t, a, s);
    }
}

void eval_at(Tree& t, const float* mu, const float* q, int64_t m, float w, int grad, float* out,
             cudaStream_t s) {
    const float s2 = (float)(t.scale * t.scale);
    double* qn = dalloc<double>(3 * m);
    int* bad = dalloc<int>(1);
    WNNC_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_normalize_queries<<<ceil_div(m, kTB), kTB, 0, s>>>(q, m, t.center[0], t.center[1], t.center[2],
                                                         t.scale, qn, bad);
    WNNC_LAUNCH_CHECK();
    int hbad = 0;
    WNNC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    WNNC_CUDA(cudaStreamSynchronize(s));
    pool_free(bad);
    if (hbad) {
        pool_free(qn);
        fail(WNNC_EINVAL, "query coordinates must be finite");
    }
    TargetSet Q;
    float4* pacc = nullptr;
    try {
        build_target_set(t, Q, qn, m, false, s);
        pacc = dalloc<float4>((size_t)Q.work.nslots * 32);
    } catch (...) {
        cudaStreamSynchronize(s);
        free_target_set(Q);
        pool_free(qn);
        throw;
    }
    pool_free(qn);
    perm_in_vec(t, mu, s2, t.mu_a, s);
    moments(t, t.mu_a, nullptr, t.params.rep_mode, t.mom, s);
    GatherArgs a = base_args(t, Q, w, pacc);
    float4* qcorr = nullptr;
    if (t.params.far_order == 1) {
        qcorr = dalloc<float4>((size_t)m);
        dipole_moments(t, t.mu_a, t.mom, t.mom_dip, s);
        if (grad) far_dipole<kOpG>(t, Q, t.mom_dip, a, qcorr, pacc, s);
        else far_dipole<kOpA>(t, Q, t.mom_dip, a, qcorr, pacc, s);
    }
    a.sval = t.mu_a;
    a.out = out;
    a.scale = (float)t.scale;
    if (Q.far_lsplit) {
        qcorr = dalloc<float4>((size_t)m);
        if (grad) local_far<kOpG>(t, Q, a, qcorr, s);
        else local_far<kOpA>(t, Q, a, qcorr, s);
    }
    if (grad) launch_gather<kOpG, kEpiStoreGrad>(t, a, s);
    else launch_gather<kOpA, kEpiStoreW>(t, a, s);
    unsigned timeouts = 0;
    wait_timeouts_async(&timeouts, s);
    WNNC_CUDA(cudaStreamSynchronize(s));
    pool_free(qcorr);
    pool_free(pacc);
    free_target_set(Q);
    check_wait_timeouts(timeouts, s);
}

// Smoothing width of iteration `it` (Sec. 4.4): from w2 at the first
// iteration down to w1 at the last, along the schedule p.schedule (the paper's
// linear one, or the cosine and exponential decays of Sec. 6.1.2).
static double schedule_width(const wnnc_iter_params& p, int it) {
    const double w1 = p.w1, w2 = p.w2;
    if (p.n_iter <= 1) return w1;
    const double t = (double)(it - 1) / (double)(p.n_iter - 1);
    if (p.schedule == 1) return w1 + (w2 - w1) * 0.5 * (1.0 + std::cos(3.14159265358979323846 * t));
    if (p.schedule == 2) return w2 * std::pow(w1 / w2, t);
    return w2 * (double)(p.n_iter - it) / (double)(p.n_iter - 1) + w1 * (double)(it - 1) / (double)(p.n_iter - 1);
}

// Alg. 3 with Alg. 2, in the sorted order, normalised units.
void iterate(Tree& t, float* mu_inout, const float* area, const wnnc_iter_params& p, cudaStream_t s,
             float* stats) {
    const int64_t n = t.n;
    const TargetSet& S = t.self;
    const int npart = std::max(std::max(S.ngroups, S.nchunks), t.nach);
    const float s2 = (float)(t.scale * t.scale);
    const int grid_n = ceil_div(n, kTB);
    float4* mu = t.mu_a;
    float4* mu_alt = t.mu_b;
    if (p.init == 1) {
        perm_in_vec(t, mu_inout, s2, mu, s);
    } else {
        WNNC_CUDA(cudaMemsetAsync(mu, 0, sizeof(float4) * n, s));
    }
    if (p.rescale == 1) {
        ProfScope ps(&t.prof, WNNC_PROF_SMALL, s);
        k_perm_in_scalar<<<grid_n, kTB, 0, s>>>(area, S.perm, n, s2, t.area_s);
        WNNC_LAUNCH_CHECK();
    }
    double* pE = t.partials;
    double* prr = t.partials + npart;
    double* pqq = t.partials + 2 * (int64_t)npart;
    const int last = p.last_iter > 0 ? p.last_iter : p.n_iter;
    const int rep_mode = t.params.rep_mode;
    const int n_rr = rep_mode == 1 ? t.nach : S.ngroups;
    // With point-centroid representatives the moments are linear in nu: those
    // of the updated field mu + alpha r follow from the moments of mu and r.
    const bool linear_mom = rep_mode == 1 && !t.params.moments_fp64;
    // The default iteration fuses A and G: both are linear and share every pair
    // term, so one pass gives A(mu) with G(mu) and one A(r) with G(r), and
    // G(mu + alpha r) = G(mu) + alpha G(r) needs no third pass.
    const bool fused = linear_mom && p.use_grad && p.use_wnnc;
    const bool dip = t.params.far_order == 1;   // first-order far terms (rep_mode 1)
    for (int it = p.first_iter; it <= last; ++it) {
        const float w = (float)schedule_width(p, it);
        float* st = stats ? stats + 4 * (int64_t)(it - p.first_iter) : nullptr;
        if (fused) {
            // s = b - A mu, with G(mu)
            moments(t, mu, nullptr, rep_mode, t.mom, s);
            GatherArgs a = base_args(t, S, w, t.part_acc);
            if (dip) {
                dipole_moments(t, mu, t.mom, t.mom_dip, s);
                far_dipole<kOpAG>(t, S, t.mom_dip, a, t.dip_corr, t.part_acc, s);
            }
            a.sval = mu;
            a.s_out = t.s_s;
            a.partial = pE;
            a.g_out = t.g_mu;
            gather_with_local<kOpAG, kEpiResidualAG>(t, S, a, s);
            // r = A^T s
            adjoint_exact(t, t.s_s, w, nullptr, t.r_s, prr, s);
            // |A r|^2, with G(r)
            moments(t, t.r_s, nullptr, rep_mode, t.mom_r, s);
            GatherArgs b = base_args(t, S, w, t.part_acc);
            if (dip) {
                dipole_moments(t, t.r_s, t.mom_r, t.mom_dip_r, s);
                far_dipole<kOpAG>(t, S, t.mom_dip_r, b, t.dip_corr, t.part_acc, s);
            }
            b.nmom = t.mom_r;
            b.sval = t.r_s;
            b.partial = pqq;
            b.g_out = t.g_r;
            gather_with_local<kOpAG, kEpiNormSqAG>(t, S, b, s);
            {
                ProfScope ps(&t.prof, WNNC_PROF_SMALL, s);
                k_reduce3<<<kRedBlocks, kTB, 0, s>>>(pE, S.ngroups, prr, n_rr, pqq, S.ngroups, t.red, t.scalars, st,
                                                     w, t.err_flag, t.red_ticket);
                WNNC_LAUNCH_CHECK();
                k_wnnc_update<<<grid_n, kTB, 0, s>>>(mu, t.r_s, t.g_mu, t.g_r, t.scalars, t.area_s, p.rescale, n,
                                                     mu_alt);
                WNNC_LAUNCH_CHECK();
            }
            std::swap(mu, mu_alt);
            continue;
        }
        if (p.use_grad) {
            // s = b - A mu
            moments(t, mu, nullptr, rep_mode, t.mom, s);
            GatherArgs a = base_args(t, S, w, t.part_acc);
            if (dip) {
                dipole_moments(t, mu, t.mom, t.mom_dip, s);
                far_dipole<kOpA>(t, S, t.mom_dip, a, t.dip_corr, t.part_acc, s);
            }
            a.sval = mu;
            a.s_out = t.s_s;
            a.partial = pE;
            gather_with_local<kOpA, kEpiResidual>(t, S, a, s);
            // r = A^T s
            if (rep_mode == 1) {
                adjoint_exact(t, t.s_s, w, nullptr, t.r_s, prr, s);
            } else {
                // the paper's s-representative treecode for A^T
                moments(t, nullptr, t.s_s, 0, t.mom, s);
                GatherArgs c = base_args(t, S, w, t.part_acc);
                c.sval_s = t.s_s;
                c.mu_out = t.r_s;
                c.partial = prr;
                launch_gather<kOpATpaper, kEpiStoreR>(t, c, s);
            }
            // |A r|^2
            float4* mom_r = linear_mom ? t.mom_r : t.mom;
            float4* mdip_r = linear_mom ? t.mom_dip_r : t.mom_dip;
            moments(t, t.r_s, nullptr, rep_mode, mom_r, s);
            GatherArgs b = base_args(t, S, w, t.part_acc);
            if (dip) {
                dipole_moments(t, t.r_s, mom_r, mdip_r, s);
                far_dipole<kOpA>(t, S, mdip_r, b, t.dip_corr, t.part_acc, s);
            }
            b.nmom = mom_r;
            b.sval = t.r_s;
            b.partial = pqq;
            gather_with_local<kOpA, kEpiNormSq>(t, S, b, s);
            {
                ProfScope ps(&t.prof, WNNC_PROF_SMALL, s);
                k_reduce3<<<kRedBlocks, kTB, 0, s>>>(pE, S.ngroups, prr, n_rr, pqq, S.ngroups, t.red, t.scalars, st,
                                                     w, t.err_flag, t.red_ticket);
                WNNC_LAUNCH_CHECK();
                k_axpy<<<grid_n, kTB, 0, s>>>(mu, t.r_s, t.scalars, n, mu_alt);
                WNNC_LAUNCH_CHECK();
                if (linear_mom && p.use_wnnc) {
                    k_node_axpy<<<ceil_div(t.nnodes, kTB), kTB, 0, s>>>(t.mom, t.mom_r, t.scalars, t.nnodes);
                    WNNC_LAUNCH_CHECK();
                    if (dip) {
                        k_axpy4<<<ceil_div(2 * (int64_t)t.nnodes, kTB), kTB, 0, s>>>(t.mom_dip, t.mom_dip_r,
                                                                                  t.scalars, 2 * (int64_t)t.nnodes);
                        WNNC_LAUNCH_CHECK();
                    }
                }
            }
            std::swap(mu, mu_alt);
        } else if (st) {
            k_stats_nograd<<<1, 1, 0, s>>>(st, w);
            WNNC_LAUNCH_CHECK();
        }
        if (p.use_wnnc) {
            if (!(linear_mom && p.use_grad)) {
                moments(t, mu, nullptr, rep_mode, t.mom, s);
                if (dip) dipole_moments(t, mu, t.mom, t.mom_dip, s);
            }
            GatherArgs g = base_args(t, S, w, t.part_acc);
            if (dip) far_dipole<kOpG>(t, S, t.mom_dip, g, t.dip_corr, t.part_acc, s);
            g.sval = mu;
            g.mu_cur = mu;
            g.mu_out = mu_alt;
            g.area = t.area_s;
            g.rescale_mode = p.rescale;
            gather_with_local<kOpG, kEpiRescale>(t, S, g, s);
            std::swap(mu, mu_alt);
        }
    }
    ProfScope ps(&t.prof, WNNC_PROF_SMALL, s);
    k_perm_out_vec<<<grid_n, kTB, 0, s>>>(mu, S.perm, n, 1.f / s2, mu_inout);
    WNNC_LAUNCH_CHECK();
}

}  // namespace wnnc
