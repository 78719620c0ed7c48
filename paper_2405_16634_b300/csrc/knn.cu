// knn.cu -- k nearest neighbours (k = 16) of every point and the local patch
// features of the learned warm start.
//
// One warp per target group (<= 32 Morton-consecutive points, one per lane).
// The warp walks the octree with a search radius r around the group's
// bounding box: nodes farther than r are skipped, leaves closer than r have
// their points staged 32 at a time in shared memory, and every lane keeps its
// 16 nearest candidates in a sorted register array.  When some lane's 16th
// distance exceeds r (its true neighbours may lie outside the box's
// r-neighbourhood), the warp doubles r and searches again; once r covers the
// whole root cube every point has been seen.  Distances are computed in the
// group's frame (exact dyadic shifts) in FP32; the candidate order among
// exactly equal distances is by traversal, not by index.
#include "common.cuh"

namespace wnnc {

namespace {

constexpr int kK = 16;
constexpr int kKnnWarps = 2;
constexpr int kKnnStack = 2048;

__device__ __forceinline__ float4 kshift(const float4& c, const float4& o, const float4& p) {
    return make_float4((c.x - o.x) + p.x, (c.y - o.y) + p.y, (c.z - o.z) + p.z, 0.f);
}

// squared gap between an FP64 box and the group box (both normalised units)
__device__ __forceinline__ double box_gap2(const double* blo, const double* bhi, const double* glo,
                                           const double* ghi) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double a = blo[k] - ghi[k], e = glo[k] - bhi[k];
        double m = fmax(fmax(a, e), 0.0);
        s += m * m;
    }
    return s;
}

__global__ void __launch_bounds__(32 * kKnnWarps)
k_knn16(int ngroups, const int* goff, const float4* pos, const float4* corig, const float4* gorig,
        const double* glo, const double* ghi, const double* nlo, const double* nhi, const int* nstart,
        const int* ncount, const int* nchild, const int* nchild0, const float4* ncell, const int* leaf_of,
        int* out_idx, float* out_d2, int* err) {
    __shared__ int stack_all[kKnnWarps][kKnnStack];
    __shared__ float4 sp_all[kKnnWarps][32];
    __shared__ int sj_all[kKnnWarps][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * kKnnWarps + wl;
    if (g >= ngroups) return;
    int* st = stack_all[wl];
    float4* sp = sp_all[wl];
    int* sj = sj_all[wl];
    const unsigned lt = (1u << lane) - 1u;
    const int i0 = goff[g], cnt_t = goff[g + 1] - i0;
    const int i = i0 + lane;
    const bool valid = lane < cnt_t;
    const float4 o = gorig[g];
    const float4 t = valid ? kshift(corig[i >> 5], o, pos[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    double bl[3], bh[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) { bl[k] = glo[3 * g + k]; bh[k] = ghi[3 * g + k]; }

    float dk[kK];
    int ik[kK];
    // The first search uses the width of the first target's leaf, which is
    // enough for most groups on a surface.  The largest over the lanes of the
    // 16th distance among each lane's 32 Morton-order neighbours (sorted
    // points i - 16 .. i + 16) bounds every lane's true 16th distance from
    // above, so a search of that radius (with the 0.1 % margin of the test
    // below) finds all the neighbours: a group the first search does not
    // finish goes straight to it instead of doubling the radius through many
    // passes (isolated points, outliers).  Fewer than 16 such neighbours: the
    // radius doubles.
    double r = (double)ncell[leaf_of[i0]].w;
    double r_bound = 0.0;
    {
        const int n = goff[ngroups];
#pragma unroll
        for (int k = 0; k < kK; ++k) dk[k] = INFINITY;
        if (valid) {
            for (int q = -kK; q <= kK; ++q) {
                const int j = i + q;
                if (q == 0 || j < 0 || j >= n) continue;
                const float4 p = kshift(corig[j >> 5], o, pos[j]);
                const float dx = p.x - t.x, dy = p.y - t.y, dz = p.z - t.z;
                float cd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
#pragma unroll
                for (int k = 0; k < kK; ++k) {
                    if (cd < dk[k]) {
                        const float td = dk[k];
                        dk[k] = cd;
                        cd = td;
                    }
                }
            }
        } else {
            dk[kK - 1] = 0.f;
        }
        float b16 = dk[kK - 1];
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) b16 = fmaxf(b16, __shfl_xor_sync(0xffffffffu, b16, o2));
        if (b16 < INFINITY) r_bound = sqrt((double)b16 / 0.999) * 1.0001;
    }
    for (;;) {
#pragma unroll
        for (int k = 0; k < kK; ++k) { dk[k] = INFINITY; ik[k] = -1; }
        const double r2 = r * r;
        if (lane == 0) st[0] = 0;
        __syncwarp();
        int top = 1;
        bool overflow = false;
        while (top > 0) {
            const int take = min(top, 32);
            const int b = lane < take ? st[top - take + lane] : -1;
            top -= take;
            __syncwarp();
            bool leaf = false, open = false;
            if (b >= 0 && box_gap2(nlo + 3 * b, nhi + 3 * b, bl, bh) <= r2) {
                if (nchild[b] == 0) leaf = true; else open = true;
            }
            // process the leaves found in this round, one after another
            unsigned lm = __ballot_sync(0xffffffffu, leaf);
            while (lm) {
                const int src_lane = __ffs(lm) - 1;
                lm &= lm - 1;
                const int lb = __shfl_sync(0xffffffffu, b, src_lane);
                const int s0 = nstart[lb], s1 = s0 + ncount[lb];
                for (int base = s0; base < s1; base += 32) {
                    const int cnt = min(32, s1 - base);
                    if (lane < cnt) {
                        const int j = base + lane;
                        sp[lane] = kshift(corig[j >> 5], o, pos[j]);
                        sj[lane] = j;
                    }
                    __syncwarp();
                    if (valid) {
                        for (int q = 0; q < cnt; ++q) {
                            const int j = sj[q];
                            if (j == i) continue;
                            const float4 p = sp[q];
                            const float dx = p.x - t.x, dy = p.y - t.y, dz = p.z - t.z;
                            float cd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            if (cd < dk[kK - 1]) {
                                int ci = j;
#pragma unroll
                                for (int k = 0; k < kK; ++k) {
                                    if (cd < dk[k]) {
                                        const float td = dk[k];
                                        const int ti = ik[k];
                                        dk[k] = cd;
                                        ik[k] = ci;
                                        cd = td;
                                        ci = ti;
                                    }
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            // push the children of opened nodes
            const int nc = open ? nchild[b] : 0;
            int inc = nc;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += u;
            }
            const int total = __shfl_sync(0xffffffffu, inc, 31);
            if (top + total > kKnnStack) {
                overflow = true;
                break;
            }
            if (open) {
                const int c0 = nchild0[b];
                for (int q = 0; q < nc; ++q) st[top + inc - nc + q] = c0 + q;
            }
            top += total;
            __syncwarp();
            (void)lt;
        }
        if (overflow) {
            if (lane == 0) atomicOr(err, kErrCapacity);
            break;
        }
        // done when every lane's 16th candidate lies within r (or r covers the cube)
        const bool ok = !valid || dk[kK - 1] <= (float)r2 * 0.999f;
        if (__all_sync(0xffffffffu, ok) || r > 8.0) break;
        r = r_bound > r ? r_bound : 2.0 * r;
    }
    if (valid) {
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            out_idx[(int64_t)kK * i + k] = ik[k];
            out_d2[(int64_t)kK * i + k] = dk[k];
        }
    }
}

// Patch features of point i (input order): the offsets of its 16 nearest
// neighbours, nearest first, divided by the 16th neighbour's distance, in
// double from the normalised coordinates, and their input indices.
__global__ void k_knn_features(int64_t n, const int* idx_sorted, const double* xs, const int64_t* perm,
                               float* feat, int* idx_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t pi = perm[i];
    const double* xi = xs + 3 * i;
    double d16 = 0.0;
    {
        const int j = idx_sorted[kK * i + kK - 1];
        if (j >= 0) {
            const double* xj = xs + 3 * (int64_t)j;
            const double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
            d16 = sqrt(dx * dx + dy * dy + dz * dz);
        }
    }
    const double inv = d16 > 0.0 ? 1.0 / d16 : 0.0;
    for (int k = 0; k < kK; ++k) {
        const int j = idx_sorted[kK * i + k];
        double f[3] = {0.0, 0.0, 0.0};
        if (j >= 0) {
            const double* xj = xs + 3 * (int64_t)j;
            f[0] = (xj[0] - xi[0]) * inv;
            f[1] = (xj[1] - xi[1]) * inv;
            f[2] = (xj[2] - xi[2]) * inv;
        }
        if (feat) {
            feat[48 * pi + 3 * k] = (float)f[0];
            feat[48 * pi + 3 * k + 1] = (float)f[1];
            feat[48 * pi + 3 * k + 2] = (float)f[2];
        }
        if (idx_out) idx_out[kK * pi + k] = j >= 0 ? (int)perm[j] : -1;
    }
}

}  // namespace

void knn16(Tree& t, int* idx_out, float* feat_out, cudaStream_t s) {
    const TargetSet& S = t.self;
    int* idx = dalloc<int>((size_t)kK * t.n);
    float* d2 = dalloc<float>((size_t)kK * t.n);
    int* err = dalloc<int>(1);
    WNNC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_knn16<<<ceil_div(S.ngroups, kKnnWarps), 32 * kKnnWarps, 0, s>>>(
        S.ngroups, S.goff, S.pos, S.corig, S.gorig, S.glo, S.ghi, t.node_lo, t.node_hi, t.node_start,
        t.node_count, t.node_nchild, t.node_child0, t.node_cell, t.leaf_of, idx, d2, err);
    WNNC_LAUNCH_CHECK();
    k_knn_features<<<ceil_div(t.n, 256), 256, 0, s>>>(t.n, idx, t.xs, S.perm, feat_out, idx_out);
    WNNC_LAUNCH_CHECK();
    int herr = 0;
    WNNC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    WNNC_CUDA(cudaStreamSynchronize(s));
    pool_free(idx);
    pool_free(d2);
    pool_free(err);
    if (herr) fail(WNNC_ECAPACITY, "kNN traversal stack overflow");
}

}  // namespace wnnc
