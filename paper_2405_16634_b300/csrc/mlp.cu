// mlp.cu -- the point-patch MLP of the learned warm start: forward, backward
// and Adam kernels.
//
// Network: 48 -> 128 -> 128 -> 128 -> 3 with ReLU after the three hidden
// layers.  Input: the 16 nearest neighbours' offsets divided by the 16th
// distance (knn.cu).  Output v; the predicted oriented unit normal is
// v / |v|.  Loss per point: 1 - (v/|v|) . y for the label normal y (mean over
// the batch).  Parameters are one flat FP32 master buffer (for Adam); every
// weight is rounded to BF16 when it is read, and all products are accumulated
// in FP32.
//
// Each layer is a small dense product X W^T over a batch of points, done as a
// shared-memory-tiled FP32 kernel (64 x 64 outputs per block, 4 x 4 per
// thread).  Weight gradients are reduced over the batch in chunks of 1024
// rows into per-chunk partials and summed in a fixed order (deterministic).
#include <cuda_bf16.h>

#include "common.cuh"

namespace wnnc {

constexpr int kIn = 48, kHid = 128, kOut = 3;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid * kHid;
constexpr int kOffW4 = kOffB3 + kHid;
constexpr int kOffB4 = kOffW4 + kOut * kHid;
constexpr int kParams = kOffB4 + kOut;     // 39683
constexpr int kChunk = 1024;               // rows per weight-gradient partial

namespace {

__device__ __forceinline__ float bf16r(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

constexpr int kT = 64, kKt = 16;

// Y[B][N] = act(X[B][K] W^T + b), W [N][K] (BF16-rounded on load).
template <bool RELU>
__global__ void __launch_bounds__(256) k_lin_fwd(const float* X, const float* W, const float* bias, float* Y,
                                                 int64_t B, int K, int N) {
    __shared__ float xs[kKt][kT + 1];
    __shared__ float ws[kKt][kT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * kT;
    const int c0 = blockIdx.y * kT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kKt) {
        for (int e = threadIdx.x; e < kT * kKt; e += 256) {
            const int rr = e / kKt, kk = e % kKt;
            const int64_t row = r0 + rr;
            const int col = c0 + rr, k = k0 + kk;
            xs[kk][rr] = (row < B && k < K) ? X[row * K + k] : 0.f;
            ws[kk][rr] = (col < N && k < K) ? bf16r(W[(int64_t)col * K + k]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKt; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = xs[kk][ty * 4 + q]; b[q] = ws[kk][tx * 4 + q]; }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t row = r0 + ty * 4 + p;
        if (row >= B) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int col = c0 + tx * 4 + q;
            if (col >= N) continue;
            float y = acc[p][q] + bias[col];
            if (RELU) y = fmaxf(y, 0.f);
            Y[row * N + col] = y;
        }
    }
}

// dX[B][K] = (dY[B][N] W[N][K]) * (H[B][K] > 0)   (gradient through the ReLU of the layer input)
__global__ void __launch_bounds__(256) k_lin_bwd_data(const float* dY, const float* W, const float* H, float* dX,
                                                      int64_t B, int K, int N) {
    __shared__ float ds[kKt][kT + 1];
    __shared__ float ws[kKt][kT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * kT;
    const int c0 = blockIdx.y * kT;
    float acc[4][4] = {};
    for (int n0 = 0; n0 < N; n0 += kKt) {
        for (int e = threadIdx.x; e < kT * kKt; e += 256) {
            const int rr = e / kKt, nn = e % kKt;
            const int64_t row = r0 + rr;
            const int col = c0 + rr, nidx = n0 + nn;
            ds[nn][rr] = (row < B && nidx < N) ? dY[row * N + nidx] : 0.f;
            ws[nn][rr] = (col < K && nidx < N) ? bf16r(W[(int64_t)nidx * K + col]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int nn = 0; nn < kKt; ++nn) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = ds[nn][ty * 4 + q]; b[q] = ws[nn][tx * 4 + q]; }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t row = r0 + ty * 4 + p;
        if (row >= B) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int col = c0 + tx * 4 + q;
            if (col >= K) continue;
            dX[row * K + col] = H[row * K + col] > 0.f ? acc[p][q] : 0.f;
        }
    }
}

// Partial weight gradient of one chunk of rows:
//   part[c][n][k] = sum_{b in chunk c} dY[b][n] X[b][k],  part[c][bias n] = sum_b dY[b][n]
__global__ void __launch_bounds__(256) k_lin_bwd_weight(const float* dY, const float* X, int64_t B, int K,
                                                        int N, float* part, int woff, int boff) {
    __shared__ float ds[kKt][kT + 1];
    __shared__ float xs[kKt][kT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int n0 = blockIdx.x * kT, k0 = blockIdx.y * kT;
    const int64_t b0 = (int64_t)blockIdx.z * kChunk, b1 = min(B, b0 + kChunk);
    float acc[4][4] = {};
    float bacc[4] = {};
    for (int64_t bb = b0; bb < b1; bb += kKt) {
        for (int e = threadIdx.x; e < kT * kKt; e += 256) {
            const int rr = e % kT, q = e / kT;
            const int64_t row = bb + q;
            ds[q][rr] = (row < b1 && n0 + rr < N) ? dY[row * N + n0 + rr] : 0.f;
            xs[q][rr] = (row < b1 && k0 + rr < K) ? X[row * K + k0 + rr] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kKt; ++q) {
            float a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) { a[p] = ds[q][ty * 4 + p]; b[p] = xs[q][tx * 4 + p]; }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[p][r] = fmaf(a[p], b[r], acc[p][r]);
                bacc[p] += a[p];
            }
        }
        __syncthreads();
    }
    float* P = part + (int64_t)blockIdx.z * kParams;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int n = n0 + ty * 4 + p;
        if (n >= N) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int k = k0 + tx * 4 + r;
            if (k < K) P[woff + n * K + k] = acc[p][r];
        }
        if (blockIdx.y == 0 && tx == 0) P[boff + n] = bacc[p];
    }
}

__global__ void k_sum_partials(const float* part, int nchunk, float* grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    float s = 0.f;
    for (int c = 0; c < nchunk; ++c) s += part[(int64_t)c * kParams + p];
    grad[p] = s;
}

// Loss per row, with c = (v/|v|).y: 1 - c (mode 0) or 1 - c^2 (mode 1, blind
// to the sign of v), and its gradient w.r.t. v divided by the batch size.
// dc/dv = (y - c v/|v|) / |v|.
__global__ void k_cos_loss(const float* V, const float* Yl, int64_t B, int mode, float* dV, double* lpart) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (b < B) {
        const float vx = V[3 * b], vy = V[3 * b + 1], vz = V[3 * b + 2];
        const float yx = Yl[3 * b], yy = Yl[3 * b + 1], yz = Yl[3 * b + 2];
        const float nv = sqrtf(vx * vx + vy * vy + vz * vz);
        float gx = 0.f, gy = 0.f, gz = 0.f;
        if (nv > 0.f) {
            const float inv = 1.f / nv;
            const float nx = vx * inv, ny = vy * inv, nz = vz * inv;
            const float c = nx * yx + ny * yy + nz * yz;
            l = mode ? 1.0 - (double)c * (double)c : 1.0 - (double)c;
            const float f = (mode ? -2.f * c : -1.f) * inv / (float)B;
            gx = f * (yx - c * nx);
            gy = f * (yy - c * ny);
            gz = f * (yz - c * nz);
        } else {
            l = 1.0;
        }
        dV[3 * b] = gx;
        dV[3 * b + 1] = gy;
        dV[3 * b + 2] = gz;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    __shared__ double sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        lpart[blockIdx.x] = s;
    }
}

__global__ void k_loss_final(const double* lpart, int np, int64_t B, float* loss) {
    double s = 0.0;
    for (int k = 0; k < np; ++k) s += lpart[k];
    *loss = (float)(s / (double)B);
}

// Adam (Kingma & Ba) with bias correction.
__global__ void k_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Warm-start field: unit direction of the network output, sign from a
// reference field (one iteration of the method), length = area per point
// (area > 0) or the reference's length (area = 0).
__global__ void k_warm_init(const float* dir, const float* ref, int64_t n, float area, float* mu) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float dx = dir[3 * i], dy = dir[3 * i + 1], dz = dir[3 * i + 2];
    const float nv = sqrtf(dx * dx + dy * dy + dz * dz);
    float len = area;
    if (area == 0.f && ref)
        len = sqrtf(ref[3 * i] * ref[3 * i] + ref[3 * i + 1] * ref[3 * i + 1] + ref[3 * i + 2] * ref[3 * i + 2]);
    float f = nv > 0.f ? len / nv : 0.f;
    if (ref) {
        const float dot = dx * ref[3 * i] + dy * ref[3 * i + 1] + dz * ref[3 * i + 2];
        if (dot < 0.f) f = -f;
    }
    mu[3 * i] = dx * f;
    mu[3 * i + 1] = dy * f;
    mu[3 * i + 2] = dz * f;
}

dim3 grid2(int64_t B, int N) { return dim3((unsigned)((B + kT - 1) / kT), (unsigned)((N + kT - 1) / kT)); }

}  // namespace

int mlp_param_count() { return kParams; }

void mlp_alloc(Mlp& m, int64_t max_batch) {
    m.max_batch = max_batch;
    m.params = dalloc<float>(kParams);
    m.m = dalloc<float>(kParams);
    m.v = dalloc<float>(kParams);
    m.grad = dalloc<float>(kParams);
    WNNC_CUDA(cudaMemset(m.params, 0, sizeof(float) * kParams));
    WNNC_CUDA(cudaMemset(m.m, 0, sizeof(float) * kParams));
    WNNC_CUDA(cudaMemset(m.v, 0, sizeof(float) * kParams));
    m.h1 = dalloc<float>(max_batch * kHid);
    m.h2 = dalloc<float>(max_batch * kHid);
    m.h3 = dalloc<float>(max_batch * kHid);
    m.out = dalloc<float>(max_batch * kOut);
    m.d1 = dalloc<float>(max_batch * kHid);
    m.d2 = dalloc<float>(max_batch * kHid);
    m.d3 = dalloc<float>(max_batch * kHid);
    m.dout = dalloc<float>(max_batch * kOut);
    m.part = dalloc<float>((size_t)ceil_div(max_batch, kChunk) * kParams);
    m.lpart = dalloc<double>(ceil_div(max_batch, 256));
}

void mlp_free(Mlp& m) {
    dfree(m.params); dfree(m.m); dfree(m.v); dfree(m.grad); dfree(m.h1); dfree(m.h2); dfree(m.h3);
    dfree(m.out); dfree(m.d1); dfree(m.d2); dfree(m.d3); dfree(m.dout); dfree(m.part); dfree(m.lpart);
}

// Forward of B <= max_batch rows into m.h1..h3 and y.
static void forward_rows(Mlp& m, const float* x, int64_t B, float* y, cudaStream_t s) {
    const float* P = m.params;
    k_lin_fwd<true><<<grid2(B, kHid), 256, 0, s>>>(x, P + kOffW1, P + kOffB1, m.h1, B, kIn, kHid);
    WNNC_LAUNCH_CHECK();
    k_lin_fwd<true><<<grid2(B, kHid), 256, 0, s>>>(m.h1, P + kOffW2, P + kOffB2, m.h2, B, kHid, kHid);
    WNNC_LAUNCH_CHECK();
    k_lin_fwd<true><<<grid2(B, kHid), 256, 0, s>>>(m.h2, P + kOffW3, P + kOffB3, m.h3, B, kHid, kHid);
    WNNC_LAUNCH_CHECK();
    k_lin_fwd<false><<<grid2(B, kOut), 256, 0, s>>>(m.h3, P + kOffW4, P + kOffB4, y, B, kHid, kOut);
    WNNC_LAUNCH_CHECK();
}

void mlp_forward(Mlp& m, const float* x, int64_t B, float* y, cudaStream_t s) {
    for (int64_t b0 = 0; b0 < B; b0 += m.max_batch) {
        const int64_t nb = std::min<int64_t>(m.max_batch, B - b0);
        forward_rows(m, x + b0 * kIn, nb, y + b0 * kOut, s);
    }
}

// Gradient of the mean loss over B <= max_batch rows into m.grad; loss to loss_dev.
void mlp_grad(Mlp& m, const float* x, const float* label, int64_t B, float* loss_dev, cudaStream_t s) {
    forward_rows(m, x, B, m.out, s);
    const int nlb = ceil_div(B, 256);
    k_cos_loss<<<nlb, 256, 0, s>>>(m.out, label, B, m.loss_mode, m.dout, m.lpart);
    WNNC_LAUNCH_CHECK();
    if (loss_dev) {
        k_loss_final<<<1, 1, 0, s>>>(m.lpart, nlb, B, loss_dev);
        WNNC_LAUNCH_CHECK();
    }
    const float* P = m.params;
    const int nch = ceil_div(B, kChunk);
    // output layer
    k_lin_bwd_weight<<<dim3(1, 2, nch), 256, 0, s>>>(m.dout, m.h3, B, kHid, kOut, m.part, kOffW4, kOffB4);
    WNNC_LAUNCH_CHECK();
    k_lin_bwd_data<<<grid2(B, kHid), 256, 0, s>>>(m.dout, P + kOffW4, m.h3, m.d3, B, kHid, kOut);
    WNNC_LAUNCH_CHECK();
    // hidden 3
    k_lin_bwd_weight<<<dim3(2, 2, nch), 256, 0, s>>>(m.d3, m.h2, B, kHid, kHid, m.part, kOffW3, kOffB3);
    WNNC_LAUNCH_CHECK();
    k_lin_bwd_data<<<grid2(B, kHid), 256, 0, s>>>(m.d3, P + kOffW3, m.h2, m.d2, B, kHid, kHid);
    WNNC_LAUNCH_CHECK();
    // hidden 2
    k_lin_bwd_weight<<<dim3(2, 2, nch), 256, 0, s>>>(m.d2, m.h1, B, kHid, kHid, m.part, kOffW2, kOffB2);
    WNNC_LAUNCH_CHECK();
    k_lin_bwd_data<<<grid2(B, kHid), 256, 0, s>>>(m.d2, P + kOffW2, m.h1, m.d1, B, kHid, kHid);
    WNNC_LAUNCH_CHECK();
    // hidden 1 (input layer weights)
    k_lin_bwd_weight<<<dim3(2, 1, nch), 256, 0, s>>>(m.d1, x, B, kIn, kHid, m.part, kOffW1, kOffB1);
    WNNC_LAUNCH_CHECK();
    k_sum_partials<<<ceil_div(kParams, 256), 256, 0, s>>>(m.part, nch, m.grad);
    WNNC_LAUNCH_CHECK();
}

void mlp_adam(Mlp& m, float lr, cudaStream_t s) {
    m.step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m.step), c2 = 1.f - powf(b2, (float)m.step);
    k_adam<<<ceil_div(kParams, 256), 256, 0, s>>>(m.params, m.grad, m.m, m.v, kParams, lr, b1, b2, 1e-8f, c1,
                                                  c2);
    WNNC_LAUNCH_CHECK();
}

void warm_init(const float* dir, const float* ref, int64_t n, float area, float* mu, cudaStream_t s) {
    k_warm_init<<<ceil_div(n, 256), 256, 0, s>>>(dir, ref, n, area, mu);
    WNNC_LAUNCH_CHECK();
}

}  // namespace wnnc
