// mlp.cu -- the point-patch MLP of the learned warm start: forward, backward
// and Adam kernels.
//
// Network: 48 -> 128 -> 128 -> 128 -> 3 with ReLU after the three hidden
// layers.  Input: the 16 nearest neighbours' offsets divided by the 16th
// distance (knn.cu).  Output v; the predicted oriented unit normal is
// v / |v|.  Loss per point: 1 - (v/|v|) . y for the label normal y (mean over
// the batch).  Parameters are one flat FP32 master buffer (for Adam); every
// parameter, weights and biases, is rounded to BF16 when it is read, and all
// products are accumulated in FP32.
//
// Forward (inference and the training forward): one fused kernel over all
// four layers on the BF16 tensor cores (mma.sync m16n8k16, FP32 accumulate).
// Each block stages the BF16-rounded weights once in shared memory, in the
// register order of the mma B operand; each warp then runs 16-row tiles
// through the four layers with the activations kept in registers (the f32
// accumulator fragment of one layer is, element for element, the A fragment
// of the next).  Activations are FP32 values; each enters the mma as a
// BF16 pair hi + lo (hi = bf16(a), lo = bf16(a - hi)), two products per
// weight tile, so an activation carries ~16 significant bits and the
// network computes what its FP32-activation definition says to ~1e-5
// relative -- BF16 weights, FP32 accumulation.
//
// Backward: each layer's data and weight gradients are small dense products
// done as shared-memory-tiled FP32 kernels (64 x 64 outputs per block, 4 x 4
// per thread).  Weight gradients are reduced over the batch in chunks of 1024
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
            float y = acc[p][q] + bf16r(bias[col]);
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

// ---------------------------------------------------------------------------
// Fused forward on the tensor cores.
// ---------------------------------------------------------------------------
constexpr int kTcWarps = 8;                          // 16-row tiles in flight per block
constexpr int kTileWords = 64;                       // one B fragment: 32 lanes x 2 registers
constexpr int kNt = kHid / 8;                        // n-tiles of a 128-wide layer
constexpr int kL1Tiles = (kIn / 16) * kNt;           // 48
constexpr int kL2Tiles = (kHid / 16) * kNt;          // 128 (layers 2 and 3)
constexpr int kL4Tiles = kHid / 16;                  // 8 (3 outputs padded to one n-tile of 8)
constexpr int kOffT1 = 0, kOffT2 = kL1Tiles, kOffT3 = kOffT2 + kL2Tiles, kOffT4 = kOffT3 + kL2Tiles;
constexpr int kWTiles = kOffT4 + kL4Tiles;           // 312 tiles = 79,872 bytes
constexpr int kBiasF = 3 * kHid + 8;
constexpr size_t kTcSmem = sizeof(uint32_t) * kWTiles * kTileWords + sizeof(float) * kBiasF;

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }

// Two FP32 values (lower index first) as BF16 pairs hi and lo = bf16(a - hi).
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    hi = bf16x2_bits(h);
    lo = bf16x2_bits(__floats2bfloat162_rn(a - hf.x, b - hf.y));
}

// D = A B + D, m16n8k16, BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragments of y = x W^T (W [N][K] row-major, N <= 8 nt_count): tile
// (kt, nt) holds, for lane 4g + t, register r: W[8nt + g][16kt + 2t + 8r]
// and the next k, BF16-rounded, zero for rows n >= N.
__device__ void fill_tiles(uint32_t* dst, const float* W, int K, int N, int nt_count) {
    const int ntiles = (K / 16) * nt_count;
    for (int e = threadIdx.x; e < ntiles * kTileWords; e += blockDim.x) {
        const int tile = e / kTileWords, word = e % kTileWords;
        const int kt = tile / nt_count, nt = tile % nt_count;
        const int lane = word >> 1, r = word & 1;
        const int n = 8 * nt + (lane >> 2), k = 16 * kt + 2 * (lane & 3) + 8 * r;
        const float a = n < N ? W[(int64_t)n * K + k] : 0.f;
        const float b = n < N ? W[(int64_t)n * K + k + 1] : 0.f;
        dst[e] = bf16x2_bits(__floats2bfloat162_rn(a, b));
    }
}

// One 128-wide layer: acc[nt] = sum over k-tiles of (hi + lo) A times the tiles.
template <int KT>
__device__ __forceinline__ void tc_layer(const uint32_t (&ahi)[KT][4], const uint32_t (&alo)[KT][4],
                                         const uint32_t* tiles, float (&acc)[kNt][4], int lane) {
#pragma unroll
    for (int nt = 0; nt < kNt; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
#pragma unroll
        for (int nt = 0; nt < kNt; ++nt) {
            const uint2 b = reinterpret_cast<const uint2*>(tiles + (kt * kNt + nt) * kTileWords)[lane];
            mma_bf16(acc[nt], ahi[kt], b.x, b.y);
            mma_bf16(acc[nt], alo[kt], b.x, b.y);
        }
    }
}

// Bias and ReLU on a layer's accumulators (rows r0 + g and r0 + g + 8,
// columns 8nt + 2t, +1), optional FP32 store of the activations, and the
// next layer's A fragments: k-tile kt takes n-tiles 2kt (columns 16kt + 2t)
// and 2kt + 1 (columns 16kt + 8 + 2t).
__device__ __forceinline__ void tc_activate(float (&acc)[kNt][4], const float* bias, float* hstore, int64_t r0,
                                            int64_t B, int lane, uint32_t (&ahi)[8][4], uint32_t (&alo)[8][4]) {
    const int g = lane >> 2, t = lane & 3;
    const int64_t ra = r0 + g, rb = ra + 8;
#pragma unroll
    for (int nt = 0; nt < kNt; ++nt) {
        const int col = 8 * nt + 2 * t;
        const float b0 = bias[col], b1 = bias[col + 1];
        acc[nt][0] = fmaxf(acc[nt][0] + b0, 0.f);
        acc[nt][1] = fmaxf(acc[nt][1] + b1, 0.f);
        acc[nt][2] = fmaxf(acc[nt][2] + b0, 0.f);
        acc[nt][3] = fmaxf(acc[nt][3] + b1, 0.f);
        if (hstore) {
            if (ra < B) *reinterpret_cast<float2*>(hstore + ra * kHid + col) = make_float2(acc[nt][0], acc[nt][1]);
            if (rb < B) *reinterpret_cast<float2*>(hstore + rb * kHid + col) = make_float2(acc[nt][2], acc[nt][3]);
        }
    }
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
        split_bf16x2(acc[2 * kt][0], acc[2 * kt][1], ahi[kt][0], alo[kt][0]);
        split_bf16x2(acc[2 * kt][2], acc[2 * kt][3], ahi[kt][1], alo[kt][1]);
        split_bf16x2(acc[2 * kt + 1][0], acc[2 * kt + 1][1], ahi[kt][2], alo[kt][2]);
        split_bf16x2(acc[2 * kt + 1][2], acc[2 * kt + 1][3], ahi[kt][3], alo[kt][3]);
    }
}

// y [B][3] = network(x [B][48]); with h1 (h1, h2, h3 non-null) the hidden
// activations are stored too (the training forward).  Persistent blocks of
// kTcWarps warps; warp w of block b takes the 16-row tiles b kTcWarps + w,
// then every gridDim.x kTcWarps tiles further.
__global__ void __launch_bounds__(32 * kTcWarps) k_mlp_fwd_tc(const float* x, const float* P, int64_t B, float* y,
                                                              float* h1, float* h2, float* h3) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* tiles = reinterpret_cast<uint32_t*>(smem_raw);
    float* bias = reinterpret_cast<float*>(tiles + kWTiles * kTileWords);
    fill_tiles(tiles + kOffT1 * kTileWords, P + kOffW1, kIn, kHid, kNt);
    fill_tiles(tiles + kOffT2 * kTileWords, P + kOffW2, kHid, kHid, kNt);
    fill_tiles(tiles + kOffT3 * kTileWords, P + kOffW3, kHid, kHid, kNt);
    fill_tiles(tiles + kOffT4 * kTileWords, P + kOffW4, kHid, kOut, 1);
    for (int e = threadIdx.x; e < kBiasF; e += blockDim.x) {
        float v = 0.f;
        if (e < kHid) v = P[kOffB1 + e];
        else if (e < 2 * kHid) v = P[kOffB2 + e - kHid];
        else if (e < 3 * kHid) v = P[kOffB3 + e - 2 * kHid];
        else if (e < 3 * kHid + kOut) v = P[kOffB4 + e - 3 * kHid];
        bias[e] = bf16r(v);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t ntiles = (B + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * kTcWarps + warp; tile < ntiles; tile += (int64_t)gridDim.x * kTcWarps) {
        const int64_t r0 = tile * 16, ra = r0 + g, rb = ra + 8;
        // layer 1 A fragments from the input rows
        uint32_t xhi[3][4], xlo[3][4];
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
            const int c = 16 * kt + 2 * t;
            float v[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cc = c + 8 * h;
                v[4 * h + 0] = ra < B ? x[ra * kIn + cc] : 0.f;
                v[4 * h + 1] = ra < B ? x[ra * kIn + cc + 1] : 0.f;
                v[4 * h + 2] = rb < B ? x[rb * kIn + cc] : 0.f;
                v[4 * h + 3] = rb < B ? x[rb * kIn + cc + 1] : 0.f;
            }
            split_bf16x2(v[0], v[1], xhi[kt][0], xlo[kt][0]);   // row g,     cols c, c+1
            split_bf16x2(v[2], v[3], xhi[kt][1], xlo[kt][1]);   // row g + 8, cols c, c+1
            split_bf16x2(v[4], v[5], xhi[kt][2], xlo[kt][2]);   // row g,     cols c+8, c+9
            split_bf16x2(v[6], v[7], xhi[kt][3], xlo[kt][3]);   // row g + 8, cols c+8, c+9
        }
        float acc[kNt][4];
        uint32_t ahi[8][4], alo[8][4];
        tc_layer<3>(xhi, xlo, tiles + kOffT1 * kTileWords, acc, lane);
        tc_activate(acc, bias, h1, r0, B, lane, ahi, alo);
        tc_layer<8>(ahi, alo, tiles + kOffT2 * kTileWords, acc, lane);
        tc_activate(acc, bias + kHid, h2, r0, B, lane, ahi, alo);
        tc_layer<8>(ahi, alo, tiles + kOffT3 * kTileWords, acc, lane);
        tc_activate(acc, bias + 2 * kHid, h3, r0, B, lane, ahi, alo);
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 8; ++kt) {
            const uint2 b = reinterpret_cast<const uint2*>(tiles + (kOffT4 + kt) * kTileWords)[lane];
            mma_bf16(o, ahi[kt], b.x, b.y);
            mma_bf16(o, alo[kt], b.x, b.y);
        }
        // lane (g, t) holds columns 2t, 2t + 1 of rows g and g + 8; columns < 3 are outputs
        const float* b4 = bias + 3 * kHid;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int col = 2 * t + q;
            if (col < kOut) {
                if (ra < B) y[ra * kOut + col] = o[q] + b4[col];
                if (rb < B) y[rb * kOut + col] = o[2 + q] + b4[col];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Backward on the tensor cores.
// ---------------------------------------------------------------------------
// B fragments of dX = dY W (W [N][K] row-major; the mma reduces over n and
// its columns are k): tile (kt over N/16, padded; nt over K/8), lane 4g + t,
// register r: W[16kt + 2t + 8r][8nt + g] and W[16kt + 2t + 8r + 1][8nt + g],
// BF16-rounded, zero for n >= N.
__device__ void fill_tiles_t(uint32_t* dst, const float* W, int K, int N, int kt_count) {
    const int nt_count = K / 8;
    const int ntiles = kt_count * nt_count;
    for (int e = threadIdx.x; e < ntiles * kTileWords; e += blockDim.x) {
        const int tile = e / kTileWords, word = e % kTileWords;
        const int kt = tile / nt_count, nt = tile % nt_count;
        const int lane = word >> 1, r = word & 1;
        const int n = 16 * kt + 2 * (lane & 3) + 8 * r, k = 8 * nt + (lane >> 2);
        const float a = n < N ? W[(int64_t)n * K + k] : 0.f;
        const float b = n + 1 < N ? W[(int64_t)(n + 1) * K + k] : 0.f;
        dst[e] = bf16x2_bits(__floats2bfloat162_rn(a, b));
    }
}

constexpr int kBwT3 = 1 * kNt;                  // dY (3 columns, padded to 16) times W4: 1 x 16 tiles
constexpr int kBwOffT3 = 0, kBwOffT2 = kBwT3, kBwOffT1 = kBwT3 + kL2Tiles;
constexpr int kBwTiles = kBwT3 + 2 * kL2Tiles;  // 272 tiles = 69,632 bytes
constexpr size_t kBwSmem = sizeof(uint32_t) * kBwTiles * kTileWords;

// ReLU mask of a layer's accumulators from its stored activations, the
// store of the gradient with respect to the pre-activations, and the next
// (earlier) layer's A fragments, as in tc_activate.
__device__ __forceinline__ void tc_relu_grad(float (&acc)[kNt][4], const float* h, float* dstore, int64_t r0,
                                             int64_t B, int lane, uint32_t (&ahi)[8][4], uint32_t (&alo)[8][4]) {
    const int g = lane >> 2, t = lane & 3;
    const int64_t ra = r0 + g, rb = ra + 8;
#pragma unroll
    for (int nt = 0; nt < kNt; ++nt) {
        const int col = 8 * nt + 2 * t;
        const float2 ha = ra < B ? *reinterpret_cast<const float2*>(h + ra * kHid + col) : make_float2(0.f, 0.f);
        const float2 hb = rb < B ? *reinterpret_cast<const float2*>(h + rb * kHid + col) : make_float2(0.f, 0.f);
        acc[nt][0] = ha.x > 0.f ? acc[nt][0] : 0.f;
        acc[nt][1] = ha.y > 0.f ? acc[nt][1] : 0.f;
        acc[nt][2] = hb.x > 0.f ? acc[nt][2] : 0.f;
        acc[nt][3] = hb.y > 0.f ? acc[nt][3] : 0.f;
        if (ra < B) *reinterpret_cast<float2*>(dstore + ra * kHid + col) = make_float2(acc[nt][0], acc[nt][1]);
        if (rb < B) *reinterpret_cast<float2*>(dstore + rb * kHid + col) = make_float2(acc[nt][2], acc[nt][3]);
    }
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
        split_bf16x2(acc[2 * kt][0], acc[2 * kt][1], ahi[kt][0], alo[kt][0]);
        split_bf16x2(acc[2 * kt][2], acc[2 * kt][3], ahi[kt][1], alo[kt][1]);
        split_bf16x2(acc[2 * kt + 1][0], acc[2 * kt + 1][1], ahi[kt][2], alo[kt][2]);
        split_bf16x2(acc[2 * kt + 1][2], acc[2 * kt + 1][3], ahi[kt][3], alo[kt][3]);
    }
}

// Gradients with respect to the three hidden pre-activations, fused:
//   d3 = (dout W4) * (h3 > 0),  d2 = (d3 W3) * (h2 > 0),  d1 = (d2 W2) * (h1 > 0)
// (dout [B][3]; h, d [B][128]).  Persistent blocks as in the forward.
__global__ void __launch_bounds__(32 * kTcWarps) k_mlp_bwd_data_tc(const float* dout, const float* P, int64_t B,
                                                                   const float* h1, const float* h2, const float* h3,
                                                                   float* d1, float* d2, float* d3) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* tiles = reinterpret_cast<uint32_t*>(smem_raw);
    fill_tiles_t(tiles + kBwOffT3 * kTileWords, P + kOffW4, kHid, kOut, 1);
    fill_tiles_t(tiles + kBwOffT2 * kTileWords, P + kOffW3, kHid, kHid, kHid / 16);
    fill_tiles_t(tiles + kBwOffT1 * kTileWords, P + kOffW2, kHid, kHid, kHid / 16);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t ntiles = (B + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * kTcWarps + warp; tile < ntiles; tile += (int64_t)gridDim.x * kTcWarps) {
        const int64_t r0 = tile * 16, ra = r0 + g, rb = ra + 8;
        // A fragments of dout: columns 2t, 2t + 1 (< 3), the rest zero
        float v[4];
        v[0] = (ra < B && 2 * t < kOut) ? dout[ra * kOut + 2 * t] : 0.f;
        v[1] = (ra < B && 2 * t + 1 < kOut) ? dout[ra * kOut + 2 * t + 1] : 0.f;
        v[2] = (rb < B && 2 * t < kOut) ? dout[rb * kOut + 2 * t] : 0.f;
        v[3] = (rb < B && 2 * t + 1 < kOut) ? dout[rb * kOut + 2 * t + 1] : 0.f;
        uint32_t ohi[1][4], olo[1][4];
        split_bf16x2(v[0], v[1], ohi[0][0], olo[0][0]);
        split_bf16x2(v[2], v[3], ohi[0][1], olo[0][1]);
        ohi[0][2] = ohi[0][3] = olo[0][2] = olo[0][3] = 0u;   // columns 8..15 of the padded k-tile
        float acc[kNt][4];
        uint32_t ahi[8][4], alo[8][4];
        tc_layer<1>(ohi, olo, tiles + kBwOffT3 * kTileWords, acc, lane);
        tc_relu_grad(acc, h3, d3, r0, B, lane, ahi, alo);
        tc_layer<8>(ahi, alo, tiles + kBwOffT2 * kTileWords, acc, lane);
        tc_relu_grad(acc, h2, d2, r0, B, lane, ahi, alo);
        tc_layer<8>(ahi, alo, tiles + kBwOffT1 * kTileWords, acc, lane);
        tc_relu_grad(acc, h1, d1, r0, B, lane, ahi, alo);
    }
}

// Weight-gradient partials of one layer over one chunk of kChunk rows:
//   part[c][woff + n K + k] = sum_{b in chunk c} dY[b][n] X[b][k],
//   part[c][boff + n]       = sum_{b in chunk c} dY[b][n]
// on the tensor cores: the mma's rows are n (16 per warp), its columns k and
// its reduction the chunk's rows; both factors are FP32 activations and enter
// as BF16 hi + lo pairs (three products: hi hi, hi lo, lo hi).  The chunk's
// rows are staged 16 at a time in shared memory.  Block = kTcWarps warps,
// warp w takes rows n = 16w .. 16w + 15 (warps past N idle).
constexpr int kWgPad = 4;
__global__ void __launch_bounds__(32 * kTcWarps) k_mlp_bwd_weight_tc(const float* dY, const float* X, int64_t B,
                                                                     int K, int N, float* part, int woff, int boff) {
    __shared__ float ds[16][kHid + kWgPad];
    __shared__ float xs[16][kHid + kWgPad];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t b0 = (int64_t)blockIdx.x * kChunk, b1 = min(B, b0 + kChunk);
    const int n0 = 16 * warp;
    const int ntk = K / 8;                 // column tiles of this layer (6 or 16)
    float acc[kNt][4];
#pragma unroll
    for (int nt = 0; nt < kNt; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    float bsum = 0.f;                      // lanes 0..15: the bias gradient of row n0 + lane
    for (int64_t bb = b0; bb < b1; bb += 16) {
        for (int e = threadIdx.x; e < 16 * kHid; e += blockDim.x) {
            const int q = e / kHid, c = e % kHid;
            const int64_t row = bb + q;
            ds[q][c] = (row < b1 && c < N) ? dY[row * N + c] : 0.f;
            xs[q][c] = (row < b1 && c < K) ? X[row * K + c] : 0.f;
        }
        __syncthreads();
        if (n0 < N) {
            if (lane < 16) {
#pragma unroll
                for (int q = 0; q < 16; ++q) bsum += ds[q][n0 + lane];
            }
            // A: rows n0 + g (+8), reduction columns 2t, 2t + 1 (+8) = batch rows of the step
            uint32_t ahi[4], alo[4];
            split_bf16x2(ds[2 * t][n0 + g], ds[2 * t + 1][n0 + g], ahi[0], alo[0]);
            split_bf16x2(ds[2 * t][n0 + g + 8], ds[2 * t + 1][n0 + g + 8], ahi[1], alo[1]);
            split_bf16x2(ds[2 * t + 8][n0 + g], ds[2 * t + 9][n0 + g], ahi[2], alo[2]);
            split_bf16x2(ds[2 * t + 8][n0 + g + 8], ds[2 * t + 9][n0 + g + 8], ahi[3], alo[3]);
#pragma unroll
            for (int nt = 0; nt < kNt; ++nt) {
                if (nt < ntk) {
                    const int k = 8 * nt + g;
                    uint32_t bhi0, blo0, bhi1, blo1;
                    split_bf16x2(xs[2 * t][k], xs[2 * t + 1][k], bhi0, blo0);
                    split_bf16x2(xs[2 * t + 8][k], xs[2 * t + 9][k], bhi1, blo1);
                    mma_bf16(acc[nt], ahi, bhi0, bhi1);
                    mma_bf16(acc[nt], ahi, blo0, blo1);
                    mma_bf16(acc[nt], alo, bhi0, bhi1);
                }
            }
        }
        __syncthreads();
    }
    if (n0 >= N) return;
    float* Pc = part + (int64_t)blockIdx.x * kParams;
#pragma unroll
    for (int nt = 0; nt < kNt; ++nt) {
        if (nt >= ntk) continue;
        const int k = 8 * nt + 2 * t;
        const int na = n0 + g, nb = na + 8;
        if (na < N) { Pc[woff + na * K + k] = acc[nt][0]; Pc[woff + na * K + k + 1] = acc[nt][1]; }
        if (nb < N) { Pc[woff + nb * K + k] = acc[nt][2]; Pc[woff + nb * K + k + 1] = acc[nt][3]; }
    }
    if (lane < 16 && n0 + lane < N) Pc[boff + n0 + lane] = bsum;
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

// Fused tensor-core forward of B rows; with keep, the hidden activations go
// to m.h1..h3 (B <= max_batch then).
static void forward_tc(Mlp& m, const float* x, int64_t B, float* y, bool keep, cudaStream_t s) {
    // the attribute is set on the current device's copy of the kernel (every call: it is cheap)
    WNNC_CUDA(cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
    int dev = 0, sms = 0, per_sm = 0;
    WNNC_CUDA(cudaGetDevice(&dev));
    WNNC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WNNC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_fwd_tc, 32 * kTcWarps, kTcSmem));
    // persistent blocks: as many as are resident at once, fewer for small batches
    const int64_t tiles = (B + 15) / 16;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * sms, (tiles + kTcWarps - 1) / kTcWarps));
    k_mlp_fwd_tc<<<grid, 32 * kTcWarps, kTcSmem, s>>>(x, m.params, B, y, keep ? m.h1 : nullptr,
                                                      keep ? m.h2 : nullptr, keep ? m.h3 : nullptr);
    WNNC_LAUNCH_CHECK();
}

// The FP32 SIMT forward of B <= max_batch rows into m.h1..h3 and y (kept for
// comparison with the tensor-core path; not used by the entry points).
[[maybe_unused]] static void forward_rows_simt(Mlp& m, const float* x, int64_t B, float* y, cudaStream_t s) {
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
    forward_tc(m, x, B, y, false, s);
}

static void k_lin_bwd_weight_tc_launch(const float* dY, const float* X, int64_t B, int K, int N, float* part,
                                       int woff, int boff, int nch, cudaStream_t s) {
    k_mlp_bwd_weight_tc<<<nch, 32 * kTcWarps, 0, s>>>(dY, X, B, K, N, part, woff, boff);
    WNNC_LAUNCH_CHECK();
}

// Gradient of the mean loss over B <= max_batch rows into m.grad; loss to loss_dev.
void mlp_grad(Mlp& m, const float* x, const float* label, int64_t B, float* loss_dev, cudaStream_t s) {
    forward_tc(m, x, B, m.out, true, s);
    const int nlb = ceil_div(B, 256);
    k_cos_loss<<<nlb, 256, 0, s>>>(m.out, label, B, m.loss_mode, m.dout, m.lpart);
    WNNC_LAUNCH_CHECK();
    if (loss_dev) {
        k_loss_final<<<1, 1, 0, s>>>(m.lpart, nlb, B, loss_dev);
        WNNC_LAUNCH_CHECK();
    }
    const float* P = m.params;
    const int nch = ceil_div(B, kChunk);
    // gradients with respect to the hidden pre-activations, fused on the tensor cores
    WNNC_CUDA(cudaFuncSetAttribute(k_mlp_bwd_data_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwSmem));
    int dev = 0, sms = 0, per_sm = 0;
    WNNC_CUDA(cudaGetDevice(&dev));
    WNNC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WNNC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_bwd_data_tc, 32 * kTcWarps, kBwSmem));
    const int64_t rtiles = (B + 15) / 16;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * sms, (rtiles + kTcWarps - 1) / kTcWarps));
    k_mlp_bwd_data_tc<<<grid, 32 * kTcWarps, kBwSmem, s>>>(m.dout, P, B, m.h1, m.h2, m.h3, m.d1, m.d2, m.d3);
    WNNC_LAUNCH_CHECK();
    // weight gradients per chunk of rows, on the tensor cores
    k_lin_bwd_weight_tc_launch(m.dout, m.h3, B, kHid, kOut, m.part, kOffW4, kOffB4, nch, s);
    k_lin_bwd_weight_tc_launch(m.d3, m.h2, B, kHid, kHid, m.part, kOffW3, kOffB3, nch, s);
    k_lin_bwd_weight_tc_launch(m.d2, m.h1, B, kHid, kHid, m.part, kOffW2, kOffB2, nch, s);
    k_lin_bwd_weight_tc_launch(m.d1, x, B, kIn, kHid, m.part, kOffW1, kOffB1, nch, s);
    k_sum_partials<<<ceil_div(kParams, 256), 256, 0, s>>>(m.part, nch, m.grad);
    WNNC_LAUNCH_CHECK();
}

// The FP32 SIMT backward of B <= max_batch rows (kept for comparison with the
// tensor-core path; not used by the entry points).
[[maybe_unused]] static void backward_simt(Mlp& m, const float* x, int64_t B, cudaStream_t s) {
    const float* P = m.params;
    const int nch = ceil_div(B, kChunk);
    k_lin_bwd_weight<<<dim3(1, 2, nch), 256, 0, s>>>(m.dout, m.h3, B, kHid, kOut, m.part, kOffW4, kOffB4);
    k_lin_bwd_data<<<grid2(B, kHid), 256, 0, s>>>(m.dout, P + kOffW4, m.h3, m.d3, B, kHid, kOut);
    k_lin_bwd_weight<<<dim3(2, 2, nch), 256, 0, s>>>(m.d3, m.h2, B, kHid, kHid, m.part, kOffW3, kOffB3);
    k_lin_bwd_data<<<grid2(B, kHid), 256, 0, s>>>(m.d3, P + kOffW3, m.h2, m.d2, B, kHid, kHid);
    k_lin_bwd_weight<<<dim3(2, 2, nch), 256, 0, s>>>(m.d2, m.h1, B, kHid, kHid, m.part, kOffW2, kOffB2);
    k_lin_bwd_data<<<grid2(B, kHid), 256, 0, s>>>(m.d2, P + kOffW2, m.h1, m.d1, B, kHid, kHid);
    k_lin_bwd_weight<<<dim3(2, 1, nch), 256, 0, s>>>(m.d1, x, B, kIn, kHid, m.part, kOffW1, kOffB1);
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
