// noalloc.cu -- winding number at query points by direct summation, with no
// device allocation at all.
//
// Who needs this: code that runs where cudaMalloc is off limits -- inside a
// host application that owns all device memory through its own pool and
// forbids other allocations, in a plugin sandbox, or in a latency-critical
// path where an allocation (which can synchronise the device) is not
// acceptable.  Such a caller passes its own input and output buffers; the only
// other memory this path touches is one fixed-size array in the library's own
// device image.
//
// The kernels here are variants of the normalisation reduction of the tree
// build (bounding box -> centre and scale) and of the gather sum of A, with
// their scratch (per-block bounding-box partials, the normalised sources)
// placed in a file-scope __device__ array instead of memory from cudaMalloc.
//
// The scratch array is shared by every call in the process on a given device
// and keeps the last call's contents; every call rewrites all of it that it
// reads (the non-finite flags are rewritten by the box reduction before the
// query kernel can set one), so nothing needs clearing, but two calls whose
// kernels overlap on the GPU (different streams, no ordering between them)
// race on it.
//
// Non-finite input.  Like every other entry point, this one rejects a NaN or
// infinite point or query coordinate with WNNC_EINVAL: the box reduction and
// the query kernel raise flags in the scratch, and the call reads the two
// flags back (an 8-byte copy into a host variable, then a wait on the stream)
// before it returns.
#include <mutex>

#include "common.cuh"

namespace wnnc {

namespace {

constexpr int kNaMaxSources = 32768;                // largest source cloud accepted
constexpr int kNaBlocks = 256;                      // bounding-box reduction blocks
constexpr int kNaThreads = 256;
constexpr size_t kNaPartBytes = sizeof(double) * 7 * kNaBlocks;   // 14 KiB: box + non-finite count
constexpr size_t kNaCsBytes = 256;                                // NaCs below, padded
constexpr size_t kNaSrcBytes = sizeof(float4) * kNaMaxSources;    // 512 KiB per array
constexpr size_t kNaScratchBytes = kNaPartBytes + kNaCsBytes + 2 * kNaSrcBytes;
constexpr int kNaMaxDevices = 64;

}  // namespace

// The scratch: about 1 MiB, held by every GPU that loads the library until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

namespace {

// Normalisation of one call, and the two non-finite flags (set to 0 by the
// box reduction of the same call, raised by the query kernel).
struct NaCs {
    double center[3];
    double scale;
    int bad_points;    // a point coordinate is NaN or infinite
    int bad_queries;   // a query coordinate is NaN or infinite
};
static_assert(sizeof(NaCs) <= kNaCsBytes, "NaCs does not fit its scratch slot");

__global__ void k_na_bbox_partial(const float* pts, int64_t n, double* part) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float f = pts[3 * i + k];
            bad |= !isfinite(f);
            double v = (double)f;
            lo[k] = fmin(lo[k], v);
            hi[k] = fmax(hi[k], v);
        }
    }
    bad = __syncthreads_or(bad);
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
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            for (int k = 0; k < 3; ++k) {
                lo[k] = fmin(lo[k], sh[0][k][w]);
                hi[k] = fmax(hi[k], sh[1][k][w]);
            }
        for (int k = 0; k < 3; ++k) { part[7 * blockIdx.x + k] = lo[k]; part[7 * blockIdx.x + 3 + k] = hi[k]; }
        part[7 * blockIdx.x + 6] = bad ? 1.0 : 0.0;
    }
}

// Same normalisation as the tree build (Sec. 5.1.1): bounding-box centre and
// the scale that maps the largest half-extent to 10/11.
__global__ void k_na_bbox_final(const double* part, int nparts, NaCs* cs) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int b = 0; b < nparts; ++b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], part[7 * b + k]);
            hi[k] = fmax(hi[k], part[7 * b + 3 + k]);
        }
        bad |= part[7 * b + 6] != 0.0;
    }
    double hmax = 0.0;
    for (int k = 0; k < 3; ++k) {
        cs->center[k] = __dmul_rn(__dadd_rn(lo[k], hi[k]), 0.5);
        double h = __dmul_rn(__dsub_rn(hi[k], lo[k]), 0.5);
        if (h > hmax) hmax = h;
    }
    cs->scale = hmax > 0.0 ? (10.0 / 11.0) / hmax : 1.0;
    cs->bad_points = bad;
    cs->bad_queries = 0;
}

// Normalised sources (float) and mu' = s^2 mu, into the scratch.
__global__ void k_na_pack(const float* pts, const float* mu, int64_t n, const NaCs* cs, float4* spos,
                          float4* smu) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = cs->scale;
    const double* c = cs->center;
    const float s2 = (float)(s * s);
    spos[i] = make_float4((float)__dmul_rn(__dsub_rn((double)pts[3 * i], c[0]), s),
                          (float)__dmul_rn(__dsub_rn((double)pts[3 * i + 1], c[1]), s),
                          (float)__dmul_rn(__dsub_rn((double)pts[3 * i + 2], c[2]), s), 0.f);
    smu[i] = make_float4(mu[3 * i] * s2, mu[3 * i + 1] * s2, mu[3 * i + 2] * s2, 0.f);
}

// Warp per 32 queries; sources staged 32 at a time through shared memory.
//   F(q) = sum_j (x_j - q) . mu_j / (4 pi r^3), terms with r < w dropped.
__global__ void __launch_bounds__(128) k_na_direct_w(const float* q, int64_t m, NaCs* cs,
                                                     const float4* spos, const float4* smu, int n, float w2,
                                                     float* out) {
    __shared__ float4 sp_all[4][32], sv_all[4][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * 4 + wl;
    const int64_t i = g * 32 + lane;
    if (g * 32 >= m) return;
    float4* sp = sp_all[wl];
    float4* sv = sv_all[wl];
    const bool valid = i < m;
    const double s = cs->scale;
    const double* c = cs->center;
    float tx = 0.f, ty = 0.f, tz = 0.f;
    if (valid) {
        const float qx = q[3 * i], qy = q[3 * i + 1], qz = q[3 * i + 2];
        if (!isfinite(qx) || !isfinite(qy) || !isfinite(qz)) cs->bad_queries = 1;
        tx = (float)__dmul_rn(__dsub_rn((double)qx, c[0]), s);
        ty = (float)__dmul_rn(__dsub_rn((double)qy, c[1]), s);
        tz = (float)__dmul_rn(__dsub_rn((double)qz, c[2]), s);
    }
    float acc = 0.f;
    for (int base = 0; base < n; base += 32) {
        const int cnt = min(32, n - base);
        if (lane < cnt) {
            sp[lane] = spos[base + lane];
            sv[lane] = smu[base + lane];
        }
        __syncwarp();
#pragma unroll 4
        for (int k = 0; k < cnt; ++k) {
            const float4 p = sp[k], v = sv[k];
            const float dx = p.x - tx, dy = p.y - ty, dz = p.z - tz;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ir = (r2 >= w2) ? rsqrtf(r2) : 0.f;
            acc = fmaf(fmaf(dx, v.x, fmaf(dy, v.y, dz * v.z)), ir * ir * ir, acc);
        }
        __syncwarp();
    }
    if (valid) out[i] = acc * kInv4Pi;
}

std::mutex g_na_mutex;
unsigned char* g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in and must never be passed
// to a kernel).
unsigned char* scratch_on_current_device() {
    int dev = 0;
    WNNC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) fail(WNNC_EINVAL, "device ordinal out of range for the no-alloc path");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(WNNC_ECUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    return g_na_ptr[dev];
}

}  // namespace

static wnnc_status na_guard(const std::string& what, void (*fn)(void*), void* ctx) {
    try {
        fn(ctx);
        return WNNC_OK;
    } catch (const Error& e) {
        set_last_error(what + ": " + e.msg);
        return e.status;
    } catch (...) {
        set_last_error(what + ": unexpected internal error");
        return WNNC_ECUDA;
    }
}

}  // namespace wnnc

using namespace wnnc;

namespace {
struct NaCall {
    const float* pts;
    int64_t n;
    const float* mu;
    const float* q;
    int64_t m;
    float w;
    float* out;
    cudaStream_t s;
};

void na_run(void* vctx) {
    NaCall& c = *static_cast<NaCall*>(vctx);
    if (!c.pts || !c.mu || !c.q || !c.out) fail(WNNC_EINVAL, "pts/mu/q/out is NULL");
    if (c.n < 1 || c.m < 1) fail(WNNC_EINVAL, "n and m must be >= 1");
    if (c.n > kNaMaxSources)
        fail(WNNC_EINVAL, "n = " + std::to_string(c.n) + " exceeds the no-alloc limit of " +
                              std::to_string(kNaMaxSources) + " source points");
    if (c.m > (int64_t)INT32_MAX * 16) fail(WNNC_EINVAL, "m too large");
    if (!(c.w >= 0.f) || !(c.w < INFINITY)) fail(WNNC_EINVAL, "w must be finite and >= 0");
    unsigned char* base = scratch_on_current_device();
    double* part = reinterpret_cast<double*>(base);
    NaCs* cs = reinterpret_cast<NaCs*>(base + kNaPartBytes);
    float4* spos = reinterpret_cast<float4*>(base + kNaPartBytes + kNaCsBytes);
    float4* smu = reinterpret_cast<float4*>(base + kNaPartBytes + kNaCsBytes + kNaSrcBytes);
    k_na_bbox_partial<<<kNaBlocks, kNaThreads, 0, c.s>>>(c.pts, c.n, part);
    WNNC_LAUNCH_CHECK();
    k_na_bbox_final<<<1, 1, 0, c.s>>>(part, kNaBlocks, cs);
    WNNC_LAUNCH_CHECK();
    k_na_pack<<<ceil_div(c.n, kNaThreads), kNaThreads, 0, c.s>>>(c.pts, c.mu, c.n, cs, spos, smu);
    WNNC_LAUNCH_CHECK();
    const float w2 = fmaxf(c.w * c.w, 0x1p-40f);   // same cut-off and coincidence floor as the tree path
    const int64_t groups = (c.m + 31) / 32;
    k_na_direct_w<<<(unsigned)((groups + 3) / 4), 128, 0, c.s>>>(c.q, c.m, cs, spos, smu, (int)c.n, w2, c.out);
    WNNC_LAUNCH_CHECK();
    // Read the two flags back: a copy into host stack memory (no allocation),
    // then a wait on the call's stream.
    int flags[2] = {0, 0};
    WNNC_CUDA(cudaMemcpyAsync(flags, &cs->bad_points, sizeof(flags), cudaMemcpyDeviceToHost, c.s));
    WNNC_CUDA(cudaStreamSynchronize(c.s));
    if (flags[0]) fail(WNNC_EINVAL, "a point coordinate is not finite");
    if (flags[1]) fail(WNNC_EINVAL, "a query coordinate is not finite");
}
}  // namespace

extern "C" wnnc_status wnnc_eval_w_direct_noalloc(const float* pts, int64_t n, const float* mu,
                                                  const float* q, int64_t m, float w, float* out,
                                                  void* stream) {
    NaCall c{pts, n, mu, q, m, w, out, static_cast<cudaStream_t>(stream)};
    return na_guard("wnnc_eval_w_direct_noalloc", na_run, &c);
}
