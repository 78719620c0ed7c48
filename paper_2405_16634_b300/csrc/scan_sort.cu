// scan_sort.cu -- device-wide exclusive scan, stable LSD radix sort and
// segment offsets, used by the tree and interaction-list construction.
#include <utility>

#include "common.cuh"

namespace wnnc {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ T warp_inclusive_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one block's thread values; the block total goes to *total.
template <class T>
__device__ T block_exclusive_scan(T v, T* total) {
    __shared__ T wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_inclusive_scan(v);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T x = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : T(0);
        T xs = warp_inclusive_scan(x);
        wsum[lane] = xs - x;
        if (lane == 31) *total = xs;
    }
    __syncthreads();
    T r = inc - v + wsum[warp];
    __syncthreads();
    return r;
}

template <class T>
__global__ void k_scan_reduce(const T* in, int64_t n, T* bsum) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    __shared__ T tot;
    block_exclusive_scan<T>(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// out[i] = sum of in[0..i) (+ block offset); out[n] = total.  In place is safe:
// each thread reads its items before the block barrier inside the scan.
template <class T>
__global__ void k_scan_apply(const T* in, T* out, int64_t n, const T* boff) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : T(0);
        s += v[k];
    }
    __shared__ T tot;
    T ex = block_exclusive_scan<T>(s, &tot) + (boff ? boff[blockIdx.x] : T(0));
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (base + kScanItems >= n && base < n) out[n] = ex;   // the thread holding the last item
}

template <class T>
__global__ void k_set_zero_total(T* out) { out[0] = 0; }

template <class T>
void exclusive_scan_impl(const T* in, T* out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        k_set_zero_total<T><<<1, 1, 0, s>>>(out);
        WNNC_LAUNCH_CHECK();
        return;
    }
    int nb = ceil_div(n, kScanTile);
    if (nb == 1) {
        k_scan_apply<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        WNNC_LAUNCH_CHECK();
        return;
    }
    T* bsum = dalloc<T>(nb + 1);
    k_scan_reduce<T><<<nb, kScanThreads, 0, s>>>(in, n, bsum);
    WNNC_LAUNCH_CHECK();
    exclusive_scan_impl<T>(bsum, bsum, nb, s);
    k_scan_apply<T><<<nb, kScanThreads, 0, s>>>(in, out, n, bsum);
    WNNC_LAUNCH_CHECK();
    // the pool frees in the order of its stream: no wait when that is s
    if (alloc_stream() != s) WNNC_CUDA(cudaStreamSynchronize(s));
    pool_free(bsum);
}

// ---------------------------------------------------------------------------
// Radix sort: RB-bit digits (8 or 9: a sort of b key bits takes the digit width
// that needs the fewest passes), tiles of 2048 keys (8 warps x 8 rounds x 32
// lanes).  Ranks inside a tile are stable: warps in order, rounds in order,
// and lanes in order within a round (peers found with match_any).
// ---------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 8;
constexpr int kRsTile = kRsThreads * kRsRounds;

template <int RB>
__global__ void k_rs_hist(const uint64_t* keys, int64_t n, int shift, int* hist, int nblocks) {
    constexpr int kB = 1 << RB;
    constexpr unsigned kMask = kB - 1u;
    __shared__ int h[kB];
    for (int d = threadIdx.x; d < kB; d += kRsThreads) h[d] = 0;
    __syncthreads();
    int64_t t0 = (int64_t)blockIdx.x * kRsTile;
    for (int k = threadIdx.x; k < kRsTile; k += kRsThreads) {
        int64_t i = t0 + k;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & kMask], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kB; d += kRsThreads) hist[d * nblocks + blockIdx.x] = h[d];
}

// Scatter of one tile: the keys are ranked stably by digit into shared memory
// (warps in order, rounds in order, lanes in order within a round), then
// written out in that order, so that each digit's keys go to consecutive
// global positions (coalesced runs instead of 32 scattered stores a warp).
// wcnt holds each warp's digit counts, then (in place) each warp's first
// tile position per digit.
template <int RB>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* kin, const uint32_t* vin,
                                                           uint64_t* kout, uint32_t* vout, int64_t n,
                                                           int shift, const int* offs, int nblocks) {
    constexpr int kB = 1 << RB;
    constexpr int kPer = kB / kRsThreads;     // digits per thread in the tile scan (1 or 2)
    constexpr unsigned kMask = kB - 1u;
    __shared__ int wcnt[kRsWarps][kB];
    __shared__ int gbase[kB];
    __shared__ int wsum[kRsWarps];
    __shared__ uint64_t skey[kRsTile];
    __shared__ uint32_t sval[kRsTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < kRsWarps * kB; i += kRsThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kRsTile;
    const int tcount = (int)(n - t0 < (int64_t)kRsTile ? n - t0 : (int64_t)kRsTile);
    const int64_t w0 = t0 + (int64_t)warp * (32 * kRsRounds);
    for (int r = 0; r < kRsRounds; ++r) {
        int64_t i = w0 + r * 32 + lane;
        bool valid = i < n;
        unsigned vmask = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            unsigned d = (unsigned)((kin[i] >> shift) & kMask);
            unsigned peers = __match_any_sync(vmask, d);
            if (lane == __ffs(peers) - 1) wcnt[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    {
        // tile-local start of each digit: thread j takes digits kPer j .. kPer j + kPer - 1,
        // an exclusive scan over the threads gives their starts
        int tot[kPer];
        int mine = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int d = kPer * threadIdx.x + q;
            tot[q] = 0;
            for (int w = 0; w < kRsWarps; ++w) tot[q] += wcnt[w][d];
            mine += tot[q];
        }
        int x = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        int ds = before + x - mine;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int d = kPer * threadIdx.x + q;
            gbase[d] = offs[d * nblocks + blockIdx.x] - ds;
            int run = ds;
            for (int w = 0; w < kRsWarps; ++w) {
                const int c = wcnt[w][d];
                wcnt[w][d] = run;
                run += c;
            }
            ds += tot[q];
        }
    }
    __syncthreads();
    for (int r = 0; r < kRsRounds; ++r) {
        int64_t i = w0 + r * 32 + lane;
        bool valid = i < n;
        unsigned vmask = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            uint64_t key = kin[i];
            unsigned d = (unsigned)((key >> shift) & kMask);
            unsigned peers = __match_any_sync(vmask, d);
            int base = wcnt[warp][d];
            int pos = base + __popc(peers & lt_mask);
            skey[pos] = key;
            if (vin) sval[pos] = vin[i];
            __syncwarp(vmask);
            if (lane == __ffs(peers) - 1) wcnt[warp][d] = base + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int p = threadIdx.x; p < tcount; p += kRsThreads) {
        const uint64_t key = skey[p];
        const int gpos = gbase[(key >> shift) & kMask] + p;
        kout[gpos] = key;
        if (vout) vout[gpos] = sval[p];
    }
}

__global__ void k_seg_off(const uint64_t* keys, int64_t n, int* off, int ng, int shift) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t g = (int64_t)(keys[i] >> shift);
    int64_t gp = i > 0 ? (int64_t)(keys[i - 1] >> shift) : -1;
    for (int64_t q = gp + 1; q <= g && q <= ng; ++q) off[q] = (int)i;
    if (i == n - 1)
        for (int64_t q = g + 1; q <= ng; ++q) off[q] = (int)n;
}

__global__ void k_fill_i32(int* p, int64_t n, int v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

void exclusive_scan_i32(const int* in, int* out, int64_t n, cudaStream_t s) {
    exclusive_scan_impl<int>(in, out, n, s);
}
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    exclusive_scan_impl<int64_t>(in, out, n, s);
}

void radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s, int lo_bit) {
    if (n <= 1 || bits <= lo_bit) return;
    if (n > (int64_t)INT32_MAX) fail(WNNC_EINVAL, "radix_sort_pairs: too many keys");
    int nb = ceil_div(n, kRsTile);
    uint64_t* k2 = dalloc<uint64_t>(n);
    uint32_t* v2 = vals ? dalloc<uint32_t>(n) : nullptr;
    // digit width: 8 bits, or 9 where that saves a pass (e.g. 18 bits: 2 passes, not 3)
    const int nbits = bits - lo_bit;
    const int passes8 = (nbits + 7) / 8, passes9 = (nbits + 8) / 9;
    const int rb = passes9 < passes8 ? 9 : 8;
    const int passes = rb == 9 ? passes9 : passes8;
    int* hist = dalloc<int>(((size_t)1 << rb) * nb + 1);
    uint64_t *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes; ++p) {
        int shift = lo_bit + rb * p;
        if (rb == 9) k_rs_hist<9><<<nb, kRsThreads, 0, s>>>(ka, n, shift, hist, nb);
        else k_rs_hist<8><<<nb, kRsThreads, 0, s>>>(ka, n, shift, hist, nb);
        WNNC_LAUNCH_CHECK();
        exclusive_scan_i32(hist, hist, ((int64_t)1 << rb) * nb, s);
        if (rb == 9) k_rs_scatter<9><<<nb, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist, nb);
        else k_rs_scatter<8><<<nb, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist, nb);
        WNNC_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        WNNC_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (vals) WNNC_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    if (alloc_stream() != s) WNNC_CUDA(cudaStreamSynchronize(s));
    pool_free(k2);
    if (v2) pool_free(v2);
    pool_free(hist);
}

void segment_offsets_hi32(const uint64_t* keys, int64_t n, int* off, int ng, cudaStream_t s, int shift) {
    if (n == 0) {
        k_fill_i32<<<ceil_div(ng + 1, 256), 256, 0, s>>>(off, ng + 1, 0);
        WNNC_LAUNCH_CHECK();
        return;
    }
    k_seg_off<<<ceil_div(n, 256), 256, 0, s>>>(keys, n, off, ng, shift);
    WNNC_LAUNCH_CHECK();
}

}  // namespace wnnc
