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

// ---------------------------------------------------------------------------
// Single-pass prefix sums across blocks (decoupled look-back).  A block takes
// the next tile index from an atomic counter, so that every tile it waits on
// belongs to a block that has started; it publishes its tile's total
// (status "aggregate") at once, then walks back over the earlier tiles (a
// warp 32 tiles at a time in the scans, a thread one tile at a time per digit
// column in the radix passes), adding their totals until it meets one whose
// inclusive prefix is known (status "inclusive"), and publishes its own
// inclusive prefix.  A look-back word
// holds the status in bits 62-63 and the (non-negative) value below, so one
// relaxed 64-bit load or store moves both.  Every wait is bounded: past
// kWaitPolls polls the block counts a timeout in g_wait_timeouts (read by
// the host, which then fails the build) and goes on.
// ---------------------------------------------------------------------------
constexpr unsigned long long kLbAgg = 1ull << 62, kLbIncl = 2ull << 62, kLbVal = (1ull << 62) - 1;
constexpr int kWaitPolls = 1 << 20;   // with back-off: well under a second of polling

__device__ unsigned g_wait_timeouts;

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void lb_store(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive prefix of tile `tile` for one look-back column (stride between
// tiles: `stride` words).  Returns the sum of the earlier tiles' values.
__device__ __forceinline__ unsigned long long lb_prefix(const unsigned long long* look, int tile, int stride) {
    unsigned long long excl = 0;
    int p = tile - 1, polls = 0;
    while (p >= 0) {
        const unsigned long long v = lb_load(look + (size_t)p * stride);
        if ((v >> 62) == 0) {
            if (++polls > kWaitPolls) {
                atomicAdd(&g_wait_timeouts, 1u);
                break;
            }
            if (polls > 64) __nanosleep(64);
            continue;
        }
        excl += v & kLbVal;
        if ((v & ~kLbVal) == kLbIncl) break;
        --p;
    }
    return excl;
}

// out[i] = sum of in[0..i); out[n] = total (in place is safe: a tile is read
// before any of its outputs is written).  look: [0] the tile counter, then one
// word per tile, zeroed by the caller.
template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_chained(const T* in, T* out, int64_t n,
                                                               unsigned long long* look) {
    __shared__ int s_tile;
    __shared__ T s_excl;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(look, 1ull);
    __syncthreads();
    const int tile = s_tile;
    const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : T(0);
        sum += v[k];
    }
    __shared__ T tot;
    T ex = block_exclusive_scan<T>(sum, &tot);
    unsigned long long* w = look + 1;
    if (threadIdx.x < 32) {
        // the first warp publishes the tile's total, then looks back 32 tiles
        // at a time: it waits for all 32 words, and adds them up to the
        // nearest inclusive one (tiles before 0 count as an inclusive 0)
        const int lane = threadIdx.x;
        const unsigned long long agg = (unsigned long long)tot & kLbVal;
        if (lane == 0) lb_store(w + tile, (tile == 0 ? kLbIncl : kLbAgg) | agg);
        unsigned long long e = 0;
        int p = tile - 1, polls = 0;
        bool gave_up = false;
        while (tile > 0 && !gave_up) {
            const int q = p - lane;
            unsigned long long v = q >= 0 ? lb_load(w + q) : kLbIncl;
            while (__any_sync(0xffffffffu, (v >> 62) == 0)) {
                if (++polls > kWaitPolls) {
                    if (lane == 0) atomicAdd(&g_wait_timeouts, 1u);
                    gave_up = true;
                    break;
                }
                if (polls > 64) __nanosleep(64);
                if ((v >> 62) == 0) v = lb_load(w + q);
            }
            const unsigned incl = __ballot_sync(0xffffffffu, (v & ~kLbVal) == kLbIncl);
            const int j = incl ? __ffs(incl) - 1 : 31;
            unsigned long long x = lane <= j ? (v & kLbVal) : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            e += x;
            if (incl) break;
            p -= 32;
        }
        if (lane == 0) {
            if (tile > 0) lb_store(w + tile, kLbIncl | ((e + agg) & kLbVal));
            s_excl = (T)e;
        }
    }
    __syncthreads();
    ex += s_excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (base + kScanItems >= n && base < n) out[n] = ex;   // the thread holding the last item
}

// One tile: out[i] = sum of in[0..i), out[n] = total.
template <class T>
__global__ void k_scan_apply(const T* in, T* out, int64_t n) {
    int64_t base = (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : T(0);
        s += v[k];
    }
    __shared__ T tot;
    T ex = block_exclusive_scan<T>(s, &tot);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (base + kScanItems >= n && base < n) out[n] = ex;
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
    const int64_t nb = ceil_div(n, kScanTile);
    if (nb == 1) {
        k_scan_apply<T><<<1, kScanThreads, 0, s>>>(in, out, n);
        WNNC_LAUNCH_CHECK();
        return;
    }
    unsigned long long* look = dalloc<unsigned long long>(nb + 1);
    WNNC_CUDA(cudaMemsetAsync(look, 0, sizeof(unsigned long long) * (nb + 1), s));
    k_scan_chained<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, look);
    WNNC_LAUNCH_CHECK();
    // the pool frees in the order of its stream: no wait when that is s
    if (alloc_stream() != s) WNNC_CUDA(cudaStreamSynchronize(s));
    pool_free(look);
}

// ---------------------------------------------------------------------------
// Radix sort: stable LSD over RB-bit digits (8 or 9: a sort of b key bits
// takes the digit width that needs the fewest passes), tiles of 2048 keys (8
// warps x 8 rounds x 32 lanes).  A pass ranks each tile's keys stably (warps
// in order, rounds in order, lanes in order within a round; peers found with
// match_any) and writes them out digit by digit.  A tile's place among the
// earlier tiles' keys of each digit comes, for sorts of few tiles, from
// decoupled look-back (one column of look-back words per digit; one counting
// kernel reads the keys once for the digit totals of every pass), so that a
// pass is one launch; for larger sorts, whose look-back chains grow long,
// from a per-pass histogram of every tile (digit-major) and its exclusive scan.
// ---------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 8;
constexpr int kRsTile = kRsThreads * kRsRounds;
constexpr int kRsMaxPasses = 8;
constexpr int kRsCountBlocks = 4 * 148;
constexpr int64_t kRsLookbackTiles = 128;   // larger sorts take the histogram-and-scan passes

template <int RB>
__global__ void __launch_bounds__(kRsThreads) k_rs_counts(const uint64_t* keys, int64_t n, int lo_bit,
                                                          int passes, int* ghist) {
    constexpr int kB = 1 << RB;
    constexpr unsigned kMask = kB - 1u;
    __shared__ int h[kRsMaxPasses * kB];
    for (int d = threadIdx.x; d < passes * kB; d += kRsThreads) h[d] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kRsThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRsThreads) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p * kB + (int)((k >> (lo_bit + RB * p)) & kMask)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < passes * kB; d += kRsThreads)
        if (h[d]) atomicAdd(&ghist[d], h[d]);
}

// Per-tile digit counts of one pass, digit-major (hist[d * nblocks + b]).
template <int RB>
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* keys, int64_t n, int shift, int* hist,
                                                        int nblocks) {
    constexpr int kB = 1 << RB;
    constexpr unsigned kMask = kB - 1u;
    __shared__ int h[kB];
    for (int d = threadIdx.x; d < kB; d += kRsThreads) h[d] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kRsTile;
    for (int k = threadIdx.x; k < kRsTile; k += kRsThreads) {
        const int64_t i = t0 + k;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & kMask], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kB; d += kRsThreads) hist[d * nblocks + blockIdx.x] = h[d];
}

// One pass.  LB: ghist holds this pass's digit totals and look [0] the tile
// counter, then kB look-back words per tile (zeroed by the caller).  !LB:
// ghist holds the exclusive scan of the digit-major tile histogram, and the
// tile is the block.  wcnt holds each warp's digit counts, then (in place)
// each warp's first tile position per digit.
template <int RB, bool LB>
__global__ void __launch_bounds__(kRsThreads) k_rs_sweep(const uint64_t* kin, const uint32_t* vin, uint64_t* kout,
                                                         uint32_t* vout, int64_t n, int shift, const int* ghist,
                                                         unsigned long long* look) {
    constexpr int kB = 1 << RB;
    constexpr int kPer = kB / kRsThreads;     // digits per thread (1 or 2)
    constexpr unsigned kMask = kB - 1u;
    __shared__ int wcnt[kRsWarps][kB];
    __shared__ int gbase[kB];
    __shared__ int wsum[kRsWarps];
    __shared__ int wsum2[kRsWarps];
    __shared__ int s_tile;
    __shared__ uint64_t skey[kRsTile];
    __shared__ uint32_t sval[kRsTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (LB && threadIdx.x == 0) s_tile = (int)atomicAdd(look, 1ull);
    for (int i = threadIdx.x; i < kRsWarps * kB; i += kRsThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int tile = LB ? s_tile : (int)blockIdx.x;
    unsigned long long* lw = look + 1;
    const int64_t t0 = (int64_t)tile * kRsTile;
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
    if (!LB) {
        // tile-local start of each digit (thread j takes digits kPer j .. kPer j + kPer - 1,
        // an exclusive scan over the threads), and the tile's global start per digit
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
            gbase[d] = ghist[(int64_t)d * gridDim.x + tile] - ds;
            int run = ds;
            for (int w = 0; w < kRsWarps; ++w) {
                const int c = wcnt[w][d];
                wcnt[w][d] = run;
                run += c;
            }
            ds += tot[q];
        }
    } else {
        // thread j takes digits kPer j .. kPer j + kPer - 1: the tile's counts
        // (published at once), their tile-local starts and the digits' global
        // starts (block scans over the threads)
        int tot[kPer];
        int mine = 0, gmine = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int d = kPer * threadIdx.x + q;
            tot[q] = 0;
            for (int w = 0; w < kRsWarps; ++w) tot[q] += wcnt[w][d];
            mine += tot[q];
            gmine += ghist[d];
            lb_store(lw + (size_t)tile * kB + d, (tile == 0 ? kLbIncl : kLbAgg) | (unsigned long long)tot[q]);
        }
        int x = mine, gx = gmine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, x, o);
            const int gu = __shfl_up_sync(0xffffffffu, gx, o);
            if (lane >= o) {
                x += u;
                gx += gu;
            }
        }
        if (lane == 31) {
            wsum[warp] = x;
            wsum2[warp] = gx;
        }
        __syncthreads();
        int before = 0, gbefore = 0;
        for (int w = 0; w < warp; ++w) {
            before += wsum[w];
            gbefore += wsum2[w];
        }
        int ds = before + x - mine;       // tile-local start of the first digit
        int gs = gbefore + gx - gmine;    // global start of the first digit
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int d = kPer * threadIdx.x + q;
            int excl = 0;
            if (tile > 0) {
                excl = (int)lb_prefix(lw + d, tile, kB);
                lb_store(lw + (size_t)tile * kB + d, kLbIncl | (unsigned long long)(excl + tot[q]));
            }
            gbase[d] = gs + excl - ds;
            int run = ds;
            for (int w = 0; w < kRsWarps; ++w) {
                const int c = wcnt[w][d];
                wcnt[w][d] = run;
                run += c;
            }
            ds += tot[q];
            gs += ghist[d];
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
    const int64_t nb = ceil_div(n, kRsTile);
    uint64_t* k2 = dalloc<uint64_t>(n);
    uint32_t* v2 = vals ? dalloc<uint32_t>(n) : nullptr;
    // digit width: 8 bits, or 9 where that saves a pass (e.g. 18 bits: 2 passes, not 3)
    const int nbits = bits - lo_bit;
    const int passes8 = (nbits + 7) / 8, passes9 = (nbits + 8) / 9;
    const int rb = passes9 < passes8 ? 9 : 8;
    const int passes = rb == 9 ? passes9 : passes8;
    if (passes > kRsMaxPasses) fail(WNNC_EINVAL, "radix_sort_pairs: too many key bits");
    const int64_t kB = int64_t(1) << rb;
    uint64_t *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    unsigned long long* ws = nullptr;
    int* hist = nullptr;
    if (nb <= kRsLookbackTiles) {
        // one zeroed block: per pass the digit totals, then per pass the tile
        // counter and kB look-back words per tile
        const int64_t hist_words = (passes * kB + 1) / 2;          // ints, in 64-bit words
        const int64_t pass_words = 1 + nb * kB;
        ws = dalloc<unsigned long long>(hist_words + passes * pass_words);
        WNNC_CUDA(cudaMemsetAsync(ws, 0, sizeof(unsigned long long) * (hist_words + passes * pass_words), s));
        int* ghist = reinterpret_cast<int*>(ws);
        const int cgrid = (int)std::min<int64_t>(kRsCountBlocks, ceil_div(n, kRsThreads));
        if (rb == 9) k_rs_counts<9><<<cgrid, kRsThreads, 0, s>>>(keys, n, lo_bit, passes, ghist);
        else k_rs_counts<8><<<cgrid, kRsThreads, 0, s>>>(keys, n, lo_bit, passes, ghist);
        WNNC_LAUNCH_CHECK();
        for (int p = 0; p < passes; ++p) {
            const int shift = lo_bit + rb * p;
            unsigned long long* look = ws + hist_words + p * pass_words;
            if (rb == 9)
                k_rs_sweep<9, true><<<(unsigned)nb, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, ghist + p * kB, look);
            else
                k_rs_sweep<8, true><<<(unsigned)nb, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, ghist + p * kB, look);
            WNNC_LAUNCH_CHECK();
            std::swap(ka, kb);
            std::swap(va, vb);
        }
    } else {
        hist = dalloc<int>(kB * nb + 1);
        for (int p = 0; p < passes; ++p) {
            const int shift = lo_bit + rb * p;
            if (rb == 9) k_rs_hist<9><<<(unsigned)nb, kRsThreads, 0, s>>>(ka, n, shift, hist, (int)nb);
            else k_rs_hist<8><<<(unsigned)nb, kRsThreads, 0, s>>>(ka, n, shift, hist, (int)nb);
            WNNC_LAUNCH_CHECK();
            exclusive_scan_i32(hist, hist, kB * nb, s);
            if (rb == 9) k_rs_sweep<9, false><<<(unsigned)nb, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist, nullptr);
            else k_rs_sweep<8, false><<<(unsigned)nb, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist, nullptr);
            WNNC_LAUNCH_CHECK();
            std::swap(ka, kb);
            std::swap(va, vb);
        }
    }
    if (ka != keys) {
        WNNC_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (vals) WNNC_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    if (alloc_stream() != s) WNNC_CUDA(cudaStreamSynchronize(s));
    pool_free(k2);
    if (v2) pool_free(v2);
    if (ws) pool_free(ws);
    if (hist) pool_free(hist);
}

void selftest_wait_timeout(cudaStream_t s) {
    // two tiles of input, one block: it takes tile 1 (the counter starts at 1)
    // and waits for tile 0's look-back word, which nothing sets
    const int64_t n = 2 * (int64_t)kScanTile;
    int* in = dalloc<int>(n);
    int* out = dalloc<int>(n + 1);
    unsigned long long* look = dalloc<unsigned long long>(3);
    WNNC_CUDA(cudaMemsetAsync(in, 0, sizeof(int) * n, s));
    WNNC_CUDA(cudaMemsetAsync(look, 0, sizeof(unsigned long long) * 3, s));
    static const unsigned long long one = 1;
    WNNC_CUDA(cudaMemcpyAsync(look, &one, sizeof(one), cudaMemcpyHostToDevice, s));
    k_scan_chained<int><<<1, kScanThreads, 0, s>>>(in, out, n, look);
    WNNC_LAUNCH_CHECK();
    unsigned seen = 0;
    wait_timeouts_async(&seen, s);
    WNNC_CUDA(cudaStreamSynchronize(s));
    pool_free(in);
    pool_free(out);
    pool_free(look);
    check_wait_timeouts(seen, s);
}

void wait_timeouts_async(unsigned* host, cudaStream_t s) {
    WNNC_CUDA(cudaMemcpyFromSymbolAsync(host, g_wait_timeouts, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s));
}

void check_wait_timeouts(unsigned seen, cudaStream_t s) {
    if (!seen) return;
    const unsigned zero = 0;
    WNNC_CUDA(cudaMemcpyToSymbolAsync(g_wait_timeouts, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, s));
    WNNC_CUDA(cudaStreamSynchronize(s));
    fail(WNNC_ETIMEOUT, "a bounded wait of a single-pass scan or sort gave up");
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
