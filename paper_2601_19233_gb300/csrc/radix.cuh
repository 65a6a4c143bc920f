// Device-wide primitives used by the binning stage: an exclusive scan of
// 32-bit counts and a stable LSD radix sort of (uint32 key, uint32 value)
// pairs, 8 bits per pass.  Only render.cu includes this header.
//
// Radix pass = upsweep (per-block digit histograms, digit-major) -> exclusive
// scan of the histograms -> downsweep (each block re-reads its elements in
// input order and scatters them; ranks among equal digits come from
// __match_any_sync inside a warp and per-warp running counts, so the order of
// equal keys is preserved: the sort is stable).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace umgs {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;  // elements per block of the scan
// Radix sorts of up to kRsSmallMax elements (the count that sizes the grid)
// take 8 elements per thread, longer ones 16 (measured at 1080p: the 4 depth
// passes over 1.2M records and the region pass over 1.85M pairs gain from
// more blocks in flight; 4 per thread was slower again).
constexpr int64_t kRsSmallMax = (int64_t)1 << 24;
inline int radix_items(int64_t n_cap) { return n_cap <= kRsSmallMax ? 8 : 16; }
inline int64_t radix_blocks(int64_t n_cap) {
    const int64_t tile = (int64_t)kRsThreads * radix_items(n_cap);
    return n_cap > 0 ? (n_cap + tile - 1) / tile : 1;
}

// ---- exclusive scan of uint32 (sum must fit in uint32) ------------------------

__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t x, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t v = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += y;
        }
        if (lane < 32) s_warp[lane] = v;
    }
    __syncthreads();
    total = s_warp[(blockDim.x >> 5) - 1];
    const uint32_t r = inc - x + (w > 0 ? s_warp[w - 1] : 0u);
    __syncthreads();
    return r;
}

// phase 1: per-block sums of kRsTile elements (a block sum that does not
// fit in 32 bits sets *overflow)
static __global__ void __launch_bounds__(kRsThreads) scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                                         uint32_t* __restrict__ bsum,
                                                                         uint32_t* __restrict__ overflow) {
    pdl_enter();
    __shared__ uint32_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
        const int64_t i = base + k * kRsThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    if (s > 0xffffffffull) atomicOr(overflow, 1u);
    uint32_t tot;
    block_exclusive_scan_256((uint32_t)s, s_warp, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// phase 2: exclusive scan of the block sums (one block); writes the grand
// total, or 0xffffffff when the total does not fit in 32 bits (then the
// offsets are meaningless and the callers treat the pairs as overflowing)
static __global__ void __launch_bounds__(1024) scan_blocks_kernel(uint32_t* __restrict__ bsum, int nb,
                                                                 uint32_t* __restrict__ total,
                                                                 uint32_t* __restrict__ overflow) {
    pdl_enter();
    __shared__ uint32_t s_warp[32];
    __shared__ unsigned long long s_tot64[32];
    const int per = (nb + 1023) / 1024;
    const int b = min((int)threadIdx.x * per, nb), e = min(b + per, nb);
    uint32_t local = 0;
    unsigned long long local64 = 0ull;
    for (int k = b; k < e; ++k) { local += bsum[k]; local64 += bsum[k]; }
    {   // the 64-bit grand total, to detect a 32-bit wrap
        unsigned long long t64 = local64;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) t64 += __shfl_xor_sync(0xffffffffu, t64, d);
        if ((threadIdx.x & 31) == 0) s_tot64[threadIdx.x >> 5] = t64;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = local;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t v = s_warp[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += y;
        }
        s_warp[lane] = v;
    }
    __syncthreads();
    uint32_t run = inc - local + (w > 0 ? s_warp[w - 1] : 0u);
    for (int k = b; k < e; ++k) { const uint32_t c = bsum[k]; bsum[k] = run; run += c; }
    if (threadIdx.x == 1023) {
        unsigned long long t64 = 0ull;
        for (int k = 0; k < 32; ++k) t64 += s_tot64[k];
        *total = (*overflow != 0u || t64 > 0xfffffffeull) ? 0xffffffffu : s_warp[31];
    }
}

// phase 3: block-local exclusive scan plus the block's prefix
static __global__ void __launch_bounds__(kRsThreads) scan_apply_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                                        const uint32_t* __restrict__ bsum,
                                                                        uint32_t* __restrict__ out) {
    pdl_enter();
    __shared__ uint32_t s_warp[32];
    // each thread handles kRsItems consecutive elements
    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)threadIdx.x * kRsItems;
    uint32_t v[kRsItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan_256(s, s_warp, tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// ---- stable LSD radix sort, 8 bits per pass -----------------------------------

// Radix passes take ITEMS elements per thread (a block sorts 256 x ITEMS):
// 16 for long inputs, 8 for short ones (more blocks in flight).
//
// Optional key map (the depth sort): ~min and max of the keys other than
// 0xffffffff (the invalid records), spread over kRadixMapSlots slots
// (mm[2s] = ~min, mm[2s+1] = max of the keys that slot saw).  Keys are then sorted by
// k - min (0xffffffff by span = max - min + 1, after every valid key), which
// orders them as k does, and a pass whose digit lies above every mapped key
// (span >> shift == 0) is skipped: its upsweep and scan do nothing and its
// downsweep copies the elements through.  mm == nullptr: keys as they are.
struct RadixMap {
    uint32_t kmin, span;
    bool on;
    __device__ __forceinline__ uint32_t key(uint32_t k) const {
        return !on ? k : (k == 0xffffffffu ? span : k - kmin);
    }
    __device__ __forceinline__ bool skip(int shift) const { return on && (span >> shift) == 0u; }
};
constexpr int kRadixMapSlots = 32;
// (called by every thread; each warp reduces the slots, one per lane)
__device__ __forceinline__ RadixMap radix_map(const uint32_t* __restrict__ mm) {
    RadixMap m;
    m.on = mm != nullptr;
    m.kmin = 0u;
    m.span = 0u;
    if (m.on) {
        const int lane = threadIdx.x & 31;
        uint32_t a = mm[2 * lane], b = mm[2 * lane + 1];
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            a = max(a, __shfl_xor_sync(0xffffffffu, a, d));
            b = max(b, __shfl_xor_sync(0xffffffffu, b, d));
        }
        const uint32_t kmin = ~a, kmax = b;
        m.kmin = kmin;
        m.span = kmax >= kmin ? kmax - kmin + 1u : 0u;  // no valid key: every key maps to 0
    }
    return m;
}
template <int ITEMS>
static __global__ void __launch_bounds__(kRsThreads) radix_upsweep_kernel(const uint32_t* __restrict__ keys,
                                                                          const uint32_t* __restrict__ n_dev,
                                                                          int64_t n_cap, int shift, int nblocks,
                                                                          uint32_t* __restrict__ hist,
                                                                          const uint32_t* __restrict__ mm) {
    pdl_enter();
    __shared__ uint32_t cnt[256];
    const RadixMap map = radix_map(mm);
    if (map.skip(shift)) return;
    const int64_t n = min((int64_t)*n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * (kRsThreads * ITEMS);
    if (base >= n) return;  // a block past the live count (capacity-sized grids): its column is not scanned
    cnt[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int64_t i = base + k * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(map.key(keys[i]) >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Digit-major histogram [256][nblocks] -> per digit, exclusive prefix over
// the live blocks (those holding elements; in place) and the digit total.
// One CTA per digit.
static __global__ void __launch_bounds__(kRsThreads) radix_hist_scan_kernel(uint32_t* __restrict__ hist, int nblocks,
                                                                            const uint32_t* __restrict__ n_dev,
                                                                            int64_t n_cap, int tile,
                                                                            uint32_t* __restrict__ dtotal, int shift,
                                                                            const uint32_t* __restrict__ mm) {
    pdl_enter();
    __shared__ uint32_t s_warp[32];
    if (radix_map(mm).skip(shift)) return;
    uint32_t* h = hist + (int64_t)blockIdx.x * nblocks;
    const int64_t n = min((int64_t)*n_dev, n_cap);
    const int live = (int)min((int64_t)nblocks, (n + tile - 1) / tile);
    const int per = (live + kRsThreads - 1) / kRsThreads;
    const int b = min((int)threadIdx.x * per, live), e = min(b + per, live);
    uint32_t local = 0;
    for (int k = b; k < e; ++k) local += h[k];
    uint32_t tot;
    uint32_t run = block_exclusive_scan_256(local, s_warp, tot);
    for (int k = b; k < e; ++k) { const uint32_t c = h[k]; h[k] = run; run += c; }
    if (threadIdx.x == 0) dtotal[blockIdx.x] = tot;
}

// Each warp owns a contiguous chunk of ITEMS * 32 elements of the block and
// ranks it round by round (32 consecutive elements per round) against a
// per-warp digit counter; per-digit scans over the warps and over the digits
// give every element its position in the block's digit-sorted order.  The
// block's elements are staged in shared memory in that order and written out
// as contiguous runs per digit (coalesced).  Input order is preserved for
// equal digits.
template <int ITEMS>
static __global__ void __launch_bounds__(kRsThreads) radix_downsweep_kernel(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, const uint32_t* __restrict__ n_dev,
    int64_t n_cap, int shift, int nblocks, const uint32_t* __restrict__ hist, const uint32_t* __restrict__ dtotal,
    uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* __restrict__ mm) {
    pdl_enter();
    const int64_t n = min((int64_t)*n_dev, n_cap);
    const RadixMap map = radix_map(mm);
    constexpr int NW = kRsThreads / 32;
    __shared__ uint32_t wcnt[NW][256];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t bstart[256];   // block-local start of each digit
    __shared__ uint32_t gstart[256];   // global start of this block's run of each digit
    __shared__ uint2 stage[kRsThreads * ITEMS];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t bbase = (int64_t)blockIdx.x * (kRsThreads * ITEMS);
    if (bbase >= n) return;  // nothing of this block is live (uniform over the block)
    if (map.skip(shift)) {  // a constant digit: the pass copies the elements through
        for (int64_t i = bbase + t; i < min(n, bbase + (int64_t)kRsThreads * ITEMS); i += kRsThreads) {
            kout[i] = kin[i];
            vout[i] = vin[i];
        }
        return;
    }
    const int64_t base = bbase + (int64_t)w * (32 * ITEMS);
    const unsigned lt = (1u << lane) - 1u;
    uint32_t key[ITEMS], val[ITEMS], rank[ITEMS], dig[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int64_t i = base + k * 32 + lane;
        const bool valid = i < n;
        key[k] = valid ? kin[i] : 0u;
        val[k] = valid ? vin[i] : 0u;
        dig[k] = valid ? ((map.key(key[k]) >> shift) & 255u) : 256u;
    }
#pragma unroll
    for (int q = 0; q < NW; ++q) wcnt[q][t] = 0;
    // global digit bases: exclusive scan of the digit totals
    uint32_t dtot;
    const uint32_t dbase = block_exclusive_scan_256(dtotal[t], s_warp, dtot);
    gstart[t] = dbase + hist[(int64_t)t * nblocks + blockIdx.x];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const unsigned peers = __match_any_sync(0xffffffffu, dig[k]);
        const uint32_t lr = __popc(peers & lt);
        const uint32_t before = dig[k] < 256u ? wcnt[w][dig[k]] : 0u;
        __syncwarp();
        if (dig[k] < 256u && lr == 0) wcnt[w][dig[k]] = before + __popc(peers);
        __syncwarp();
        rank[k] = before + lr;
    }
    __syncthreads();
    uint32_t cnt_t = 0;
    {   // digit t: exclusive offsets over the warps (block-local)
#pragma unroll
        for (int q = 0; q < NW; ++q) { const uint32_t c = wcnt[q][t]; wcnt[q][t] = cnt_t; cnt_t += c; }
    }
    uint32_t btot;
    bstart[t] = block_exclusive_scan_256(cnt_t, s_warp, btot);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
        if (dig[k] < 256u) stage[bstart[dig[k]] + wcnt[w][dig[k]] + rank[k]] = make_uint2(key[k], val[k]);
    __syncthreads();
    for (int i = t; i < (int)btot; i += kRsThreads) {
        const uint2 e = stage[i];
        const uint32_t d = (map.key(e.x) >> shift) & 255u;
        const uint32_t pos = gstart[d] + (uint32_t)i - bstart[d];
        kout[pos] = e.x;
        vout[pos] = e.y;
    }
}

}  // namespace umgs
