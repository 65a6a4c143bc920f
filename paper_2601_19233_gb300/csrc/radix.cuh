// Device-wide primitives used by the binning stage: an exclusive scan of
// 32-bit counts and a stable LSD radix sort of (uint32 key, uint32 value)
// pairs, 8 bits per pass.  Only render.cu includes this header.
//
// Radix pass = upsweep (per-block digit histograms, digit-major) -> exclusive
// scan of the histograms -> downsweep (each block re-reads its elements in
// input order and scatters them; ranks among equal digits come from
// match_digit8 inside a warp and per-warp running counts, so the order of
// equal keys is preserved: the sort is stable).  The binning stage's own
// sorts use the single-sweep passes at the end of this file.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace umgs {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;  // elements per block of the scan
// Radix passes take 8 elements per thread at every size (measured on the
// 64-view 800^2 workload: 38M depth keys and the region pairs sorted with 8
// per thread instead of 16 took the render from 15.4 to 14.7 ms, the
// 16-element pass kernel holding 128 registers at two CTAs per SM; at 1080p
// the passes already used 8).  kRsSmallMax keeps the 16-element kernels
// selectable (above it) without a size in practice reaching it.
constexpr int64_t kRsSmallMax = (int64_t)1 << 62;
inline int radix_items(int64_t n_cap) { return n_cap <= kRsSmallMax ? 8 : 16; }
inline int64_t radix_blocks(int64_t n_cap) {
    const int64_t tile = (int64_t)kRsThreads * radix_items(n_cap);
    return n_cap > 0 ? (n_cap + tile - 1) / tile : 1;
}

// The lanes of the (converged) warp whose 8-bit digit d equals this lane's,
// among the lanes with `valid` set (0 for an invalid lane): eight ballots,
// one per digit bit.  Used instead of __match_any_sync, which measured far
// slower here (about 280 cycles per instruction in a histogram kernel).
__device__ __forceinline__ unsigned match_digit8(uint32_t d, bool valid) {
    unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
        const bool on = (d >> bit) & 1u;
        const unsigned b = __ballot_sync(0xffffffffu, on);
        peers &= on ? b : ~b;
    }
    return valid ? peers : 0u;
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
        const unsigned peers = match_digit8(dig[k], dig[k] < 256u);
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

// ---- single-sweep primitives (decoupled look-back) ----------------------------
//
// The binning stage's radix passes and scans run as one kernel each: a block
// publishes, per counter, a 64-bit word in a look-back array (bits 62-63 the
// flag: 0 nothing yet, 1 the block's own count, 2 the inclusive prefix up to
// and including the block; bits 0-61 the value) and finds its exclusive
// prefix by walking back over its predecessors' words until an inclusive one.
// A block takes its tile index from an atomic counter as it starts, so every
// block it waits for has started before it and is resident or finished, and
// every block publishes its own count before it waits: the waits end.  Each
// wait is still bounded (kLbSpinMax polls in all); one that runs out sets
// status bit kStatusLookbackTimeout, takes 0 and lets the kernel finish, and
// the render reports UMGS_ERR_TIMEOUT.
constexpr uint64_t kLbAgg = 1ull << 62, kLbInc = 2ull << 62, kLbVal = (1ull << 62) - 1;
constexpr int kLbSpinMax = 1 << 20;
constexpr uint32_t kStatusLookbackTimeout = 16;

__device__ __forceinline__ void lb_store(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t lb_load(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// One thread's look-back over counter c of blocks b-1, b-2, ... (`stride`
// counters per block): the sum of their counts.  Eight predecessors per step,
// loaded together, so that the walk back to the nearest inclusive word takes
// an eighth of the dependent loads.
__device__ __forceinline__ uint64_t lookback_thread(const uint64_t* __restrict__ lb, int64_t b, int stride, int c,
                                                    uint32_t* __restrict__ err) {
    constexpr int WIN = 8;
    uint64_t excl = 0;
    int spins = 0;
    for (int64_t hi = b - 1; hi >= 0; hi -= WIN) {
        uint64_t w[WIN];
#pragma unroll
        for (int k = 0; k < WIN; ++k) w[k] = hi - k >= 0 ? lb_load(lb + (hi - k) * stride + c) : kLbInc;
#pragma unroll
        for (int k = 0; k < WIN; ++k) {
            while ((w[k] >> 62) == 0) {
                if (++spins > kLbSpinMax) {
                    atomicOr(err, kStatusLookbackTimeout);
                    w[k] = kLbInc;
                    break;
                }
                if (spins > 32) __nanosleep(64);
                w[k] = lb_load(lb + (hi - k) * stride + c);
            }
        }
        bool done = false;
#pragma unroll
        for (int k = 0; k < WIN; ++k) {
            if (!done) {
                excl += w[k] & kLbVal;
                done = (w[k] >> 62) == 2;
            }
        }
        if (done) break;
    }
    return excl;
}

// A whole warp's look-back over one counter per block: 32 predecessors per
// step, summed up to the nearest inclusive word.  Every lane returns the sum.
__device__ __forceinline__ uint64_t lookback_warp(const uint64_t* __restrict__ lb, int64_t b,
                                                  uint32_t* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    uint64_t excl = 0;
    int spins = 0;
    for (int64_t hi = b - 1; hi >= 0; hi -= 32) {
        const int64_t p = hi - lane;
        uint64_t w;
        while (true) {  // (the loop is warp-uniform: spins is the same in every lane)
            w = p >= 0 ? lb_load(lb + p) : kLbInc;
            if (__all_sync(0xffffffffu, (w >> 62) != 0)) break;
            if (++spins > kLbSpinMax) {
                if (lane == 0) atomicOr(err, kStatusLookbackTimeout);
                w = kLbInc;
                break;
            }
            if (spins > 32) __nanosleep(64);
        }
        const unsigned inc = __ballot_sync(0xffffffffu, (w >> 62) == 2);
        const int first = inc ? __ffs(inc) - 1 : 31;
        uint64_t v = lane <= first ? (w & kLbVal) : 0ull;
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
        excl += v;
        if (inc) break;
    }
    return excl;
}

// Digits of the depth sort (8 bits per pass, LSD): passes 0 and 1 take the
// raw low 16 key bits, passes 2 and 3 the high part h = (k >> 16) - kmin16
// (kmin16 the high half of the smallest valid key; culled records, key
// 0xffffffff, take h = hspan, after every valid key).  h is a monotone map
// of k >> 16 over the valid keys, so (h, k & 0xffff) orders them as k does.
// Valid keys are the bits of positive depths (below 0x7f800000), so h fits
// 16 bits; pass 3 runs only when some h exceeds 255 (depths spanning more
// than 255 x 2^16 float steps): at 1080p the depths 1.6 to 4.4 need 3 passes.
// Passes 0 and 1 need no minimum, so their digit counts come from the key
// pass itself (prim_keys_kernel); pass 2's counts are the raw third byte's
// counts rotated by kmin16 (plus the culled records at hspan); pass 3's are
// counted by pass 2.
struct DepthDigits {
    uint32_t kmin16, hspan;
    __device__ __forceinline__ uint32_t h(uint32_t k) const { return k == 0xffffffffu ? hspan : (k >> 16) - kmin16; }
    __device__ __forceinline__ uint32_t digit(uint32_t k, int pass) const {
        return pass < 2 ? (k >> (8 * pass)) & 255u : pass == 2 ? h(k) & 255u : h(k) >> 8;
    }
    __device__ __forceinline__ bool skip(int pass) const { return pass == 3 && hspan <= 255u; }
    // passes that run: the sorted keys end in the second buffer when odd
    __device__ __forceinline__ int passes_run() const { return hspan <= 255u ? 3 : 4; }
};
// (called by every thread; from the ~min / max slots of radix_map)
__device__ __forceinline__ DepthDigits depth_digits(const uint32_t* __restrict__ mm) {
    const RadixMap m = radix_map(mm);  // kmin = smallest valid key, span = max - min + 1 (0: no valid key)
    DepthDigits d;
    d.kmin16 = m.kmin >> 16;
    d.hspan = m.span == 0u ? 0u : ((m.kmin + (m.span - 1u)) >> 16) - d.kmin16 + 1u;
    return d;
}

constexpr int kHistThreads = 1024;  // block size of the binning kernels that count digits


// Look-back words of one radix pass: per tile one 32-bit word per digit
// (bit 31 set once written, the tile's count below it), and per group of
// kLbGroup consecutive tiles one 64-bit word per digit (kLbAgg / kLbInc
// flags: the group's total, then its inclusive prefix over the groups).
constexpr int kLbGroup = 32;
struct PassLookback {
    uint32_t* tiles;   // [tiles][256]
    uint64_t* groups;  // [groups][256]
};
__host__ __device__ inline int64_t lookback_groups(int64_t tiles) { return (tiles + kLbGroup - 1) / kLbGroup; }
// bytes of one pass's look-back words for `tiles` tiles
inline int64_t lookback_bytes(int64_t tiles) {
    return tiles * 256 * (int64_t)sizeof(uint32_t) + lookback_groups(tiles) * 256 * (int64_t)sizeof(uint64_t);
}
inline PassLookback lookback_layout(void* base, int64_t tiles) {
    PassLookback l;
    l.tiles = static_cast<uint32_t*>(base);
    l.groups = reinterpret_cast<uint64_t*>(static_cast<char*>(base) + tiles * 256 * sizeof(uint32_t));
    return l;
}

__device__ __forceinline__ void lb_store32(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lb_load32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive prefix of digit c's counts over the tiles before tile b, in two
// levels: the tiles of b's own group before it (one word each, read eight at a
// time), then the groups before b's group (lookback_thread over the group
// words).  The last tile of a group publishes the group's total and, once its
// own look-back is done, the group's inclusive prefix, so that a walk back
// crosses groups, not tiles: with every tile of a pass resident at once, a
// chain of (tiles / 32) / 8 dependent loads instead of tiles / 8.
__device__ __forceinline__ uint64_t lookback_two_level(const PassLookback& lb, int64_t b, int c, uint32_t cnt,
                                                       uint32_t* __restrict__ err) {
    const int64_t g = b / kLbGroup, g0 = g * kLbGroup;
    uint32_t intra = 0;
    int spins = 0;
    for (int64_t j0 = g0; j0 < b; j0 += 8) {
        uint32_t w[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = j0 + k < b ? lb_load32(lb.tiles + (j0 + k) * 256 + c) : 0x80000000u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            while (!(w[k] >> 31)) {
                if (++spins > kLbSpinMax) {
                    atomicOr(err, kStatusLookbackTimeout);
                    w[k] = 0x80000000u;
                    break;
                }
                if (spins > 32) __nanosleep(64);
                w[k] = lb_load32(lb.tiles + (j0 + k) * 256 + c);
            }
            intra += w[k] & 0x7fffffffu;
        }
    }
    const bool last = (b % kLbGroup) == kLbGroup - 1;
    uint64_t* const gw = lb.groups + g * 256 + c;
    if (last) lb_store(gw, (g == 0 ? kLbInc : kLbAgg) | (uint64_t)(intra + cnt));
    const uint64_t gex = g > 0 ? lookback_thread(lb.groups, g, 256, c, err) : 0ull;
    if (last && g > 0) lb_store(gw, kLbInc | (gex + intra + cnt));
    return gex + intra;
}

// One pass of the single-sweep stable LSD radix sort on the 8-bit digit at
// `shift` (DEPTH: the depth sort's pass shift / 8, DepthDigits): ghist holds
// the pass's global digit counts (depth pass 2: the raw third-byte counts,
// rotated here; n_culled the culled records; pass 2 counts pass 3's digits
// into hist3 when pass 3 runs).  A block ranks its tile of elements like the downsweep above
// (warp-local ranks from match_digit8, per-warp digit counters, block
// digit offsets), publishes its 256 digit counts, stages its elements in
// shared memory in block-local digit order, looks back per digit (thread d
// for digit d, lookback_two_level) for the counts of the tiles before it, and
// scatters the staged elements to digit base + look-back prefix + block-local
// rank as contiguous runs per digit.  Tiles are taken in order of the atomic
// counter, so equal digits keep their input order: the sort is stable.
// lb_next (the next pass's look-back words, or null tiles) gets this block's
// words cleared.  A depth pass 3 that DepthDigits skips does nothing (every
// digit is 0: the elements stay where they are, and the reader takes them
// from there, DepthDigits::passes_run).
template <int ITEMS, bool DEPTH>
static __global__ void __launch_bounds__(kRsThreads, ITEMS == 8 ? 4 : 2) onesweep_pass_kernel(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, const uint32_t* __restrict__ n_dev,
    int64_t n_cap, int shift, const uint32_t* __restrict__ ghist, PassLookback lb, PassLookback lb_next,
    uint32_t* __restrict__ counter, uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
    const uint32_t* __restrict__ mm, const uint32_t* __restrict__ n_culled, uint32_t* __restrict__ hist3,
    uint32_t* __restrict__ err) {
    pdl_enter();
    constexpr int NW = kRsThreads / 32;
    constexpr int TILE = kRsThreads * ITEMS;
    __shared__ uint32_t wcnt[NW][256];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t bstart[256];   // block-local start of each digit
    __shared__ uint32_t gstart[256];   // global start of this block's run of each digit
    __shared__ uint2 stage[TILE];
    __shared__ uint32_t s_id;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) s_id = atomicAdd(counter, 1u);
    __syncthreads();
    const int64_t b = s_id;
    const int pass = shift / 8;  // (depth sort)
    const DepthDigits dd = DEPTH ? depth_digits(mm) : DepthDigits{0u, 0u};
    const int64_t n = min((int64_t)*n_dev, n_cap);
    const int64_t bbase = b * TILE;
    if (bbase >= n) return;  // nothing of this tile is live (uniform over the block)
    if (lb_next.tiles) {
        lb_next.tiles[b * 256 + t] = 0u;
        if (b % kLbGroup == 0) lb_next.groups[(b / kLbGroup) * 256 + t] = 0ull;
    }
    if (DEPTH && dd.skip(pass)) return;
    const auto digit = [&](uint32_t k) { return DEPTH ? dd.digit(k, pass) : (k >> shift) & 255u; };
    const int64_t base = bbase + (int64_t)w * (32 * ITEMS);
    const unsigned lt = (1u << lane) - 1u;
    uint32_t key[ITEMS], val[ITEMS], rank[ITEMS], dig[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int64_t i = base + k * 32 + lane;
        const bool valid = i < n;
        key[k] = valid ? kin[i] : 0u;
        val[k] = valid ? vin[i] : 0u;
        dig[k] = valid ? digit(key[k]) : 256u;
    }
#pragma unroll
    for (int q = 0; q < NW; ++q) wcnt[q][t] = 0;
    __syncthreads();
    if (DEPTH && pass == 2 && !dd.skip(3)) {  // the digit counts of pass 3 (wcnt[0] as a scratch histogram)
#pragma unroll
        for (int k = 0; k < ITEMS; ++k)
            if (dig[k] < 256u) atomicAdd(&wcnt[0][dd.h(key[k]) >> 8], 1u);
        __syncthreads();
        if (wcnt[0][t]) atomicAdd(&hist3[t], wcnt[0][t]);
        __syncthreads();
        wcnt[0][t] = 0;
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const unsigned peers = match_digit8(dig[k], dig[k] < 256u);
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
    lb_store32(lb.tiles + b * 256 + t, 0x80000000u | cnt_t);
    uint32_t dtot, btot;
    // pass 2 of the depth sort: the raw third-byte counts of the valid keys,
    // rotated to h's low byte, and the culled records at hspan
    const uint32_t gh = (DEPTH && pass == 2)
                            ? ghist[(t + dd.kmin16) & 255u] + ((uint32_t)t == (dd.hspan & 255u) ? *n_culled : 0u)
                            : ghist[t];
    const uint32_t dbase = block_exclusive_scan_256(gh, s_warp, dtot);
    bstart[t] = block_exclusive_scan_256(cnt_t, s_warp, btot);
    __syncthreads();
    // (the block-local order needs no look-back: stage first)
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
        if (dig[k] < 256u) stage[bstart[dig[k]] + wcnt[w][dig[k]] + rank[k]] = make_uint2(key[k], val[k]);
    const uint64_t excl = lookback_two_level(lb, b, t, cnt_t, err);
    gstart[t] = dbase + (uint32_t)excl;
    __syncthreads();
    for (int i = t; i < (int)btot; i += kRsThreads) {
        const uint2 e = stage[i];
        const uint32_t d = digit(e.x);
        const uint32_t pos = gstart[d] + (uint32_t)i - bstart[d];
        kout[pos] = e.x;
        vout[pos] = e.y;
    }
}

// Exclusive scan of n values of an input functor into int64 out[0..n) with
// out[n] = the total (also *total32, 0xffffffff when it does not fit), one
// kernel: 256 threads x ITEMS consecutive values per block, block scan, warp
// look-back over the blocks' totals (lb: one word per block).  ITEMS = 1 for
// a functor that does work of its own per value (all values in parallel).
template <class In, int ITEMS>
static __global__ void __launch_bounds__(kRsThreads) scan_lookback_kernel(In in, int64_t n,
                                                                          int64_t* __restrict__ out,
                                                                          uint32_t* __restrict__ total32,
                                                                          uint64_t* __restrict__ lb,
                                                                          uint32_t* __restrict__ counter,
                                                                          uint32_t* __restrict__ err) {
    pdl_enter();
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_id;
    __shared__ unsigned long long s_excl;
    const int t = threadIdx.x;
    if (t == 0) s_id = atomicAdd(counter, 1u);
    __syncthreads();
    const int64_t b = s_id;
    const int64_t base = b * (kRsThreads * ITEMS) + (int64_t)t * ITEMS;
    uint32_t v[ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        v[k] = base + k < n ? in(base + k) : 0u;
        s += v[k];
    }
    uint32_t btot;
    uint32_t run = block_exclusive_scan_256(s, s_warp, btot);
    if (t < 32) {
        if (t == 0) lb_store(lb + b, (b == 0 ? kLbInc : kLbAgg) | btot);
        const uint64_t excl = lookback_warp(lb, b, err);
        if (t == 0) {
            if (b > 0) lb_store(lb + b, kLbInc | (excl + btot));
            s_excl = excl;
        }
    }
    __syncthreads();
    uint64_t o = s_excl + run;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        if (base + k < n) out[base + k] = (int64_t)o;
        o += v[k];
        if (base + k == n - 1) {
            out[n] = (int64_t)o;
            *total32 = o >= 0xffffffffull ? 0xffffffffu : (uint32_t)o;
        }
    }
}

}  // namespace umgs
