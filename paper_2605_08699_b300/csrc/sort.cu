// K2 device prefix scan and K4 LSD radix sort (8-bit digits, stable).
//
// The prefix scan is reduce-then-scan: every kernel reads only data written
// by earlier kernels in stream order, so none of its CTAs waits on another.
//
// The radix sort has two paths.
//  - One-sweep (every input below 2^30 keys, i.e. every sort of the render
//    path): one read of the keys builds the digit histograms of all passes,
//    then each pass is a single scatter kernel.  A CTA claims the next chunk,
//    ranks its keys with one warp ballot per digit bit, publishes its digit
//    counts and finds the earlier chunks' counts by decoupled look-back.  That
//    look-back SPINS on other CTAs' status words.  Every spin is bounded: a CTA
//    only waits on chunks claimed by CTAs that started before it (so the wait
//    ends in any correct run), and after kSpinLimit polls it sets a timeout
//    flag in device memory and finishes its pass with its writes kept inside
//    the output; the host turns the flag into TIGAS_ERR_TIMEOUT.
//  - Reduce-then-scan (inputs of 2^30 keys or more, whose counts do not fit
//    the look-back's 30-bit status words): per pass a histogram kernel
//    (4096-key tiles -> table[digit][tile]), an exclusive scan of that table,
//    and a scatter that ranks each tile stably with warp match.any and
//    per-warp digit counters; no CTA waits on another.
#include <vector>

#include "kernels.cuh"

namespace tigas {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTileN = kThreads * kItems;   // 4096 elements per CTA
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kFull = 0xFFFFFFFFu;

__device__ inline uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread across a 256-thread CTA.
// Returns the exclusive prefix; *total receives the CTA sum.
__device__ inline uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_sums /*[kWarps + 1]*/, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kWarps ? warp_sums[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int d = 1; d < kWarps; d <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < kWarps) warp_sums[lane] = wi - w;     // exclusive warp offsets
        if (lane == kWarps - 1) warp_sums[kWarps] = wi;  // CTA total
    }
    __syncthreads();
    uint32_t res = warp_sums[warp] + inc - x;
    if (total) *total = warp_sums[kWarps];
    __syncthreads();
    return res;
}

struct GatherLoader {
    const uint32_t* in;
    const uint32_t* order;
    __device__ inline uint32_t operator()(uint64_t k) const { return in[order ? order[k] : k]; }
};

// --------------------------------------------------------------- scan

__global__ void __launch_bounds__(kThreads)
k_scan_reduce(GatherLoader ld, uint64_t n, uint32_t* __restrict__ block_sums, unsigned long long* total64) {
    __shared__ uint32_t ws[kWarps + 1];
    uint64_t base = (uint64_t)blockIdx.x * kTileN;
    uint32_t s = 0;
#pragma unroll 4
    for (int k = 0; k < kItems; ++k) {
        uint64_t idx = base + (uint64_t)k * kThreads + threadIdx.x;
        if (idx < n) s += ld(idx);
    }
    uint32_t tot;
    block_exclusive_scan(s, ws, &tot);
    if (threadIdx.x == 0) {
        block_sums[blockIdx.x] = tot;
        if (total64) atomicAdd(total64, (unsigned long long)tot);
    }
}

__device__ inline uint32_t pad_idx(uint32_t i) { return i + (i >> 5); }

__global__ void __launch_bounds__(kThreads)
k_scan_down(GatherLoader ld, uint64_t n, const uint32_t* __restrict__ block_offsets, uint32_t* __restrict__ out,
            unsigned long long* total64_single) {
    __shared__ uint32_t buf[kTileN + kTileN / 32];
    __shared__ uint32_t ws[kWarps + 1];
    const uint64_t base = (uint64_t)blockIdx.x * kTileN;
#pragma unroll 4
    for (int k = 0; k < kItems; ++k) {
        uint32_t li = k * kThreads + threadIdx.x;
        uint64_t idx = base + li;
        buf[pad_idx(li)] = idx < n ? ld(idx) : 0u;
    }
    __syncthreads();
    uint32_t v[kItems];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        v[j] = buf[pad_idx(threadIdx.x * kItems + j)];
        s += v[j];
    }
    uint32_t tot;
    uint32_t pre = block_exclusive_scan(s, ws, &tot);
    uint32_t off = (block_offsets ? block_offsets[blockIdx.x] : 0u) + pre;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        buf[pad_idx(threadIdx.x * kItems + j)] = off;
        off += v[j];
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kItems; ++k) {
        uint32_t li = k * kThreads + threadIdx.x;
        uint64_t idx = base + li;
        if (idx < n) out[idx] = buf[pad_idx(li)];
    }
    if (total64_single && threadIdx.x == 0) *total64_single = tot;
}

uint64_t scan_blocks(uint64_t n) { return (n + kTileN - 1) / kTileN; }

}  // namespace

size_t scan_tmp_words(uint64_t n) {
    uint64_t b = scan_blocks(n);
    if (b <= 1) return 0;
    return 2 * b + scan_tmp_words(b);
}

// tmp layout: [block sums b][block offsets b][tmp of the recursive scan]
Status launch_scan_u32(const uint32_t* in, const uint32_t* order, uint32_t* out, uint64_t n, uint64_t* total64,
                       uint32_t* tmp, cudaStream_t st, bool total_zeroed) {
    if (n == 0) {
        if (total64) TIGAS_CUDA_TRY(cudaMemsetAsync(total64, 0, sizeof(uint64_t), st));
        return {};
    }
    uint64_t b = scan_blocks(n);
    GatherLoader ld{in, order};
    if (b == 1) {
        k_scan_down<<<1, kThreads, 0, st>>>(ld, n, nullptr, out, (unsigned long long*)total64);
        TIGAS_LAUNCHED();
        return {};
    }
    if (b > 0x7FFFFFFFull) return {TIGAS_ERR_INVALID, "scan too large"};
    uint32_t* sums = tmp;
    uint32_t* offs = tmp + b;
    if (total64 && !total_zeroed) TIGAS_CUDA_TRY(cudaMemsetAsync(total64, 0, sizeof(uint64_t), st));
    k_scan_reduce<<<(unsigned)b, kThreads, 0, st>>>(ld, n, sums, (unsigned long long*)total64);
    TIGAS_LAUNCHED();
    TIGAS_TRY(launch_scan_u32(sums, nullptr, offs, b, nullptr, tmp + 2 * b, st));
    k_scan_down<<<(unsigned)b, kThreads, 0, st>>>(ld, n, offs, out, nullptr);
    TIGAS_LAUNCHED();
    return {};
}

// ------------------------------------------------------------ radix sort

namespace {

__device__ inline uint32_t count_of(uint64_t n_cap, const uint64_t* d_n) {
    uint64_t n = d_n ? *d_n : n_cap;
    return (uint32_t)(n < n_cap ? n : n_cap);
}

template <typename K>
__global__ void __launch_bounds__(kThreads)
k_radix_hist(const K* __restrict__ keys, uint64_t n_cap, const uint64_t* d_n, int shift, uint32_t mask,
             uint32_t num_tiles, uint32_t* __restrict__ table) {
    __shared__ uint32_t hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t n = count_of(n_cap, d_n);
    const uint64_t base = (uint64_t)blockIdx.x * kTileN;
    const int lane = threadIdx.x & 31;
    if (base < n) {
#pragma unroll 4
        for (int k = 0; k < kItems; ++k) {
            uint64_t idx = base + (uint64_t)k * kThreads + threadIdx.x;
            bool in = idx < n;
            uint32_t m = __ballot_sync(kFull, in);
            if (in) {
                uint32_t d = (uint32_t)(keys[idx] >> shift) & mask;
                uint32_t peers = __match_any_sync(m, d);
                if (lane == __ffs(peers) - 1) atomicAdd(&hist[d], (uint32_t)__popc(peers));
            }
        }
    }
    __syncthreads();
    table[(size_t)threadIdx.x * num_tiles + blockIdx.x] = hist[threadIdx.x];
}

template <typename K>
struct ScatterSmem {
    K keys[kTileN];
    uint32_t vals[kTileN];
    uint32_t whist[kWarps][256];
    uint32_t dstart[256];
    uint32_t gbase[256];
    uint32_t ws[kWarps + 1];
};

template <typename K>
__global__ void __launch_bounds__(kThreads)
k_radix_scatter(const K* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, K* __restrict__ keys_out,
                uint32_t* __restrict__ vals_out, uint64_t n_cap, const uint64_t* d_n, int shift, uint32_t mask,
                uint32_t num_tiles, const uint32_t* __restrict__ table) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<K>& sm = *reinterpret_cast<ScatterSmem<K>*>(smem_raw);
    const uint32_t n = count_of(n_cap, d_n);
    const uint64_t base = (uint64_t)blockIdx.x * kTileN;
    if (base >= n) return;
    const uint32_t valid = (n - base) < (uint64_t)kTileN ? (uint32_t)(n - base) : (uint32_t)kTileN;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (int k = threadIdx.x; k < kWarps * 256; k += kThreads) (&sm.whist[0][0])[k] = 0;

    // load: warp w owns tile-local elements [w*512, (w+1)*512), 32 per round
    K key[kItems];
    uint32_t val[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        uint32_t li = warp * (kItems * 32) + r * 32 + lane;
        if (li < valid) {
            key[r] = keys_in[base + li];
            val[r] = vals_in ? vals_in[base + li] : (uint32_t)(base + li);
        } else {
            key[r] = ~K(0);          // padding sorts after every valid key of this tile
            val[r] = 0;
        }
    }
    __syncthreads();

    // stable warp-local ranks: per-warp digit counters, one round at a time
    uint32_t dr[kItems];   // digit << 16 | warp-local rank
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        uint32_t d = (uint32_t)(key[r] >> shift) & mask;
        uint32_t peers = __match_any_sync(kFull, d);
        uint32_t before = sm.whist[warp][d];
        uint32_t rank = before + __popc(peers & lt);
        __syncwarp();
        if (lane == __ffs(peers) - 1) sm.whist[warp][d] = before + __popc(peers);
        __syncwarp();
        dr[r] = (d << 16) | rank;
    }
    __syncthreads();

    // per digit: exclusive prefix over warps, CTA total, and start in the tile
    {
        const uint32_t d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            uint32_t c = sm.whist[w][d];
            sm.whist[w][d] = run;
            run += c;
        }
        uint32_t start = block_exclusive_scan(run, sm.ws, nullptr);
        sm.dstart[d] = start;
        sm.gbase[d] = d <= mask ? table[(size_t)d * num_tiles + blockIdx.x] : 0u;
    }
    __syncthreads();

    // reorder through shared memory
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        uint32_t d = dr[r] >> 16;
        uint32_t pos = sm.dstart[d] + sm.whist[warp][d] + (dr[r] & 0xFFFFu);
        sm.keys[pos] = key[r];
        sm.vals[pos] = val[r];
    }
    __syncthreads();

    // write runs of equal digits to their global offsets
#pragma unroll 4
    for (int k = 0; k < kItems; ++k) {
        uint32_t j = k * kThreads + threadIdx.x;
        if (j < valid) {
            K kk = sm.keys[j];
            uint32_t d = (uint32_t)(kk >> shift) & mask;
            uint32_t g = sm.gbase[d] + (j - sm.dstart[d]);
            keys_out[g] = kk;
            vals_out[g] = sm.vals[j];
        }
    }
}

uint32_t sort_tiles(uint64_t n_cap) { return (uint32_t)((n_cap + kTileN - 1) / kTileN); }

// Function attributes are per device: the set-up below runs once per device
// ordinal under kMaxDevices (*slot), and on every call for a higher one (-1).
Status current_device_slot(int* slot) {
    int dev = 0;
    TIGAS_CUDA_TRY(cudaGetDevice(&dev));
    *slot = dev >= 0 && dev < kMaxDevices ? dev : -1;
    return {};
}

template <typename K>
Status ensure_scatter_smem() {
    static std::atomic<bool> done[kMaxDevices];
    int slot = -1;
    TIGAS_TRY(current_device_slot(&slot));
    if (slot >= 0 && done[slot].load()) return {};
    TIGAS_CUDA_TRY(cudaFuncSetAttribute(k_radix_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(ScatterSmem<K>)));
    if (slot >= 0) done[slot].store(true);
    return {};
}

size_t rts_tmp_words(uint64_t n_cap) {
    uint64_t tiles = sort_tiles(n_cap);
    if (tiles == 0) tiles = 1;
    uint64_t table = 256 * tiles;
    return 2 * table + scan_tmp_words(table);
}

// Reduce-then-scan passes: used for inputs of 2^30 elements or more (the
// one-sweep status words hold 30-bit counts).
template <typename K>
Status radix_sort_rts(const K* keys_in, const uint32_t* values_in, K* keys_alt, uint32_t* values_alt, K* keys_out,
                      uint32_t* values_out, uint64_t n_cap, const uint64_t* d_n, int begin_bit, int end_bit,
                      uint32_t* tmp, cudaStream_t st) {
    const int passes = (end_bit - begin_bit + 7) / 8;
    TIGAS_TRY(ensure_scatter_smem<K>());
    const size_t smem = sizeof(ScatterSmem<K>);
    const uint32_t tiles = sort_tiles(n_cap);
    uint32_t* table = tmp;
    uint32_t* scanned = tmp + (size_t)256 * tiles;
    uint32_t* scan_tmp = scanned + (size_t)256 * tiles;
    const K* src_k = keys_in;
    const uint32_t* src_v = values_in;
    for (int p = 0; p < passes; ++p) {
        int shift = begin_bit + 8 * p;
        int nb = min(8, end_bit - shift);
        uint32_t mask = (1u << nb) - 1u;
        bool to_out = ((passes - 1 - p) % 2) == 0;
        K* dk = to_out ? keys_out : keys_alt;
        uint32_t* dv = to_out ? values_out : values_alt;
        k_radix_hist<K><<<tiles, kThreads, 0, st>>>(src_k, n_cap, d_n, shift, mask, tiles, table);
        TIGAS_LAUNCHED();
        TIGAS_TRY(launch_scan_u32(table, nullptr, scanned, (uint64_t)256 * tiles, nullptr, scan_tmp, st));
        k_radix_scatter<K><<<tiles, kThreads, smem, st>>>(src_k, src_v, dk, dv, n_cap, d_n, shift, mask, tiles,
                                                          scanned);
        TIGAS_LAUNCHED();
        src_k = dk;
        src_v = dv;
    }
    return {};
}

}  // namespace

// ------------------------------------------------------ one-sweep passes
//
// One read of the keys builds the global digit histogram of every pass.  Each
// pass is then a single scatter kernel: a CTA claims the next chunk of keys
// (chunk ids follow the order CTAs start in), ranks its keys stably, publishes
// its per-digit counts, and finds the count of each digit in all earlier
// chunks by decoupled look-back over their published counts.  A CTA only waits
// on chunks claimed by CTAs that started before it, which publish before they
// wait themselves, so the waits always end; each wait is still bounded: after
// kSpinLimit polls the CTA records a timeout flag and goes on (its writes stay
// inside the output by the bounds check, the host reports the error).  The
// look-back reads a window of predecessors per round (4 in the depth sort, 2
// in the pair sorts: measured ahead of 8 and 16, whose extra loads mostly find
// counts the walk no longer needs), so a CTA of the first wave, whose
// predecessors have mostly published only their own counts, needs a fraction
// of the dependent round trips of a one-by-one walk.

namespace {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 2u << 30;
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 22;


// Tile shape of a scatter pass: T threads x I keys.  With an 8-byte payload a
// CTA takes half the keys so that keys, values and payloads still fit two CTAs
// per SM.
// Payload modes of the one-sweep passes: kPayNone, kPayWithValues (an 8-byte
// payload and the 4-byte values), kPayOnly (the payload identifies each key:
// no value stream, and no value staging in shared memory).
constexpr int kPayNone = 0, kPayWithValues = 1, kPayOnly = 2;
template <typename K, int PAY>
struct OsCfg;
#ifndef TIGAS_OS_THREADS
#define TIGAS_OS_THREADS 384
#endif
#ifndef TIGAS_OS_ITEMS
#define TIGAS_OS_ITEMS 12
#endif
#ifndef TIGAS_OS_PAY_THREADS
#define TIGAS_OS_PAY_THREADS 384
#endif
#ifndef TIGAS_OS_PAY_ITEMS
#define TIGAS_OS_PAY_ITEMS 12
#endif
#ifndef TIGAS_OS_PAY_BLOCKS
#define TIGAS_OS_PAY_BLOCKS 3
#endif
// 64-bit keys (the last slice's (tile, depth) pairs): a tile of 512 x 8 keys,
// 2 CTAs per SM (pair sorts 0.716 -> 0.712 ms per 8-view launch set against
// 256 x 16; 256 x 16 at 3 CTAs per SM: 0.718; a tile holds at least 4096 keys)
#ifndef TIGAS_OS64_THREADS
#define TIGAS_OS64_THREADS 512
#endif
#ifndef TIGAS_OS64_ITEMS
#define TIGAS_OS64_ITEMS 8
#endif
#ifndef TIGAS_OS64_BLOCKS
#define TIGAS_OS64_BLOCKS 2
#endif
#ifndef TIGAS_OS_BLOCKS
#define TIGAS_OS_BLOCKS 3   // CTAs per SM of the keys-and-values tile (0: (2 x 512) / threads)
#endif
template <int PAY>
struct OsCfg<uint32_t, PAY> {
    // Keys and values: 3 CTAs of 384 x 12 per SM (measured ahead of 512 x 16 x 2 and
    // 384 x 16 x 3 on the pair sorts).  Keys, values and payload: 2 CTAs of 512 x 8.
    // Payload only: without staged values a 384 x 12 tile fits 3 CTAs per SM (measured
    // fastest of 256 x 16 x {2, 3}, 384 x 12 x 3 and 512 x 8 x 2 on the 24M-entry depth sort).
    static constexpr int kT = PAY == kPayOnly ? TIGAS_OS_PAY_THREADS : PAY ? 512 : TIGAS_OS_THREADS;
    static constexpr int kI = PAY == kPayOnly ? TIGAS_OS_PAY_ITEMS : PAY ? 8 : TIGAS_OS_ITEMS;
    static constexpr int kMinBlocks = PAY == kPayOnly ? TIGAS_OS_PAY_BLOCKS
                                      : (TIGAS_OS_BLOCKS > 0 && !PAY) ? TIGAS_OS_BLOCKS : (2 * 512) / kT;
};
template <int PAY>
struct OsCfg<uint64_t, PAY> {
    static_assert(!PAY, "payloads are carried by 32-bit key sorts only");
    static constexpr int kT = TIGAS_OS64_THREADS, kI = TIGAS_OS64_ITEMS, kMinBlocks = TIGAS_OS64_BLOCKS;
};

// Where one pass reads and writes (device memory, written by k_os_bases once
// every pass's digit histogram is known).  A pass whose digit is the same for
// all keys is an identity permutation and is skipped; the passes that run
// ping-pong so that the last one writes the output buffers.
struct OsRoute {
    const void* src_k;
    const uint32_t* src_v;   // null: the value is the key's input position
    const uint2* src_p;      // null: no payload
    void* dst_k;
    uint32_t* dst_v;
    uint2* dst_p;
    // the first pass of a partial sort: where the far keys (digit 255) go, the
    // output buffers, which the later passes over the near keys do not reach
    void* far_k;             // null: no partial sort
    uint32_t* far_v;
    uint2* far_p;
    uint32_t active;
    int32_t next;            // deferred histograms: the next pass that runs (its digits counted here), or -1
};
constexpr int kRouteWords = (int)(sizeof(OsRoute) / 4);

struct OsBuffers {
    const void* in_k;
    const uint32_t* in_v;
    const uint2* in_p;
    void* alt_k;
    uint32_t* alt_v;
    uint2* alt_p;
    void* out_k;
    uint32_t* out_v;
    uint2* out_p;
};

__device__ inline uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ inline void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The value whose digits are sorted.  With a key range [kmin, kmax] (32-bit
// keys only): k - kmin, and 0xFFFFFFFF (the "culled" key) -> kmax - kmin + 1,
// an order-preserving map onto [0, kmax - kmin + 1], so the high digits of
// keys spanning less than 2^24 are all zero and their pass is skipped.
// With a split threshold thr (range[3] set): m = k - kmin below thr -> (q << 8)
// | r for m = 255 q + r (the same order; the low byte never reaches 255), and
// m >= thr or 0xFFFFFFFF -> 0xFFFFFFFF, the first pass's digit 255.
struct KeyMap {
    uint32_t kmin = 0, span = 0, thr = 0;
    bool on = false, split = false;
    __device__ inline void load(const uint32_t* range) {
        on = range != nullptr;
        if (on) {
            kmin = range[0];
            span = range[1] - kmin + 1u;
            split = range[3] != 0u;
            thr = range[2];
        }
    }
    __device__ static inline uint32_t base255(uint32_t m) {
        const uint32_t q = m / 255u;
        return (q << 8) | (m - q * 255u);
    }
    __device__ inline uint32_t operator()(uint32_t k) const {
        if (!on) return k;
        if (!split) return k == 0xFFFFFFFFu ? span : k - kmin;
        const uint32_t m = k - kmin;
        return k == 0xFFFFFFFFu || m >= thr ? 0xFFFFFFFFu : base255(m);
    }
    __device__ inline uint64_t operator()(uint64_t k) const { return k; }
    // the largest mapped key other than a split's far keys
    __device__ inline uint32_t top() const { return !split ? span : thr == 0u ? 0u : base255(thr - 1u); }
};

// Lanes of the warp whose digit equals this lane's: the AND over the digit's
// bits of the ballot of lanes agreeing on that bit (warp multisplit).  Always
// all 8 bits, with no test of the pass's digit width: a narrower digit has
// zero high bits, whose ballots leave the mask unchanged (measured: depth sort
// 0.849 -> 0.739 ms, pair sorts 0.638 -> 0.615 ms against a width test per
// bit).  Each bit's agreement is one XNOR of the ballot with the lane's bit
// spread to a mask (0.730 -> 0.701 and 0.612 -> 0.589 ms against a select of
// the ballot or its complement).
__device__ inline uint32_t digit_peers(uint32_t d) {
    uint32_t peers = kFull;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint32_t m = 0u - ((d >> b) & 1u);   // all ones when the bit is set
        const uint32_t bal = __ballot_sync(kFull, m != 0u);
        peers &= ~(bal ^ m);   // lanes that agree on the bit
    }
    return peers;
}

// Exclusive scan of one value per thread over a CTA of T threads.
template <int T>
__device__ inline uint32_t cta_exclusive_scan(uint32_t x, uint32_t* ws /*[T/32 + 1]*/) {
    constexpr int W = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < W ? ws[lane] : 0u;
        uint32_t iv = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, iv, d);
            if (lane >= d) iv += y;
        }
        if (lane < W) ws[lane] = iv - v;
    }
    __syncthreads();
    const uint32_t r = ws[warp] + inc - x;
    __syncthreads();
    return r;
}

// Global digit histograms of every pass in one read (run-length aggregated
// shared-memory counts, so keys with few distinct digits do not serialise;
// measured ahead of a warp-uniform-digit fast path with one atomic per warp).
// VEC: 32-bit keys 16-byte aligned, read as KB 16-byte vectors of 4
// consecutive keys per thread per step (2 measured ahead of 1 and 4: depth
// sort 0.693 -> 0.681 ms, pair sorts 0.558 -> 0.546 ms against scalar loads);
// consecutive keys also lengthen the runs of equal high digits.  Otherwise KB
// scalar keys per thread per step, all loads issued before any count: 8 for
// key/value sorts, 4 for mapped sorts (measured on scalar loads).
template <typename K, int KB, bool VEC, bool DIRECT>
__global__ void __launch_bounds__(512, 2)
k_os_hist(const K* __restrict__ keys, uint64_t n_cap, const uint64_t* d_n, int begin_bit, int end_bit,
          uint32_t* __restrict__ ghist, const uint32_t* __restrict__ range, uint4* __restrict__ status,
          uint64_t chunks, uint32_t chunk_keys, int count_passes, unsigned long long* __restrict__ bits_or) {
    constexpr int kP = (int)sizeof(K);   // most passes this key width can need
    __shared__ uint32_t h[kP][256];
    __shared__ unsigned long long s_or[2];
    const int passes = (end_bit - begin_bit + 7) / 8;
    const uint32_t n = count_of(n_cap, d_n);
    const uint64_t used = ((uint64_t)n + chunk_keys - 1) / chunk_keys;
    const uint64_t per_pass = used * 64, total = per_pass * (uint64_t)passes;
    // a grid sized for the capacity: a CTA with neither keys nor table entries
    // to clear leaves at once (its histogram would be empty)
    {
        const uint64_t first = (uint64_t)blockIdx.x * blockDim.x;
        if (first * (VEC ? 4u * KB : (uint64_t)KB) >= n && (status == nullptr || first >= total)) return;
    }
    // clear the scatter passes' look-back tables (no pass has started yet): per
    // pass, the entries of the chunks that hold keys (256 words = 64 uint4 each)
    if (status != nullptr) {
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
             i += (uint64_t)gridDim.x * blockDim.x) {
            const uint64_t p = i / per_pass;
            status[p * chunks * 64 + (i - p * per_pass)] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    KeyMap km;
    km.load(range);
    // mapped keys lie in [0, top]: digits above its top bit are zero for every key,
    // so their histograms are not counted (they stay zero, and the pass is skipped);
    // a split's far keys count as digit 255 in the passes that are counted, which
    // places no near key (255 is the last digit) and the later passes never read
    int hp = passes;
    if (km.on) {
        const uint32_t top = km.top();
        const int bits = top == 0u ? 1 : 32 - __clz((int)top);
        const int need = (bits - begin_bit + 7) / 8;
        hp = need < 1 ? 1 : (need < passes ? need : passes);
    }
    // deferred histograms: only the first pass's digits are counted here (each
    // scatter pass counts the next one's), and the keys' bits that vary
    // (bits_or: OR of the keys, OR of their complements) tell which passes run
    if (count_passes < hp) hp = count_passes;
    for (int i = threadIdx.x; i < hp * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    if (threadIdx.x < 2) s_or[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned long long k_or = 0, k_nor = 0;
    const bool skip_far = km.split;   // a partial sort's far keys take no later pass
    uint32_t cur[kP], run[kP];
#pragma unroll
    for (int p = 0; p < kP; ++p) { cur[p] = 0xFFFFFFFFu; run[p] = 0; }
    // DIRECT (a partial sort counting its first digit only): a near key's digit
    // is its rank mod 255, which differs from key to key, so run lengths would
    // not merge counts; one atomic per key instead, with no divergent branch
    // (depth sort 0.546 -> 0.534 ms).  Its own instantiation: the branch alone
    // cost the pair sorts 0.005 ms.
    const bool direct = DIRECT && skip_far && hp == 1 && end_bit - begin_bit >= 8;
    // one key into every pass's run-length count
    auto count = [&](K k) {
        if (bits_or && !(skip_far && k == ~K(0))) {
            k_or |= (unsigned long long)k;
            k_nor |= (unsigned long long)(K)~k;
        }
        if (direct) {
            atomicAdd(&h[0][(uint32_t)(k >> begin_bit) & 0xFFu], 1u);
            return;
        }
#pragma unroll
        for (int p = 0; p < kP; ++p) {
            if (p < hp) {
                const int sh = begin_bit + 8 * p;
                const int nb = min(8, end_bit - sh);
                const uint32_t d = (uint32_t)(k >> sh) & ((1u << nb) - 1u);
                if (d == cur[p]) {
                    ++run[p];
                } else {
                    if (run[p]) atomicAdd(&h[p][cur[p]], run[p]);
                    cur[p] = d;
                    run[p] = 1;
                }
            }
        }
    };
    if constexpr (VEC && sizeof(K) == 4) {
        // 16-byte loads of 4 consecutive keys (keys 16-byte aligned), KB of them per
        // thread per step; the n % 4 last keys by the first threads of CTA 0
        const uint4* __restrict__ kv4 = reinterpret_cast<const uint4*>(keys);
        const uint64_t nv = n / 4;
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * KB;
        for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x * KB + threadIdx.x; v0 < nv; v0 += stride) {
            uint4 q[KB];
#pragma unroll
            for (int b = 0; b < KB; ++b) {
                const uint64_t vi = v0 + (uint64_t)b * blockDim.x;
                q[b] = vi < nv ? kv4[vi] : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int b = 0; b < KB; ++b) {
                if (v0 + (uint64_t)b * blockDim.x >= nv) break;
                count(km(K(q[b].x)));
                count(km(K(q[b].y)));
                count(km(K(q[b].z)));
                count(km(K(q[b].w)));
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < n - nv * 4) count(km(keys[nv * 4 + threadIdx.x]));
    } else {
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * KB;
        for (uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x) * KB + threadIdx.x; i0 < n; i0 += stride) {
            K kv[KB];
#pragma unroll
            for (int b = 0; b < KB; ++b) {
                const uint64_t i = i0 + (uint64_t)b * blockDim.x;
                kv[b] = i < n ? km(keys[i]) : K(0);
            }
#pragma unroll
            for (int b = 0; b < KB; ++b) {
                if (i0 + (uint64_t)b * blockDim.x >= n) break;
                count(kv[b]);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < kP; ++p)
        if (p < hp && run[p]) atomicAdd(&h[p][cur[p]], run[p]);
    if (bits_or) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            k_or |= __shfl_xor_sync(kFull, k_or, d);
            k_nor |= __shfl_xor_sync(kFull, k_nor, d);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicOr(&s_or[0], k_or);
            atomicOr(&s_or[1], k_nor);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < hp * 256; i += blockDim.x) {
        uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&ghist[i], c);
    }
    if (bits_or && threadIdx.x < 2 && s_or[threadIdx.x]) atomicOr(&bits_or[threadIdx.x], s_or[threadIdx.x]);
}

// ghist[p][256] -> exclusive digit bases gbase[p][256], and every pass's route:
// pass 0 always runs, a later pass only if more than one of its digits occurs.
// Deferred histograms (bits_or given): only pass 0's histogram is known here
// (its bases are written; each later pass's scatter computes its own from the
// histogram the pass before it counted), and a later pass runs if a bit of
// its digit varies among the keys (bits_or: OR of the keys' digit bits and of
// their complements; the digits cover bits [begin_bit, end_bit)).
// near_out (a partial sort whose threshold came from a sample of the keys):
// the near keys are those whose first digit is not 255, so their count is
// written here; if the threshold cuts the kept keys (range[2] <= range[1] -
// range[0]) and fewer than near_target are near, the overflow bit of flags is
// set (the launch set is rendered again without the partial sort).
__global__ void __launch_bounds__(256) k_os_bases(const uint32_t* __restrict__ ghist, uint32_t* __restrict__ gbase,
                                                  int passes, OsRoute* __restrict__ routes, OsBuffers bufs,
                                                  uint32_t* __restrict__ n_active_out, bool near_split,
                                                  const unsigned long long* __restrict__ bits_or, int begin_bit,
                                                  int end_bit, uint64_t n_cap, const uint64_t* d_n_later,
                                                  uint64_t* __restrict__ near_out, uint64_t near_target,
                                                  const uint32_t* __restrict__ range, uint32_t* __restrict__ flags) {
    __shared__ uint32_t ws[9];
    __shared__ uint32_t act[8];
    // the count the later passes run over
    const uint32_t n_later = near_out ? (uint32_t)(count_of(n_cap, nullptr) - ghist[255]) : count_of(n_cap, d_n_later);
    if (near_out && threadIdx.x == 0) {
        *near_out = n_later;
        const uint32_t top = range[1] - range[0];
        if (range[0] <= range[1] && range[2] <= top && n_later < near_target) atomicOr(flags, 1u);
    }
    const int width = end_bit - begin_bit;   // 1 .. 64
    const unsigned long long varies =
        bits_or ? ((bits_or[0] & bits_or[1]) >> begin_bit) & (width >= 64 ? ~0ull : (1ull << width) - 1ull) : 0ull;
    for (int p = 0; p < passes; ++p) {
        if (bits_or && p > 0) {
            const uint32_t digit_var = (uint32_t)((varies >> (8 * p)) & 0xFFull);
            if (threadIdx.x == 0) act[p] = digit_var != 0u ? 1u : 0u;
            if (digit_var == 0u) {
                // a pass that does not run: every key has the same digit c (the bits of
                // the OR of the keys), so its bases are 0 up to c and the count after
                const uint32_t c = (uint32_t)((bits_or[0] >> (begin_bit + 8 * p)) & 0xFFull);
                gbase[p * 256 + threadIdx.x] = threadIdx.x <= c ? 0u : n_later;
            }
            continue;
        }
        const uint32_t x = ghist[p * 256 + threadIdx.x];
        const uint32_t e = cta_exclusive_scan<256>(x, ws);
        gbase[p * 256 + threadIdx.x] = e;
        const int nz = __syncthreads_count(x != 0u);
        if (threadIdx.x == 0) act[p] = (p == 0 || nz > 1) ? 1u : 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int n_act = 0;
        for (int p = 0; p < passes; ++p) n_act += (int)act[p];
        if (n_active_out) *n_active_out = (uint32_t)n_act;
        const void* sk = bufs.in_k;
        const uint32_t* sv = bufs.in_v;
        const uint2* spp = bufs.in_p;
        int i = 0;
        for (int p = 0; p < passes; ++p) {
            OsRoute r{};
            r.active = act[p];
            if (act[p]) {
                const bool to_out = ((n_act - 1 - i) % 2) == 0;
                r.src_k = sk;
                r.src_v = sv;
                r.src_p = spp;
                r.dst_k = to_out ? bufs.out_k : bufs.alt_k;
                r.dst_v = to_out ? bufs.out_v : bufs.alt_v;
                r.dst_p = bufs.in_p ? (to_out ? bufs.out_p : bufs.alt_p) : nullptr;
                if (near_split && i == 0) {
                    r.far_k = bufs.out_k;
                    r.far_v = bufs.out_v;
                    r.far_p = bufs.in_p ? bufs.out_p : nullptr;
                }
                r.next = -1;
                for (int q = p + 1; q < passes; ++q)
                    if (act[q]) {
                        r.next = q;
                        break;
                    }
                sk = r.dst_k;
                sv = r.dst_v;
                spp = r.dst_p;
                ++i;
            }
            routes[p] = r;
        }
    }
}

// Decoupled look-back of one digit: the sum of the counts of chunks before
// `chunk`, walking back kLookWin chunks per round (independent loads in flight),
// adding aggregates until an inclusive prefix and re-polling a chunk not yet
// published.  Publishes this chunk's inclusive prefix; `publish_agg` first
// publishes its own count (when the caller has not already done so).
template <int kLookWin>
__device__ inline uint32_t lookback_exclusive(uint32_t* status, uint32_t chunk, uint32_t d, uint32_t cnt,
                                              bool publish_agg, uint32_t* flags, int spin_limit) {
    uint32_t* my = status + (size_t)chunk * 256 + d;
    if (chunk == 0) {
        if (publish_agg) st_relaxed(my, kFlagPre | (cnt & kValMask));
        return 0u;
    }
    if (publish_agg) st_relaxed(my, kFlagAgg | (cnt & kValMask));
    uint32_t excl = 0;
    int64_t j = (int64_t)chunk - 1;
    int spins = 0;
    while (j >= 0) {
        uint32_t sv[kLookWin];
#pragma unroll
        for (int t = 0; t < kLookWin; ++t)
            sv[t] = j - t >= 0 ? ld_relaxed(status + (size_t)(j - t) * 256 + d) : kFlagPre;
        bool found = false, stalled = false;
#pragma unroll
        for (int t = 0; t < kLookWin; ++t) {
            if (found || stalled) continue;
            const uint32_t fl = sv[t] & kFlagMask;
            if (fl == 0) {
                stalled = true;
                continue;
            }
            excl += sv[t] & kValMask;
            --j;
            found = fl == kFlagPre;
        }
        if (found) break;
        if (stalled) {
            if (++spins > spin_limit) {
                atomicOr(flags, kSortTimeoutFlag);
                break;
            }
            if (spins > 32) __nanosleep(32);
        }
    }
    st_relaxed(my, kFlagPre | ((excl + cnt) & kValMask));
    return excl;
}

template <typename K, int PAY>
struct OsSmem {
    static constexpr int T = OsCfg<K, PAY>::kT, I = OsCfg<K, PAY>::kI, N = T * I, W = T / 32;
    K keys[N];
    uint32_t vals[PAY == kPayOnly ? 1 : N];
    uint2 pays[PAY ? N : 1];
    uint32_t whist[W][256];
    uint32_t dstart[256];
    uint32_t gshift[256];   // global position of the digit's first key in this tile, minus its tile position
    uint32_t bases[256];    // deferred histograms: this pass's digit bases
    uint32_t nhist[256];    // deferred histograms: the next pass's digit counts of this tile
    uint32_t ws[W + 1];
    uint32_t chunk;
};

template <typename K, int PAY, bool MAP>
__global__ void __launch_bounds__(OsCfg<K, PAY>::kT, OsCfg<K, PAY>::kMinBlocks)
k_os_scatter(const OsRoute* __restrict__ route, uint64_t n_cap, const uint64_t* d_n, int shift, int nbits,
             uint32_t* __restrict__ gbase, uint32_t* status, uint32_t* chunk_counter, uint32_t* flags,
             int spin_limit, const uint32_t* __restrict__ range, uint32_t* __restrict__ ghist_all, int pass,
             int begin_bit, int end_bit) {
    if (route->active == 0u) return;   // identity pass: skipped by every CTA
    // a grid sized for the capacity (graph replays size the pair sorts for the
    // largest slice): CTAs past the keys leave before claiming a chunk, so the
    // CTAs that stay claim exactly the chunks that hold keys (measured: pair
    // sorts 0.543 -> 0.515 ms)
    if ((uint64_t)blockIdx.x * (OsCfg<K, PAY>::kT * OsCfg<K, PAY>::kI) >= count_of(n_cap, d_n)) return;
    const K* __restrict__ keys_in = static_cast<const K*>(route->src_k);
    const uint32_t* __restrict__ vals_in = route->src_v;
    const uint2* __restrict__ pays_in = route->src_p;
    K* __restrict__ keys_out = static_cast<K*>(route->dst_k);
    uint32_t* __restrict__ vals_out = route->dst_v;
    uint2* __restrict__ pays_out = route->dst_p;
    // a partial sort's first pass: digit 255 (the far keys) goes to the output buffers
    K* const far_k = static_cast<K*>(route->far_k);
    uint32_t* const far_v = route->far_v;
    uint2* const far_p = route->far_p;
    // deferred histograms (ghist_all given): a later pass's digit bases come from the
    // count the pass before it made, and a pass counts the digits of the next one
    const uint32_t* const hist_this = ghist_all && pass > 0 ? ghist_all + 256 * pass : nullptr;
    const int next = ghist_all ? route->next : -1;
    uint32_t* const hist_next = next > 0 ? ghist_all + 256 * next : nullptr;
    const int nshift = begin_bit + 8 * (next > 0 ? next : 0);
    const int next_bits = min(8, end_bit - nshift);
    const bool has_vals = PAY != kPayOnly && vals_out != nullptr;   // no value stream: the payload identifies each key
    // The payload sort (few, large launches) walks back for its digit offsets
    // only after its tile is sorted in shared memory, so the wait overlaps that
    // work (measured: depth sort 0.856 -> 0.849 ms); the key/value sorts of the
    // slices (many small launches, one wave each) walk back first, as the later
    // inclusive prefix lengthens their chain (0.643 -> 0.700 ms when walked late).
    constexpr bool kLate = PAY == kPayOnly;
    // look-back window and leader test, per sort (measured on the 8-view launch set):
    // depth sort 4 predecessors and the first-peer leader, pair sorts 2 and the
    // no-lower-peer leader
    constexpr int kWin = PAY == kPayOnly ? 4 : 2;
    constexpr bool kLowerLeader = PAY != kPayOnly;
    const uint32_t mask = (1u << nbits) - 1u;
    constexpr int T = OsCfg<K, PAY>::kT, I = OsCfg<K, PAY>::kI, N = T * I, W = T / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OsSmem<K, PAY>& sm = *reinterpret_cast<OsSmem<K, PAY>*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    KeyMap km;
    if (MAP) km.load(range);
    const uint32_t n = count_of(n_cap, d_n);
    if (hist_next)
        for (int k = threadIdx.x; k < 256; k += T) sm.nhist[k] = 0;
    if (hist_this) {
        // deferred histograms: the digit bases from the count the previous pass made
        const uint32_t x = threadIdx.x < 256 ? hist_this[threadIdx.x] : 0u;
        const uint32_t e = cta_exclusive_scan<T>(x, sm.ws);
        if (threadIdx.x < 256) {
            sm.bases[threadIdx.x] = e;
            if (blockIdx.x == 0) gbase[threadIdx.x] = e;   // for readers after the sort
        }
    }
    // Persistent CTAs: each claims chunks in order until none is left (a grid of
    // at most the resident CTAs), so a small sort launches no CTAs that only leave.
    // A claimed chunk's predecessors are held by running CTAs, so every look-back ends.
    for (;;) {
        if (threadIdx.x == 0) sm.chunk = atomicAdd(chunk_counter, 1u);
        for (int k = threadIdx.x; k < W * 256; k += T) (&sm.whist[0][0])[k] = 0;
        __syncthreads();
        const uint32_t chunk = sm.chunk;
        const uint64_t base = (uint64_t)chunk * N;
        if (base >= n) break;   // CTA-uniform; no later chunk waits on it
        const uint32_t valid = (n - base) < (uint64_t)N ? (uint32_t)(n - base) : (uint32_t)N;

        K key[I];
        uint32_t val[I];
        uint2 pay[PAY ? I : 1];
    #pragma unroll
        for (int r = 0; r < I; ++r) {
            const uint32_t li = warp * (I * 32) + r * 32 + lane;
            if (li < valid) {
                key[r] = keys_in[base + li];
                if constexpr (MAP) key[r] = km(key[r]);   // stored mapped: later passes need no map
                val[r] = !has_vals ? 0u : vals_in ? vals_in[base + li] : (uint32_t)(base + li);
                if (PAY) pay[r] = pays_in[base + li];
            } else {
                key[r] = ~K(0);
                val[r] = 0;
                if (PAY) pay[r] = make_uint2(0u, 0u);
            }
        }
        if (hist_next) {
            // the next pass's digit counts (a partial sort's far keys take no later pass)
            const uint32_t nmask = (1u << next_bits) - 1u;
    #pragma unroll
            for (int r = 0; r < I; ++r) {
                const uint32_t li = warp * (I * 32) + r * 32 + lane;
                if (li < valid && !(far_k != nullptr && key[r] == ~K(0)))
                    atomicAdd(&sm.nhist[(uint32_t)(key[r] >> nshift) & nmask], 1u);
            }
        }
        uint32_t dr[I];
        const uint32_t lt = lanemask_lt();
    #pragma unroll
        for (int r = 0; r < I; ++r) {
            // padding keys (all ones) take the largest digit, so they sort after every
            // key; a mapped key is at most the map's span, below all ones
            const uint32_t d = (uint32_t)(key[r] >> shift) & mask;
            // peers by one ballot per digit bit (measured faster here than match.any
            // with shared-memory atomics)
            const uint32_t peers = digit_peers(d);
            const uint32_t before = sm.whist[warp][d];
            const uint32_t lower = peers & lt;   // peers in lower lanes
            __syncwarp();
            if (kLowerLeader ? lower == 0u : lane == __ffs(peers) - 1) sm.whist[warp][d] = before + __popc(peers);
            __syncwarp();
            dr[r] = (d << 16) | (before + __popc(lower));
        }
        __syncthreads();

        // per digit: prefix over warps, the CTA's count, and look-back for earlier chunks
        uint32_t cnt = 0;
        if (threadIdx.x < 256) {
            const uint32_t d = threadIdx.x;
    #pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint32_t c = sm.whist[w][d];
                sm.whist[w][d] = cnt;
                cnt += c;
            }
            // padding keys (digit == mask) are not part of this chunk's counts
            if (d == mask) cnt -= (uint32_t)(N - valid);
            if constexpr (kLate) {
                // this chunk's counts now; the walk back waits until the tile is sorted in shared memory
                st_relaxed(status + (size_t)chunk * 256 + d, (chunk == 0 ? kFlagPre : kFlagAgg) | (cnt & kValMask));
            } else {
                const uint32_t excl = lookback_exclusive<kWin>(status, chunk, d, cnt, true, flags, spin_limit);
                sm.gshift[d] = (d <= mask ? (hist_this ? sm.bases[d] : gbase[d]) : 0u) + excl;   // tile position subtracted below
            }
        }
        // restore the padding count for the in-tile layout (padding sorts last)
        const uint32_t local_cnt = threadIdx.x < 256 ? cnt + ((threadIdx.x == mask) ? (uint32_t)(N - valid) : 0u) : 0u;
        const uint32_t start = cta_exclusive_scan<T>(local_cnt, sm.ws);
        if (threadIdx.x < 256) {
            sm.dstart[threadIdx.x] = start;
            if constexpr (!kLate) sm.gshift[threadIdx.x] -= start;
        }
        __syncthreads();

    #pragma unroll
        for (int r = 0; r < I; ++r) {
            const uint32_t d = dr[r] >> 16;
            const uint32_t pos = sm.dstart[d] + sm.whist[warp][d] + (dr[r] & 0xFFFFu);
            sm.keys[pos] = key[r];
            if (has_vals) sm.vals[pos] = val[r];
            if (PAY) sm.pays[pos] = pay[r];
        }
        if constexpr (kLate) {
            if (threadIdx.x < 256) {
                const uint32_t d = threadIdx.x;
                const uint32_t excl = lookback_exclusive<kWin>(status, chunk, d, cnt, false, flags, spin_limit);
                sm.gshift[d] = (d <= mask ? (hist_this ? sm.bases[d] : gbase[d]) : 0u) + excl - start;
            }
        }
        __syncthreads();
    #pragma unroll 4
        for (int k = 0; k < I; ++k) {
            const uint32_t j = k * T + threadIdx.x;
            if (j < valid) {
                const K kk = sm.keys[j];
                const uint32_t d = (uint32_t)(kk >> shift) & mask;
                const uint32_t g = sm.gshift[d] + j;
                if (g < n) {
                    const bool far = far_k != nullptr && d == 255u;
                    (far ? far_k : keys_out)[g] = kk;
                    if (has_vals) (far ? far_v : vals_out)[g] = sm.vals[j];
                    if (PAY) (far ? far_p : pays_out)[g] = sm.pays[j];
                }
            }
        }
        __syncthreads();   // the next chunk's claim and counts reuse the shared arrays
    }
    if (hist_next && threadIdx.x < 256 && sm.nhist[threadIdx.x]) atomicAdd(&hist_next[threadIdx.x], sm.nhist[threadIdx.x]);
}

template <typename K, int PAY, bool MAP>
Status ensure_os_smem() {
    static std::atomic<bool> done[kMaxDevices];
    int slot = -1;
    TIGAS_TRY(current_device_slot(&slot));
    if (slot >= 0 && done[slot].load()) return {};
    TIGAS_CUDA_TRY(cudaFuncSetAttribute(k_os_scatter<K, PAY, MAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(OsSmem<K, PAY>)));
    // the largest shared-memory carveout, so that two CTAs fit per SM
    TIGAS_CUDA_TRY(
        cudaFuncSetAttribute(k_os_scatter<K, PAY, MAP>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    if (slot >= 0) done[slot].store(true);
    return {};
}

uint64_t os_chunks(uint64_t n_cap) { return (n_cap + 4095) / 4096; }   // upper bound for every tile shape

#ifndef TIGAS_OS_HIST_CTAS
#define TIGAS_OS_HIST_CTAS 2   // histogram CTAs per SM at most (grid-stride over the keys)
#endif
#ifndef TIGAS_OS_SCATTER_CTAS
#define TIGAS_OS_SCATTER_CTAS 0   // persistent scatter CTAs per SM (0: as many as are resident)
#endif
#ifndef TIGAS_OS_PERSIST
#define TIGAS_OS_PERSIST 1
#endif
#ifndef TIGAS_OS_DEFER
#define TIGAS_OS_DEFER 1
#endif
// tmp layout: chunk counters [8], flags [1], (unused) [1], OR of the keys and
// of their complements [2 x u64], (unused) [1], active passes [1], ghist [8][256],
// gbase [8][256], routes [8], status [pass][chunks][256] (cleared by the
// histogram kernel); the words a sort of p passes needs zeroed on entry are
// the first radix_zero_words(p) (counters, flags and p histograms), and the
// status table starts 16-byte aligned
constexpr size_t kOsHead = (16 + 8 * 256 * 2 + 8 * kRouteWords + 3) / 4 * 4;
static_assert((16 + 8 * 256 * 2) % 2 == 0, "routes hold pointers: 8-byte aligned");
size_t os_tmp_words(uint64_t n_cap) { return kOsHead + 8 * os_chunks(n_cap) * 256; }

template <typename K, int PAY, bool MAP>
Status radix_sort_onesweep(const K* keys_in, const uint32_t* values_in, K* keys_alt, uint32_t* values_alt,
                           K* keys_out, uint32_t* values_out, uint64_t n_cap, const uint64_t* d_n, int begin_bit,
                           int end_bit, uint32_t* tmp, cudaStream_t st, uint32_t* flags, const SortExtras* ex) {
    constexpr int T = OsCfg<K, PAY>::kT, N = OsCfg<K, PAY>::kT * OsCfg<K, PAY>::kI;
    static_assert(N >= 4096, "the status table (os_chunks) assumes chunks of at least 4096 keys");
    const int passes = (end_bit - begin_bit + 7) / 8;
    TIGAS_TRY((ensure_os_smem<K, PAY, MAP>()));
    uint32_t* counters = tmp;
    uint32_t* own_flags = counters + 8;
    uint32_t* ghist = tmp + 16;
    uint32_t* gbase = ghist + 8 * 256;
    OsRoute* routes = reinterpret_cast<OsRoute*>(gbase + 8 * 256);
    uint32_t* status = tmp + kOsHead;
    if (!flags) flags = own_flags;
    const uint32_t* range = MAP ? ex->key_range : nullptr;
    const uint64_t chunks = (n_cap + N - 1) / N;
    if (!(ex && ex->tmp_zeroed))
        TIGAS_CUDA_TRY(cudaMemsetAsync(tmp, 0, radix_zero_words(passes) * sizeof(uint32_t), st));
    // enough CTAs for eight grid strides of 4 keys per thread, at most 8 per SM
    constexpr int kHistKeys = MAP ? 4 : 8;
    constexpr int kHistVecs = 2;
    const bool vec = sizeof(K) == 4 && (reinterpret_cast<uintptr_t>(keys_in) & 15u) == 0;
    // eight grid strides, at most TIGAS_OS_HIST_CTAS CTAs per SM (a vector step covers 4
    // keys per load; measured on the 8-view launch set at 8 / 4 / 2 / 1 CTAs per SM:
    // 3.208 / 3.201 / 3.189 / 3.250 ms, the grid sized for a slice's pair capacity
    // leaving most of 8 per SM idle)
    const uint64_t hist_step = (uint64_t)512 * (vec ? kHistVecs * 4 : kHistKeys) * 8;
    const uint64_t hist_ctas = (n_cap + hist_step - 1) / hist_step;
    constexpr uint64_t kHistMax = (uint64_t)kSmCount * TIGAS_OS_HIST_CTAS;
    const unsigned hgrid = (unsigned)(hist_ctas < kSmCount ? kSmCount : (hist_ctas > kHistMax ? kHistMax : hist_ctas));
    // deferred histograms: the histogram kernel counts the first pass's digits
    // (and ORs the keys' bits, which tell the passes that run), each scatter
    // pass the next one's
    const bool deferred = TIGAS_OS_DEFER && passes > 1;
    unsigned long long* bits_or = deferred ? reinterpret_cast<unsigned long long*>(counters + 10) : nullptr;
    const int count_passes = deferred ? 1 : passes;
    const bool direct = MAP && ex != nullptr && ex->near_split && count_passes == 1;
    if (vec && direct)
        k_os_hist<K, kHistVecs, true, true><<<hgrid, 512, 0, st>>>(keys_in, n_cap, d_n, begin_bit, end_bit, ghist,
                                                                    range, reinterpret_cast<uint4*>(status), chunks,
                                                                    (uint32_t)N, count_passes, bits_or);
    else if (vec)
        k_os_hist<K, kHistVecs, true, false><<<hgrid, 512, 0, st>>>(keys_in, n_cap, d_n, begin_bit, end_bit, ghist,
                                                                     range, reinterpret_cast<uint4*>(status), chunks,
                                                                     (uint32_t)N, count_passes, bits_or);
    else
        k_os_hist<K, kHistKeys, false, false><<<hgrid, 512, 0, st>>>(keys_in, n_cap, d_n, begin_bit, end_bit, ghist,
                                                                      range, reinterpret_cast<uint4*>(status), chunks,
                                                                      (uint32_t)N, count_passes, bits_or);
    TIGAS_LAUNCHED();
    OsBuffers bufs{keys_in, values_in, PAY ? ex->pay_in : nullptr, keys_alt, values_alt, PAY ? ex->pay_alt : nullptr,
                   keys_out, values_out, PAY ? ex->pay_out : nullptr};
    const bool split = MAP && ex->near_split;
    // a sampled threshold: the near count comes from the first digit's histogram
    uint64_t* near_out = split && ex->near_sampled ? const_cast<uint64_t*>(ex->d_near) : nullptr;
    k_os_bases<<<1, 256, 0, st>>>(ghist, gbase, passes, routes, bufs, counters + 15, split, bits_or, begin_bit,
                                  end_bit, n_cap, split ? ex->d_near : d_n, near_out, split ? ex->near_target : 0,
                                  range, flags);
    TIGAS_LAUNCHED();
    // scatter CTAs: persistent, at most the CTAs resident at once
    const uint64_t resident = (uint64_t)kSmCount * (TIGAS_OS_SCATTER_CTAS > 0 ? TIGAS_OS_SCATTER_CTAS : OsCfg<K, PAY>::kMinBlocks);
    const unsigned sgrid = (unsigned)(TIGAS_OS_PERSIST && chunks > resident ? resident : chunks);
    for (int p = 0; p < passes; ++p) {
        const int shift = begin_bit + 8 * p;
        const int nb = min(8, end_bit - shift);
        // a partial sort's later passes run over the near keys only
        const uint64_t* pn = split && p > 0 ? ex->d_near : d_n;
        if (MAP && p > 0) {
            // the first pass (always run) stored mapped keys: later passes read them as they are
            TIGAS_TRY((ensure_os_smem<K, PAY, false>()));
            k_os_scatter<K, PAY, false><<<sgrid, T, sizeof(OsSmem<K, PAY>), st>>>(
                routes + p, n_cap, pn, shift, nb, gbase + p * 256, status + (size_t)p * chunks * 256, counters + p,
                flags, kSpinLimit, nullptr, deferred ? ghist : nullptr, p, begin_bit, end_bit);
        } else {
            k_os_scatter<K, PAY, MAP><<<sgrid, T, sizeof(OsSmem<K, PAY>), st>>>(
                routes + p, n_cap, pn, shift, nb, gbase + p * 256, status + (size_t)p * chunks * 256, counters + p,
                flags, kSpinLimit, range, deferred ? ghist : nullptr, p, begin_bit, end_bit);
        }
        TIGAS_LAUNCHED();
    }
    return {};
}

}  // namespace

namespace {
// Look-back probe layout (words): keys [2N], sorted keys [2N], sorted values
// [2N], digit histogram [256], digit bases [256], status [2][256], misc [8]
// (chunk counter, own flags word), routes [2].
constexpr uint64_t kProbeN = 2 * (uint64_t)OsCfg<uint32_t, kPayNone>::kT * OsCfg<uint32_t, kPayNone>::kI;
constexpr size_t kProbeKeys = 0, kProbeOut = kProbeN, kProbeVals = 2 * kProbeN, kProbeHist = 3 * kProbeN,
                 kProbeBase = kProbeHist + 256, kProbeStatus = kProbeBase + 256, kProbeMisc = kProbeStatus + 2 * 256,
                 kProbeRoute = kProbeMisc + 8, kProbeWords = kProbeRoute + 2 * kRouteWords;
static_assert(kProbeRoute % 2 == 0, "routes hold pointers: 8-byte aligned");

// Probe inputs: distinct-ish keys, zeroed tables, the chunk counter at 1 (the
// only CTA claims chunk 1) and the probe's own flags word at 0.
__global__ void k_probe_init(uint32_t* __restrict__ buf) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < kProbeRoute;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t v = 0;
        if (i < kProbeOut) v = (uint32_t)((i * 2654435761u) >> 7);
        else if (i == kProbeMisc) v = 1u;
        if (i < kProbeOut || i >= kProbeHist) buf[i] = v;
    }
}
}  // namespace

size_t debug_lookback_words() { return kProbeWords; }

// One scatter CTA of a two-chunk, one-pass sort that claims chunk 1 while no
// CTA ever runs chunk 0: its look-back waits on counts nobody publishes, so
// every wait runs out after spin_limit polls and the CTA ORs the timeout flag
// into *flags.  Bounds, by reading: the digit bases come from the histogram of
// both chunks, so every scattered position is below 2N = kProbeN and lands in
// the out / vals regions; the status table holds 2 x 256 words.
Status debug_lookback_enqueue(int spin_limit, uint32_t* buf, uint32_t* flags, cudaStream_t st) {
    using K = uint32_t;
    constexpr int T = OsCfg<K, kPayNone>::kT;
    if (spin_limit < 1 || spin_limit > (1 << 20)) return {TIGAS_ERR_INVALID, "spin limit out of 1..2^20"};
    if (reinterpret_cast<uintptr_t>(buf) & 15u) return {TIGAS_ERR_INVALID, "probe buffer not 16-byte aligned"};
    TIGAS_TRY((ensure_os_smem<K, kPayNone, false>()));
    K* keys = buf + kProbeKeys;
    K* out = buf + kProbeOut;
    uint32_t* vals = buf + kProbeVals;
    uint32_t* ghist = buf + kProbeHist;
    uint32_t* gbase = buf + kProbeBase;
    uint32_t* status = buf + kProbeStatus;
    uint32_t* misc = buf + kProbeMisc;
    OsRoute* route = reinterpret_cast<OsRoute*>(buf + kProbeRoute);
    k_probe_init<<<16, 256, 0, st>>>(buf);
    OsBuffers bufs{keys, nullptr, nullptr, out, vals, nullptr, out, vals, nullptr};
    k_os_hist<K, 8, false, false><<<4, 512, 0, st>>>(keys, kProbeN, nullptr, 0, 8, ghist, nullptr, nullptr, 0, 1, 1,
                                               nullptr);
    k_os_bases<<<1, 256, 0, st>>>(ghist, gbase, 1, route, bufs, nullptr, false, nullptr, 0, 8, kProbeN, nullptr,
                                  nullptr, 0, nullptr, nullptr);
    k_os_scatter<K, kPayNone, false><<<1, T, sizeof(OsSmem<K, kPayNone>), st>>>(
        route, kProbeN, nullptr, 0, 8, gbase, status, misc, flags ? flags : misc + 1, spin_limit, nullptr, nullptr,
        0, 0, 8);
    g_launches.fetch_add(4, std::memory_order_relaxed);
    TIGAS_CUDA_TRY(cudaGetLastError());
    return {};
}

Status debug_lookback_timeout(int spin_limit, bool* timed_out) {
    *timed_out = false;
    if (spin_limit < 1 || spin_limit > (1 << 20)) return {TIGAS_ERR_INVALID, "spin limit out of 1..2^20"};
    uint32_t* buf = nullptr;
    TIGAS_CUDA_TRY(device_alloc(&buf, kProbeWords * sizeof(uint32_t)));
    Status st = debug_lookback_enqueue(spin_limit, buf, nullptr, nullptr);
    uint32_t flags = 0;
    cudaError_t e = cudaSuccess;
    if (st.ok()) e = cudaDeviceSynchronize();
    if (st.ok() && e == cudaSuccess)
        e = cudaMemcpy(&flags, buf + kProbeMisc + 1, sizeof(flags), cudaMemcpyDeviceToHost);
    if (st.ok() && e != cudaSuccess)
        st = {TIGAS_ERR_CUDA, std::string("look-back timeout probe: ") + cudaGetErrorString(e)};
    cudaFree(buf);
    *timed_out = (flags & kSortTimeoutFlag) != 0;
    return st;
}

namespace {
// Histogram of (k - kmin) >> shift over the kept keys (run-length aggregated
// shared-memory counts, as in the sort's histogram), then, in the CTA that
// finishes last, the first bin whose inclusive count reaches the target.
constexpr int kSplitThreads = 1024;
#ifndef TIGAS_SPLIT_KEYS
#define TIGAS_SPLIT_KEYS 8
#endif
__global__ void __launch_bounds__(kSplitThreads)
k_near_split(const uint32_t* __restrict__ keys, uint32_t n, uint32_t* __restrict__ range, uint64_t target,
             uint32_t* __restrict__ ghist, uint64_t* __restrict__ d_near, uint32_t* __restrict__ sort_zero,
             int n_sort_zero, uint32_t stride) {
    __shared__ uint32_t h[kSplitBins];
    __shared__ uint32_t ws[kSplitThreads / 32 + 1];
    __shared__ int last;
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < n_sort_zero; i += kSplitThreads) sort_zero[i] = 0u;
    for (int i = threadIdx.x; i < kSplitBins; i += kSplitThreads) h[i] = 0;
    __syncthreads();
    const uint32_t kmin = range[0], kmax = range[1];
    const bool any = kmin <= kmax;   // at least one kept key
    const uint32_t top = any ? kmax - kmin : 0u;
    const int bits = top == 0u ? 0 : 32 - __clz((int)top);
    const int shift = bits > 11 ? bits - 11 : 0;   // top >> shift < kSplitBins
    uint32_t cur = 0xFFFFFFFFu, run = 0;
    auto count = [&](uint32_t k) {
        if (k == 0xFFFFFFFFu) return;   // culled: never near
        const uint32_t b = (k - kmin) >> shift;
        if (b == cur) {
            ++run;
        } else {
            if (run) atomicAdd(&h[cur], run);
            cur = b;
            run = 1;
        }
    };
    const uint4* __restrict__ k4 = reinterpret_cast<const uint4*>(keys);
    const uint32_t nv = n / 4;
    // every key, or (stride > 1) every stride-th group of 4
    for (uint64_t v = ((uint64_t)blockIdx.x * kSplitThreads + threadIdx.x) * stride; v < nv;
         v += (uint64_t)gridDim.x * kSplitThreads * stride) {
        const uint4 q = k4[v];
        count(q.x);
        count(q.y);
        count(q.z);
        count(q.w);
    }
    if (stride == 1 && blockIdx.x == 0 && threadIdx.x < n - nv * 4) count(keys[nv * 4 + threadIdx.x]);
    if (run) atomicAdd(&h[cur], run);
    __syncthreads();
    for (int i = threadIdx.x; i < kSplitBins; i += kSplitThreads)
        if (h[i]) atomicAdd(&ghist[i], h[i]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ghist[kSplitBins], 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // every CTA's counts are in: thread t holds bins 2t and 2t + 1
    static_assert(kSplitBins == 2 * kSplitThreads, "two bins per thread");
    const uint32_t c0 = __ldcg(&ghist[2 * threadIdx.x]), c1 = __ldcg(&ghist[2 * threadIdx.x + 1]);
    const uint32_t ex = cta_exclusive_scan<kSplitThreads>(c0 + c1, ws);
    // the count to reach: with a sample, the target's share of the sampled keys
    // and a margin of 1 % of them (the sort checks the exact near count)
    uint64_t want = target;
    if (stride > 1) {
        const uint64_t ns = 4ull * ((nv + stride - 1) / stride);   // keys sampled, culled ones included
        want = (target * ns + n - 1) / n + ns / 100 + 64;
    }
    if (threadIdx.x == kSplitThreads - 1) {
        const uint64_t kept = (uint64_t)ex + c0 + c1;
        if (want > kept) {   // every kept key is near
            range[2] = any ? top + 1u : 0u;
            if (stride == 1) *d_near = kept;
            range[3] = 1u;
        }
    }
    if (want >= 1 && (uint64_t)ex < want && want <= (uint64_t)ex + c0 + c1) {
        const bool first = (uint64_t)ex + c0 >= want;
        const uint64_t bin = 2u * threadIdx.x + (first ? 0u : 1u);
        const uint64_t thr = (bin + 1u) << shift;
        range[2] = (uint32_t)(thr < (uint64_t)top + 1u ? thr : (uint64_t)top + 1u);
        if (stride == 1) *d_near = (uint64_t)ex + c0 + (first ? 0u : c1);
        range[3] = 1u;
    }
}
}  // namespace

Status launch_near_split(const uint32_t* keys, uint64_t n, uint32_t* key_range, uint64_t target, uint32_t* hist,
                         uint64_t* d_near, uint32_t* sort_zero, int n_sort_zero, int sample, cudaStream_t st) {
    if (n == 0 || n >= 0xFFFFFFFFull || target == 0) return {TIGAS_ERR_INVALID, "split: empty or oversized sort"};
    if (reinterpret_cast<uintptr_t>(keys) & 15u) return {TIGAS_ERR_INVALID, "split: keys not 16-byte aligned"};
    if (sample < 1) return {TIGAS_ERR_INVALID, "split: sample stride below 1"};
    // about TIGAS_SPLIT_KEYS keys per thread (of those read), at most two CTAs
    // per SM: a thread's loads of a sample lie a stride apart, so each is a DRAM
    // round trip, and fewer of them per thread shorten the kernel's latency chain
    const uint64_t per_cta = (uint64_t)kSplitThreads * TIGAS_SPLIT_KEYS * (uint64_t)sample;
    uint64_t grid = (n + per_cta - 1) / per_cta;
    if (grid > 2 * (uint64_t)kSmCount) grid = 2 * (uint64_t)kSmCount;
    k_near_split<<<(unsigned)grid, kSplitThreads, 0, st>>>(keys, (uint32_t)n, key_range, target, hist, d_near,
                                                           sort_zero, sort_zero ? n_sort_zero : 0,
                                                           (uint32_t)sample);
    TIGAS_LAUNCHED();
    return {};
}

const uint32_t* radix_active_passes(const uint32_t* tmp) { return tmp + 15; }
const uint32_t* radix_digit_bases(const uint32_t* tmp, int pass) { return tmp + 16 + 8 * 256 + 256 * pass; }
size_t radix_zero_words(int passes) { return 16 + 256 * (size_t)passes; }

size_t radix_tmp_words(uint64_t n_cap) {
    size_t a = rts_tmp_words(n_cap), b = os_tmp_words(n_cap);
    return a > b ? a : b;
}

template <typename K>
Status radix_sort(const K* keys_in, const uint32_t* values_in, K* keys_alt, uint32_t* values_alt, K* keys_out,
                  uint32_t* values_out, uint64_t n_cap, const uint64_t* d_n, int begin_bit, int end_bit,
                  uint32_t* tmp, cudaStream_t st, int* passes_out, uint32_t* flags, const SortExtras* ex) {
    const int kbits = (int)(8 * sizeof(K));
    if (begin_bit < 0 || end_bit > kbits || begin_bit > end_bit) return {TIGAS_ERR_INVALID, "bad sort bit range"};
    if (n_cap >= 0xFFFFFFFFull) return {TIGAS_ERR_INVALID, "sort too large"};
    const bool pay = ex && ex->pay_in;
    const bool ext = ex && (ex->key_range || ex->pay_in || ex->near_split);   // beyond tmp_zeroed
    if (ext && (sizeof(K) != 4 || (pay && (!ex->pay_alt || !ex->pay_out))))
        return {TIGAS_ERR_INVALID, "key range and payload need 32-bit keys and all three payload buffers"};
    if (ex && ex->near_split && (!ex->key_range || !ex->d_near || d_n || begin_bit != 0 || end_bit != 32))
        return {TIGAS_ERR_INVALID, "a partial sort needs a key range, the near count and all 32 bits of every key"};
    if ((!values_out || !values_alt) && (values_out || values_alt || values_in || !pay))
        return {TIGAS_ERR_INVALID, "values may be omitted only together, and only with a payload"};
    const int passes = (end_bit - begin_bit + 7) / 8;
    if (passes_out) *passes_out = passes;
    if (n_cap == 0) return {};
    if (passes == 0) {
        TIGAS_CUDA_TRY(cudaMemcpyAsync(keys_out, keys_in, n_cap * sizeof(K), cudaMemcpyDeviceToDevice, st));
        if (values_in && values_out)
            TIGAS_CUDA_TRY(cudaMemcpyAsync(values_out, values_in, n_cap * 4, cudaMemcpyDeviceToDevice, st));
        if (pay) TIGAS_CUDA_TRY(cudaMemcpyAsync(ex->pay_out, ex->pay_in, n_cap * 8, cudaMemcpyDeviceToDevice, st));
        return {};
    }
    if (n_cap < (1ull << 30)) {
        if constexpr (sizeof(K) == 4) {
            const bool map = ex && ex->key_range;
            if (pay && !values_out) {
                if (map)
                    return radix_sort_onesweep<K, kPayOnly, true>(keys_in, values_in, keys_alt, values_alt, keys_out,
                                                                  values_out, n_cap, d_n, begin_bit, end_bit, tmp,
                                                                  st, flags, ex);
                return radix_sort_onesweep<K, kPayOnly, false>(keys_in, values_in, keys_alt, values_alt, keys_out,
                                                               values_out, n_cap, d_n, begin_bit, end_bit, tmp, st,
                                                               flags, ex);
            }
            if (pay && map)
                return radix_sort_onesweep<K, kPayWithValues, true>(keys_in, values_in, keys_alt, values_alt,
                                                                    keys_out, values_out, n_cap, d_n, begin_bit,
                                                                    end_bit, tmp, st, flags, ex);
            if (pay)
                return radix_sort_onesweep<K, kPayWithValues, false>(keys_in, values_in, keys_alt, values_alt,
                                                                     keys_out, values_out, n_cap, d_n, begin_bit,
                                                                     end_bit, tmp, st, flags, ex);
            if (map)
                return radix_sort_onesweep<K, kPayNone, true>(keys_in, values_in, keys_alt, values_alt, keys_out,
                                                              values_out, n_cap, d_n, begin_bit, end_bit, tmp, st,
                                                              flags, ex);
        }
        return radix_sort_onesweep<K, kPayNone, false>(keys_in, values_in, keys_alt, values_alt, keys_out,
                                                       values_out, n_cap, d_n, begin_bit, end_bit, tmp, st, flags, ex);
    }
    if (ext || (ex && ex->tmp_zeroed)) return {TIGAS_ERR_INVALID, "sort extras need fewer than 2^30 keys"};
    return radix_sort_rts<K>(keys_in, values_in, keys_alt, values_alt, keys_out, values_out, n_cap, d_n, begin_bit,
                             end_bit, tmp, st);
}

template Status radix_sort<uint32_t>(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint32_t*,
                                     uint64_t, const uint64_t*, int, int, uint32_t*, cudaStream_t, int*, uint32_t*,
                                     const SortExtras*);
template Status radix_sort<uint64_t>(const uint64_t*, const uint32_t*, uint64_t*, uint32_t*, uint64_t*, uint32_t*,
                                     uint64_t, const uint64_t*, int, int, uint32_t*, cudaStream_t, int*, uint32_t*,
                                     const SortExtras*);

}  // namespace tigas
