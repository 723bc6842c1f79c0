// K2 device prefix scan and K4 LSD radix sort.
//
// Both are reduce-then-scan designs: every kernel reads only data written by
// earlier kernels in stream order, so no CTA ever waits on another CTA (no
// spin loops, nothing that can hang a shared GPU).
//
// Radix sort: 8-bit digits, stable.  Per pass:
//   1. hist:    each 4096-key tile counts its digits -> table[digit][tile]
//   2. scan:    exclusive scan of the digit-major table gives, for every
//               (digit, tile), the global output offset of that tile's first
//               key with that digit
//   3. scatter: each tile ranks its keys stably (warp match + per-warp digit
//               counters), reorders them in shared memory, and writes runs of
//               equal digits to their global offsets (coalesced).
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
                       uint32_t* tmp, cudaStream_t st) {
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
    if (total64) TIGAS_CUDA_TRY(cudaMemsetAsync(total64, 0, sizeof(uint64_t), st));
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

template <typename K>
Status ensure_scatter_smem() {
    static std::atomic<bool> done{false};
    if (done.load()) return {};
    TIGAS_CUDA_TRY(cudaFuncSetAttribute(k_radix_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(ScatterSmem<K>)));
    done.store(true);
    return {};
}

}  // namespace

size_t radix_tmp_words(uint64_t n_cap) {
    uint64_t tiles = sort_tiles(n_cap);
    if (tiles == 0) tiles = 1;
    uint64_t table = 256 * tiles;
    return 2 * table + scan_tmp_words(table);
}

template <typename K>
Status radix_sort(const K* keys_in, const uint32_t* values_in, K* keys_alt, uint32_t* values_alt, K* keys_out,
                  uint32_t* values_out, uint64_t n_cap, const uint64_t* d_n, int begin_bit, int end_bit,
                  uint32_t* tmp, cudaStream_t st, int* passes_out) {
    const int kbits = (int)(8 * sizeof(K));
    if (begin_bit < 0 || end_bit > kbits || begin_bit > end_bit) return {TIGAS_ERR_INVALID, "bad sort bit range"};
    if (n_cap >= 0xFFFFFFFFull) return {TIGAS_ERR_INVALID, "sort too large"};
    const int passes = (end_bit - begin_bit + 7) / 8;
    if (passes_out) *passes_out = passes;
    if (n_cap == 0) return {};
    if (passes == 0) {
        TIGAS_CUDA_TRY(cudaMemcpyAsync(keys_out, keys_in, n_cap * sizeof(K), cudaMemcpyDeviceToDevice, st));
        if (values_in)
            TIGAS_CUDA_TRY(cudaMemcpyAsync(values_out, values_in, n_cap * 4, cudaMemcpyDeviceToDevice, st));
        return {};
    }
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

template Status radix_sort<uint32_t>(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint32_t*,
                                     uint64_t, const uint64_t*, int, int, uint32_t*, cudaStream_t, int*);
template Status radix_sort<uint64_t>(const uint64_t*, const uint32_t*, uint64_t*, uint32_t*, uint64_t*, uint32_t*,
                                     uint64_t, const uint64_t*, int, int, uint32_t*, cudaStream_t, int*);

}  // namespace tigas
