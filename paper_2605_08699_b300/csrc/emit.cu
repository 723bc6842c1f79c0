// K3 duplicate-and-key emit and K5 tile-range identification.
//
// Emit: every kept (Gaussian, view) entry owns the tiles of its rectangle.
// A warp takes 32 consecutive entries of the scan order, whose outputs are
// one contiguous run starting at offsets[k of lane 0]; its lanes then write
// that run cooperatively (lane j writes run positions j, j+32, ...), finding
// each position's owner by binary search over the warp's exclusive counts.
// All 32 lanes store to consecutive addresses: fully coalesced writes.
#include "kernels.cuh"

namespace tigas {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

struct ViewTiles {
    uint32_t tile_base;
    uint32_t TX;
};

constexpr int kEmitThreads = 256;

// Each warp takes 32 consecutive entries of the emit order per step
// (grid-stride over steps).  Per lane: the entry's first tile id (view base +
// row base + x_lo), its rect width and a reciprocal of it, so a pair's tile is
// base + (t / w) * TX + t % w with no integer division.
template <bool WIDE>
__global__ void __launch_bounds__(kEmitThreads)
k_emit(const uint32_t* __restrict__ order, const uint32_t* __restrict__ offsets, SplatArrays sp,
       const ViewParams* __restrict__ views_g, int V, uint32_t n_per_view, uint64_t n_entries,
       void* __restrict__ keys_out, uint32_t* __restrict__ values, uint64_t pair_cap,
       uint32_t* __restrict__ overflow) {
    constexpr int W = kEmitThreads / 32;
    __shared__ ViewTiles vt[kMaxViews];
    __shared__ uint32_t s_excl[W][32];
    __shared__ uint32_t s_e[W][32];
    __shared__ uint32_t s_base[W][32];
    __shared__ uint32_t s_wtx[W][32];      // rect width | TX << 16
    __shared__ float s_inv[W][32];
    for (int k = threadIdx.x; k < V; k += blockDim.x) vt[k] = {views_g[k].tile_base, (uint32_t)views_g[k].TX};
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t n_steps = (n_entries + 31) / 32;
    const uint64_t warp_stride = (uint64_t)gridDim.x * W;
    for (uint64_t ws = (uint64_t)blockIdx.x * W + warp; ws < n_steps; ws += warp_stride) {
        const uint64_t k = ws * 32 + lane;
        uint32_t e = 0, cnt = 0, off = 0, base = 0, wtx = 1;
        float inv = 0.0f;
        if (k < n_entries) {
            e = order ? order[k] : (uint32_t)k;
            cnt = sp.tiles[e];
            off = offsets[k];
            if (cnt) {
                const uint2 r = sp.rect[e];
                const uint32_t xlo = r.x & 0x3FFu, ylo = r.y & 0x3FFu, xhi = (r.x >> 10) & 0x3FFu;
                const uint32_t v = e / n_per_view;
                const uint32_t w = xhi - xlo;
                base = vt[v].tile_base + ylo * vt[v].TX + xlo;
                wtx = w | (vt[v].TX << 16);
                inv = 1.0f / (float)w;
            }
        }
        uint32_t inc = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, inc, d);
            if (lane >= d) inc += y;
        }
        const uint32_t total = __shfl_sync(kFull, inc, 31);
        const uint32_t gbase = __shfl_sync(kFull, off, 0);
        if (total == 0) continue;   // warp-uniform
        __syncwarp();
        s_excl[warp][lane] = inc - cnt;
        s_e[warp][lane] = e;
        s_base[warp][lane] = base;
        s_wtx[warp][lane] = wtx;
        s_inv[warp][lane] = inv;
        __syncwarp();
        for (uint32_t j = lane; j < total; j += 32) {
            // owner: last lane whose exclusive count is <= j (steps keep lo + step <= 31)
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (s_excl[warp][lo + step] <= j) lo += step;
            const uint32_t t = j - s_excl[warp][lo];
            const uint32_t ee = s_e[warp][lo];
            const uint32_t wt = s_wtx[warp][lo];
            const uint32_t w = wt & 0xFFFFu, TX = wt >> 16;
            // t / w by a reciprocal: exact for t < 2^18, w <= 512 ((t + 0.5)/w is >= 0.5/w from an integer)
            const uint32_t row = (uint32_t)(((float)t + 0.5f) * s_inv[warp][lo]);
            const uint32_t tile = s_base[warp][lo] + row * TX + (t - row * w);
            const uint64_t pos = (uint64_t)gbase + j;
            if (pos < pair_cap) {
                if (WIDE)
                    reinterpret_cast<uint64_t*>(keys_out)[pos] = ((uint64_t)tile << 32) | sp.depth_key[ee];
                else
                    reinterpret_cast<uint32_t*>(keys_out)[pos] = tile;
                values[pos] = ee;
            } else {
                atomicOr(overflow, 1u);
            }
        }
    }
}

// ranges[t] = [first, last + 1) of tile t in the sorted keys: two binary
// searches (first key with tile >= t, first with tile >= t + 1) per tile, one
// thread per tile.  An empty tile gets [s, s) with s where its keys would
// start, so starts are the cumulative list lengths in tile order.  The last
// key (the largest) must name a valid tile, else *overflow gets bit 2.
template <typename K>
__device__ inline uint64_t lower_bound_tile(const K* __restrict__ keys, uint64_t n, int shift, uint32_t t) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if ((uint32_t)(keys[mid] >> shift) < t) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <typename K>
__global__ void __launch_bounds__(256)
k_ranges(const K* __restrict__ keys, uint64_t n_cap, const uint64_t* d_n, int shift, uint2* __restrict__ ranges,
         uint32_t n_tiles, uint32_t* __restrict__ overflow) {
    uint64_t n = d_n ? *d_n : n_cap;
    if (n > n_cap) n = n_cap;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0 && n > 0 && (uint32_t)(keys[n - 1] >> shift) >= n_tiles) atomicOr(overflow, 2u);
    if (t >= n_tiles) return;
    const uint64_t a = lower_bound_tile(keys, n, shift, t);
    const uint64_t b = lower_bound_tile(keys, n, shift, t + 1);
    ranges[t] = make_uint2((uint32_t)a, (uint32_t)b);
}

}  // namespace

namespace {
unsigned emit_grid(uint64_t n_entries) {
    const uint64_t want = (n_entries + kEmitThreads - 1) / kEmitThreads;
    const uint64_t cap = (uint64_t)kSmCount * 32;   // grid-stride beyond 32 CTAs per SM
    return (unsigned)(want < cap ? want : cap);
}
}  // namespace

Status launch_emit_u32(const uint32_t* order, const uint32_t* offsets, const SplatArrays& sp,
                       const ViewParams* views, int V, uint32_t n_per_view, uint64_t n_entries, uint32_t* keys,
                       uint32_t* values, uint64_t pair_cap, uint32_t* overflow, cudaStream_t st) {
    if (n_entries == 0) return {};
    k_emit<false><<<emit_grid(n_entries), kEmitThreads, 0, st>>>(order, offsets, sp, views, V, n_per_view, n_entries,
                                                                keys, values, pair_cap, overflow);
    TIGAS_LAUNCHED();
    return {};
}

Status launch_emit_u64(const uint32_t* offsets, const SplatArrays& sp, const ViewParams* views, int V,
                       uint32_t n_per_view, uint64_t n_entries, uint64_t* keys, uint32_t* values,
                       uint64_t pair_cap, uint32_t* overflow, cudaStream_t st) {
    if (n_entries == 0) return {};
    k_emit<true><<<emit_grid(n_entries), kEmitThreads, 0, st>>>(nullptr, offsets, sp, views, V, n_per_view, n_entries,
                                                               keys, values, pair_cap, overflow);
    TIGAS_LAUNCHED();
    return {};
}

template <typename K>
Status launch_ranges(const K* keys, uint64_t n_cap, const uint64_t* d_n, int shift, uint2* ranges,
                     uint32_t n_tiles, uint32_t* overflow, cudaStream_t st) {
    if (n_tiles == 0) return {};
    dim3 grid((n_tiles + 255) / 256);
    k_ranges<K><<<grid, 256, 0, st>>>(keys, n_cap, d_n, shift, ranges, n_tiles, overflow);
    TIGAS_LAUNCHED();
    return {};
}

template Status launch_ranges<uint32_t>(const uint32_t*, uint64_t, const uint64_t*, int, uint2*, uint32_t,
                                        uint32_t*, cudaStream_t);
template Status launch_ranges<uint64_t>(const uint64_t*, uint64_t, const uint64_t*, int, uint2*, uint32_t,
                                        uint32_t*, cudaStream_t);

}  // namespace tigas
