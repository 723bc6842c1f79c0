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

template <bool WIDE>
__global__ void __launch_bounds__(256)
k_emit(const uint32_t* __restrict__ order, const uint32_t* __restrict__ offsets, SplatArrays sp,
       const ViewParams* __restrict__ views_g, int V, uint32_t n_per_view, uint64_t n_entries,
       void* __restrict__ keys_out, uint32_t* __restrict__ values, uint64_t pair_cap,
       uint32_t* __restrict__ overflow) {
    __shared__ ViewTiles vt[kMaxViews];
    __shared__ uint32_t s_excl[8][32];
    __shared__ uint32_t s_e[8][32];
    __shared__ uint2 s_rect[8][32];
    for (int k = threadIdx.x; k < V; k += blockDim.x) vt[k] = {views_g[k].tile_base, (uint32_t)views_g[k].TX};
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t e = 0, cnt = 0, off = 0;
    uint2 rect = make_uint2(0, 0);
    if (k < n_entries) {
        e = order ? order[k] : (uint32_t)k;
        cnt = sp.tiles[e];
        off = offsets[k];
        if (cnt) rect = sp.rect[e];
    }
    uint32_t inc = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += y;
    }
    const uint32_t total = __shfl_sync(kFull, inc, 31);
    const uint32_t gbase = __shfl_sync(kFull, off, 0);
    if (total == 0) return;   // warp-uniform
    s_excl[warp][lane] = inc - cnt;
    s_e[warp][lane] = e;
    s_rect[warp][lane] = rect;
    __syncwarp();
    for (uint32_t j = lane; j < total; j += 32) {
        // owner: last lane whose exclusive count is <= j (steps keep lo + step <= 31)
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (s_excl[warp][lo + step] <= j) lo += step;
        const uint32_t t = j - s_excl[warp][lo];
        const uint32_t ee = s_e[warp][lo];
        const uint2 r = s_rect[warp][lo];
        const uint32_t xlo = r.x & 0xFFFFu, ylo = r.x >> 16, xhi = r.y & 0xFFFFu;
        const uint32_t w = xhi - xlo;
        const uint32_t ty = ylo + t / w, tx = xlo + t % w;
        const uint32_t v = ee / n_per_view;
        const uint32_t tile = vt[v].tile_base + ty * vt[v].TX + tx;
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

// ranges[t] = [first, last + 1) of tile t in the sorted keys; an empty tile
// gets [s, s) with s the position where its keys would start, so starts are
// the cumulative list lengths in tile order.  A thread at a key change from
// tile a to tile b also fills the empty tiles a+1 .. b-1.
template <typename K>
__global__ void __launch_bounds__(256)
k_ranges(const K* __restrict__ keys, uint64_t n_cap, const uint64_t* d_n, int shift, uint2* __restrict__ ranges,
         uint32_t n_tiles, uint32_t* __restrict__ overflow) {
    uint64_t n = d_n ? *d_n : n_cap;
    if (n > n_cap) n = n_cap;
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = (uint32_t)(keys[i] >> shift);
    if (t >= n_tiles) {
        atomicOr(overflow, 2u);
        return;
    }
    const uint32_t prev = i == 0 ? 0xFFFFFFFFu : (uint32_t)(keys[i - 1] >> shift);
    if (prev != t) {
        ranges[t].x = (uint32_t)i;
        const uint32_t first_gap = i == 0 ? 0u : prev + 1;
        for (uint32_t e = first_gap; e < t && e < n_tiles; ++e) ranges[e] = make_uint2((uint32_t)i, (uint32_t)i);
    }
    if (i == n - 1) {
        ranges[t].y = (uint32_t)n;
        for (uint32_t e = t + 1; e < n_tiles; ++e) ranges[e] = make_uint2((uint32_t)n, (uint32_t)n);
    } else if ((uint32_t)(keys[i + 1] >> shift) != t) {
        ranges[t].y = (uint32_t)(i + 1);
    }
}

}  // namespace

Status launch_emit_u32(const uint32_t* order, const uint32_t* offsets, const SplatArrays& sp,
                       const ViewParams* views, int V, uint32_t n_per_view, uint64_t n_entries, uint32_t* keys,
                       uint32_t* values, uint64_t pair_cap, uint32_t* overflow, cudaStream_t st) {
    if (n_entries == 0) return {};
    dim3 grid((unsigned)((n_entries + 255) / 256));
    k_emit<false><<<grid, 256, 0, st>>>(order, offsets, sp, views, V, n_per_view, n_entries, keys, values,
                                        pair_cap, overflow);
    TIGAS_LAUNCHED();
    return {};
}

Status launch_emit_u64(const uint32_t* offsets, const SplatArrays& sp, const ViewParams* views, int V,
                       uint32_t n_per_view, uint64_t n_entries, uint64_t* keys, uint32_t* values,
                       uint64_t pair_cap, uint32_t* overflow, cudaStream_t st) {
    if (n_entries == 0) return {};
    dim3 grid((unsigned)((n_entries + 255) / 256));
    k_emit<true><<<grid, 256, 0, st>>>(nullptr, offsets, sp, views, V, n_per_view, n_entries, keys, values,
                                       pair_cap, overflow);
    TIGAS_LAUNCHED();
    return {};
}

template <typename K>
Status launch_ranges(const K* keys, uint64_t n_cap, const uint64_t* d_n, int shift, uint2* ranges,
                     uint32_t n_tiles, uint32_t* overflow, cudaStream_t st) {
    TIGAS_CUDA_TRY(cudaMemsetAsync(ranges, 0, sizeof(uint2) * n_tiles, st));
    if (n_cap == 0) return {};
    dim3 grid((unsigned)((n_cap + 255) / 256));
    k_ranges<K><<<grid, 256, 0, st>>>(keys, n_cap, d_n, shift, ranges, n_tiles, overflow);
    TIGAS_LAUNCHED();
    return {};
}

template Status launch_ranges<uint32_t>(const uint32_t*, uint64_t, const uint64_t*, int, uint2*, uint32_t,
                                        uint32_t*, cudaStream_t);
template Status launch_ranges<uint64_t>(const uint64_t*, uint64_t, const uint64_t*, int, uint2*, uint32_t,
                                        uint32_t*, cudaStream_t);

}  // namespace tigas
