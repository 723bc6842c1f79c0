// Depth-sliced schedule of the hot path.
//
// The per-tile blend consumes a tile's depth-ordered list front to back and
// stops once every pixel's transmittance has fallen below the threshold; in
// dense scenes that happens after a small fraction of the list.  Here the
// depth-ordered entries (all views) are cut into slices, nearest first.  Each
// slice runs the same steps as the whole frame -- count, scan, duplicate-and-
// key emit, radix sort by tile, tile ranges, blend -- but only for tiles that
// still have a pixel running, with every pixel's (C, T) carried across slices.
// Within a tile, all pairs of slice s precede those of slice s + 1 in depth
// order and the stable sort keeps depth order inside a slice, so each pixel
// composites the same entries in the same order as over the whole list: the
// frame is identical, but pairs of tiles that already stopped are never
// emitted, sorted or read.
#include "kernels.cuh"
#include "sliced.cuh"

namespace tigas {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

__device__ inline int view_of_tile(const uint32_t* s_tb, int V, uint32_t g) {
    int lo = 0, hi = V;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_tb[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

// floor(clamp(x, 0, 1) 255 + 0.5) with one rounding of the fused x 255 + 0.5
__device__ inline uint8_t to_u8(float x) {
    return (uint8_t)__float2uint_rd(__fmaf_rn(fminf(fmaxf(x, 0.0f), 1.0f), 255.0f, 0.5f));
}

// Per-launch-set clearing for the slices, a thread per tile: done bits, strip
// words (row bits: the tile's rows that stopped; kStripSeen / kStripSeenNow:
// the tile carries (C, T) from a blended slice), and the slice totals.  No pixel is touched: a tile's first
// blend starts from (C, T) = (0, 1), and k_fill_unseen writes the background
// of tiles no slice blended.
__global__ void __launch_bounds__(256)
k_init_slices(uint32_t total_tiles, uint32_t* __restrict__ done, uint32_t* __restrict__ strips,
              unsigned long long* __restrict__ totals, int n_totals, const uint32_t* __restrict__ word_src,
              uint32_t* __restrict__ word_dst) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g == 0 && word_src) *word_dst = *word_src;
    if (g < total_tiles) {
        strips[g] = 0u;
        if ((g & 31u) == 0u) done[g >> 5] = 0u;
    }
    if (g < (uint32_t)n_totals) totals[g] = 0ull;
}

// Background outputs of the tiles that no slice blended (a warp per tile).
__global__ void __launch_bounds__(256)
k_fill_unseen(const ViewParams* __restrict__ views_g, int V, uint32_t total_tiles, const uint32_t* __restrict__ strips,
              float bg_r, float bg_g, float bg_b) {
    __shared__ uint32_t s_tb[kMaxViews];
    for (int k = threadIdx.x; k < V; k += blockDim.x) s_tb[k] = views_g[k].tile_base;
    __syncthreads();
    const uint32_t g = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (g >= total_tiles) return;
    if (strips[g] & (kStripSeen | kStripSeenNow)) return;   // warp-uniform
    const int lane = threadIdx.x & 31;
    const int v = view_of_tile(s_tb, V, g);
    const ViewParams& vp = views_g[v];
    const uint32_t local = g - s_tb[v];
    const int px = (int)(local % vp.TX) * kTile + (lane & 15);
    const int ty0 = (int)(local / vp.TX) * kTile;
    const uchar4 b8 = make_uchar4(to_u8(bg_r), to_u8(bg_g), to_u8(bg_b), 0);
#pragma unroll
    for (int k = 0; k < kTile / 2; ++k) {
        const int py = ty0 + (lane >> 4) + 2 * k;
        if (px >= vp.W || py >= vp.H) continue;
        const size_t pix = (size_t)py * vp.W + px;
        if (vp.out_rgba8) reinterpret_cast<uchar4*>(vp.out_rgba8)[pix] = b8;
        if (vp.out_rgba_f32) reinterpret_cast<float4*>(vp.out_rgba_f32)[pix] = make_float4(bg_r, bg_g, bg_b, 0.f);
    }
}

__device__ inline bool tile_done(const uint32_t* __restrict__ done, uint32_t t) {
    return (done[t >> 5] >> (t & 31)) & 1u;
}

// Running-tile table of each view (one CTA per view): every row's prefix
// count of tiles not done (a warp per row, 32 columns per step, ballot and
// prefix popcount), then the prefix down every column.  Tables up to
// kSatSmem words are built in shared memory and copied out once.
constexpr uint32_t kSatSmem = 12288;   // 48 KB

__global__ void __launch_bounds__(1024)
k_running_sat(const ViewParams* __restrict__ views_g, const uint32_t* __restrict__ done, uint32_t* __restrict__ sat,
              uint32_t* __restrict__ slice_zero, int n_zero, uint32_t* __restrict__ sort_zero, int n_sort_zero) {
    __shared__ uint32_t tab[kSatSmem];
    if (blockIdx.x == 0) {
        if ((int)threadIdx.x < n_zero) slice_zero[threadIdx.x] = 0u;
        for (int i = threadIdx.x; i < n_sort_zero; i += blockDim.x) sort_zero[i] = 0u;
    }
    const ViewParams& vp = views_g[blockIdx.x];
    const uint32_t TX = (uint32_t)vp.TX, TY = (uint32_t)vp.TY, W1 = TX + 1;
    const bool in_smem = (TY + 1) * W1 <= kSatSmem;
    uint32_t* s = in_smem ? tab : sat + vp.sat_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    for (uint32_t x = threadIdx.x; x <= TX; x += blockDim.x) s[x] = 0u;
    for (uint32_t y = warp; y < TY; y += n_warps) {
        uint32_t* row = s + (y + 1) * W1;
        const uint32_t t0 = vp.tile_base + y * TX;
        if (lane == 0) row[0] = 0u;
        uint32_t carry = 0;
        for (uint32_t x0 = 0; x0 < TX; x0 += 32) {
            const uint32_t x = x0 + lane, t = t0 + x;
            const bool run = x < TX && !((done[t >> 5] >> (t & 31)) & 1u);
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, run);
            if (x < TX) row[x + 1] = carry + __popc(b & (0xFFFFFFFFu >> (31 - lane)));
            carry += __popc(b);
        }
    }
    __syncthreads();
    for (uint32_t x = threadIdx.x + 1; x <= TX; x += blockDim.x) {
        uint32_t c = 0;
        for (uint32_t y = 1; y <= TY; ++y) {
            c += s[y * W1 + x];
            s[y * W1 + x] = c;
        }
    }
    if (in_smem) {
        __syncthreads();
        uint32_t* g = sat + vp.sat_base;
        for (uint32_t i = threadIdx.x; i < (TY + 1) * W1; i += blockDim.x) g[i] = tab[i];
    }
}

// With count(k) = tiles of entry k's rectangle that are not done, for k in
// [a, b), and count(b) = 0 (the closing zero): inblock[k - a] = the sum of
// count over the entries of k's block (kScanBlock consecutive entries) before
// k, and sums[j] = block j's total.  An entry's pair offset is then its
// block's offset (an exclusive scan of sums) plus inblock, so no pass over
// the counts follows (measured against writing the counts and scanning them
// in a separate pass: scan stage 0.256 -> 0.231 ms, emit 0.262 -> 0.275 ms
// per 8-view launch set).  One CTA per block.
template <bool COMPACT, int kCountThreads>
__global__ void __launch_bounds__(kCountThreads)
k_count_slice(const uint2* __restrict__ rect_sorted, uint64_t a, uint64_t b, const ViewParams* __restrict__ views_g,
              int V, const uint32_t* __restrict__ sat, uint32_t* __restrict__ inblock, uint32_t* __restrict__ sums,
              uint32_t* __restrict__ list, uint32_t* __restrict__ n_list, uint32_t list_cap) {
    constexpr int kCountItems = (int)kScanBlock / kCountThreads;
    constexpr int kW = kCountThreads / 32;
    __shared__ uint32_t s_sb[kMaxViews], s_w1[kMaxViews], ws[kW + 1];
    __shared__ uint32_t buf[kScanBlock + kScanBlock / 32];   // the block's counts, then their prefixes
    for (int k = threadIdx.x; k < V; k += kCountThreads) {
        s_sb[k] = views_g[k].sat_base;
        s_w1[k] = (uint32_t)views_g[k].TX + 1u;
    }
    __syncthreads();
    const uint64_t n = b - a + 1;   // with the closing zero
    const uint64_t base = (uint64_t)blockIdx.x * kScanBlock;
    auto pad = [](uint32_t i) { return i + (i >> 5); };
    // all of the thread's rectangles first (independent loads in flight), then
    // the table lookups; past the slice an empty rectangle counts 0
    uint2 rr[kCountItems];
#pragma unroll
    for (int r = 0; r < kCountItems; ++r) {
        const uint64_t i = base + (uint64_t)r * kCountThreads + threadIdx.x;
        rr[r] = i < b - a ? rect_sorted[a + i] : make_uint2(0u, 0u);
    }
#pragma unroll
    for (int r = 0; r < kCountItems; ++r) {
        const TileRect tr = unpack_rect<COMPACT>(rr[r]);
        const bool ne = tr.xhi > tr.xlo && tr.yhi > tr.ylo;
        // an empty rectangle looks up word 0 of the table (always present), so every
        // lookup is unconditional and they all go out together
        const uint32_t* s = sat + (ne ? s_sb[tr.v] : 0u);
        const uint32_t w1 = ne ? s_w1[tr.v] : 0u;
        const uint32_t xl = ne ? tr.xlo : 0u, xh = ne ? tr.xhi : 0u, yl = ne ? tr.ylo : 0u, yh = ne ? tr.yhi : 0u;
        buf[pad((uint32_t)(r * kCountThreads) + threadIdx.x)] =
            s[yh * w1 + xh] - s[yl * w1 + xh] - s[yh * w1 + xl] + s[yl * w1 + xl];
    }
    __syncthreads();
    // the block's exclusive prefix: each thread scans kCountItems consecutive
    // counts, the threads' totals are scanned across the block
    uint32_t v[kCountItems];
    uint32_t tsum = 0, nzmask = 0;   // nzmask bit q: the thread's entry q has pairs
    static_assert(kCountItems <= 32, "one mask bit per entry of the thread");
#pragma unroll
    for (int q = 0; q < kCountItems; ++q) {
        v[q] = buf[pad(threadIdx.x * kCountItems + q)];
        tsum += v[q];
        nzmask |= (v[q] > 0u ? 1u : 0u) << q;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = tsum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = lane < kW ? ws[lane] : 0u;
        uint32_t wi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < kW) ws[lane] = wi - x;   // exclusive warp offsets
        if (lane == kW - 1) ws[kW] = wi;     // the block's total
    }
    __syncthreads();
    uint32_t off = ws[warp] + incl - tsum;
#pragma unroll
    for (int q = 0; q < kCountItems; ++q) {
        buf[pad(threadIdx.x * kCountItems + q)] = off;
        off += v[q];
    }
    if (list) {
        // the block's entries with pairs, appended to the list (blocks in any order,
        // each block's in entry order): the emit then visits those alone
        const uint32_t nz = __popc(nzmask);
        uint32_t zi = nz;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, zi, d);
            if (lane >= d) zi += y;
        }
        __shared__ uint32_t zs[kW + 1];
        if (lane == 31) zs[warp] = zi;
        __syncthreads();
        if (warp == 0) {
            const uint32_t x = lane < kW ? zs[lane] : 0u;
            uint32_t wi = x;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, wi, d);
                if (lane >= d) wi += y;
            }
            if (lane < kW) zs[lane] = wi - x;
            if (lane == kW - 1) zs[kW] = wi ? atomicAdd(n_list, wi) : 0u;   // the block's first list slot
        }
        __syncthreads();
        uint32_t at = zs[kW] + zs[warp] + zi - nz;
        for (uint32_t m = nzmask; m; m &= m - 1u, ++at)
            if (at < list_cap) list[at] = (uint32_t)(base + (uint64_t)threadIdx.x * kCountItems + (__ffs(m) - 1));
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kCountItems; ++r) {
        const uint64_t i = base + (uint64_t)r * kCountThreads + threadIdx.x;
        if (i < n) inblock[i] = buf[pad((uint32_t)(r * kCountThreads) + threadIdx.x)];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = ws[kW];
}

// Pairs (tile, entry) of the slice for tiles not done, in depth order: entry
// k's pairs from its pair offset pos on, its live tiles in row-major order.  The
// warp writes the pairs of its 32 entries (m: the lanes whose entry has
// pairs; r, e, pos: each lane's rectangle, entry and first pair position)
// with its lanes spread over the tiles of several entries at once: the
// rectangles are laid end to end (an exclusive prefix of their areas), lane
// l takes tile slot f0 + l of that sequence, finds its entry by a binary
// search over the lanes' prefixes, and ranks its tile among the live tiles of
// the same entry (the ballot bits of that entry's lanes in the step, plus the
// live tiles the entry had in earlier steps).  Stores stay coalesced, and
// entries of a few tiles share a step instead of taking one each (measured
// against one entry per step: emit 0.300 -> 0.261 ms per 8-view launch set).
// WIDE: 64-bit keys (tile << 32 | dk), dk the lane's entry's depth key minus
// the smallest kept one, for a slice whose entries are not in depth order.
template <bool COMPACT, bool WIDE>
__device__ inline void emit_warp_segmented(uint32_t m, uint2 r, uint32_t e, uint32_t pos, uint32_t dk,
                                           const uint32_t* s_tb, const uint32_t* s_tx,
                                           const uint32_t* __restrict__ done, uint32_t* __restrict__ keys,
                                           uint32_t* __restrict__ values, uint64_t pair_cap,
                                           uint32_t* __restrict__ overflow) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const TileRect tr = unpack_rect<COMPACT>(r);
    const bool has = (m >> lane) & 1u;
    const uint32_t w = has ? tr.xhi - tr.xlo : 1u;
    const uint32_t area = has ? w * (tr.yhi - tr.ylo) : 0u;
    const uint32_t tx = s_tx[has ? tr.v : 0u];
    const uint32_t t0 = s_tb[has ? tr.v : 0u] + tr.ylo * tx + tr.xlo;
    const float rinv = __fdividef(1.0f, (float)w);   // approximate: the row estimate is corrected below
    uint32_t incl = area;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    const uint32_t pre = incl - area;
    const uint32_t A = __shfl_sync(kFull, incl, 31);
    uint32_t carry = 0;   // live tiles of the step's first entry in the steps before
    for (uint32_t f0 = 0; f0 < A; f0 += 32) {
        const uint32_t f = f0 + (uint32_t)lane;
        int j = 0;   // the last lane whose prefix is <= f
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t pj = __shfl_sync(kFull, pre, j + step);
            if (pj <= f) j += step;
        }
        const uint32_t pj = __shfl_sync(kFull, pre, j), wj = __shfl_sync(kFull, w, j);
        const uint32_t txj = __shfl_sync(kFull, tx, j), t0j = __shfl_sync(kFull, t0, j);
        const uint32_t posj = __shfl_sync(kFull, pos, j), ej = __shfl_sync(kFull, e, j);
        const uint32_t dkj = WIDE ? __shfl_sync(kFull, dk, j) : 0u;
        const float rj = __shfl_sync(kFull, rinv, j);
        const bool valid = f < A;
        const uint32_t local = valid ? f - pj : 0u;
        uint32_t row = (uint32_t)((float)local * rj);   // local / wj, corrected (local < 2^20)
        if (row * wj > local) --row;
        else if ((row + 1u) * wj <= local) ++row;
        const uint32_t t = t0j + row * txj + (local - row * wj);
        const bool live = valid && !((done[t >> 5] >> (t & 31)) & 1u);
        const uint32_t bm = __ballot_sync(kFull, live);
        const uint32_t first = pj > f0 ? pj - f0 : 0u;   // the step's first lane of entry j
        const uint32_t rank = __popc(bm & lt & ~((1u << first) - 1u)) + (pj < f0 ? carry : 0u);
        if (live) {
            const uint64_t p = (uint64_t)posj + rank;
            if (p < pair_cap) {
                if (WIDE)
                    reinterpret_cast<uint2*>(keys)[p] = make_uint2(dkj, t);
                else
                    keys[p] = t;
                values[p] = ej;
            } else {
                atomicOr(overflow, 1u);
            }
        }
        carry = __shfl_sync(kFull, rank + (live ? 1u : 0u), 31);
    }
}

// Each warp takes 32 J consecutive entries, lane l the entries 32 j + l: all
// of its pair offsets are loaded at once (entry k's offset is
// block_offs[(k - a) / kScanBlock] + inblock[k - a]; its count is the next
// entry's offset minus its own, and the offset of b is the slice total), then
// its rectangles, then the entries with pairs are written group by group.  A
// larger J launches fewer CTAs for slices of many entries whose tiles have
// mostly stopped.  COMPACT: the entry id travels in the rectangle's second
// word (order unused).  WIDE: 64-bit (tile, depth) keys (depth_key: the keys
// in entry order, key_range[0] their smallest kept value).
constexpr int kEmitThreads = 256;
#ifndef TIGAS_COUNT_BIG
#define TIGAS_COUNT_BIG 2   // a count of fewer than this many blocks per SM takes 1024-thread CTAs
#endif
#ifndef TIGAS_EMIT_WAVES
#define TIGAS_EMIT_WAVES 4   // waves of 8 CTAs per SM an emit keeps when it takes more entries per lane
#endif
#ifndef TIGAS_LIST_CTAS
#define TIGAS_LIST_CTAS 8
#endif
template <bool COMPACT, int J, bool WIDE>
__global__ void __launch_bounds__(kEmitThreads)
k_emit_slice(const uint32_t* __restrict__ order, const uint2* __restrict__ rect_sorted, uint64_t a, uint64_t b,
             const uint32_t* __restrict__ inblock, const uint32_t* __restrict__ block_offs,
             const ViewParams* __restrict__ views_g, int V,
             const uint32_t* __restrict__ done, uint32_t* __restrict__ keys, uint32_t* __restrict__ values,
             uint64_t pair_cap, uint32_t* __restrict__ overflow, const uint32_t* __restrict__ depth_key,
             const uint32_t* __restrict__ key_range) {
    __shared__ uint32_t s_tb[kMaxViews], s_tx[kMaxViews];
    for (int k = threadIdx.x; k < V; k += blockDim.x) {
        s_tb[k] = views_g[k].tile_base;
        s_tx[k] = (uint32_t)views_g[k].TX;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t wbase = a + ((uint64_t)blockIdx.x * (kEmitThreads / 32) + warp) * (32u * J);
    if (wbase >= b) return;   // warp-uniform
    uint32_t pos[J], cnt[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const uint64_t k = wbase + 32u * j + lane;
        pos[j] = k <= b ? block_offs[(k - a) / kScanBlock] + inblock[k - a] : 0u;
    }
    const uint64_t kend = wbase + 32u * J;
    const uint32_t tail = kend <= b ? block_offs[(kend - a) / kScanBlock] + inblock[kend - a] : 0u;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const uint32_t up = __shfl_down_sync(kFull, pos[j], 1);
        const uint32_t first = __shfl_sync(kFull, pos[j + 1 < J ? j + 1 : j], 0);
        const uint32_t next = lane < 31 ? up : (j + 1 < J ? first : tail);
        cnt[j] = wbase + 32u * j + lane < b ? next - pos[j] : 0u;
    }
    uint2 rr[J];
    uint32_t ee[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const uint64_t k = wbase + 32u * j + lane;
        rr[j] = cnt[j] > 0 ? rect_sorted[k] : make_uint2(0u, 0u);
        ee[j] = COMPACT ? rr[j].y : (cnt[j] > 0 ? order[k] : 0u);
    }
    uint32_t dk[J];
    const uint32_t kmin = WIDE ? key_range[0] : 0u;
#pragma unroll
    for (int j = 0; j < J; ++j) dk[j] = WIDE && cnt[j] > 0 ? depth_key[ee[j]] - kmin : 0u;
#pragma unroll
    for (int j = 0; j < J; ++j) {   // unrolled: the per-lane arrays stay in registers
        const uint32_t m = __ballot_sync(kFull, cnt[j] > 0);
        if (m)
            emit_warp_segmented<COMPACT, WIDE>(m, rr[j], ee[j], pos[j], dk[j], s_tb, s_tx, done, keys, values,
                                               pair_cap, overflow);
    }
}

// The same pairs from the list of the slice's entries with pairs (entry
// indices relative to a, n_list of them, in any order): persistent warps take
// 32 list entries at a time.  For a late slice, whose entries mostly meet only
// stopped tiles, this visits the few with pairs instead of every entry.
template <bool COMPACT, bool WIDE>
__global__ void __launch_bounds__(kEmitThreads)
k_emit_list(const uint32_t* __restrict__ order, const uint2* __restrict__ rect_sorted, uint64_t a,
            const uint32_t* __restrict__ inblock, const uint32_t* __restrict__ block_offs,
            const uint32_t* __restrict__ list, const uint32_t* __restrict__ n_list, uint32_t list_cap,
            const ViewParams* __restrict__ views_g, int V, const uint32_t* __restrict__ done,
            uint32_t* __restrict__ keys, uint32_t* __restrict__ values, uint64_t pair_cap,
            uint32_t* __restrict__ overflow, const uint32_t* __restrict__ depth_key,
            const uint32_t* __restrict__ key_range) {
    __shared__ uint32_t s_tb[kMaxViews], s_tx[kMaxViews];
    for (int k = threadIdx.x; k < V; k += blockDim.x) {
        s_tb[k] = views_g[k].tile_base;
        s_tx[k] = (uint32_t)views_g[k].TX;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n_all = *n_list, n = min(n_all, list_cap);
    // a list that outgrew its capacity (more entries with pairs than pair slots) left
    // entries out: the pair buffers overflowed too, and the frame is rendered again
    if (n_all > list_cap && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(overflow, 1u);
    const uint32_t kmin = WIDE ? key_range[0] : 0u;
    const uint64_t stride = (uint64_t)gridDim.x * kEmitThreads;
    for (uint64_t w = ((uint64_t)blockIdx.x * (kEmitThreads / 32) + warp) * 32u; w < n; w += stride) {
        const uint64_t li = w + lane;
        uint32_t pos = 0, cnt = 0, ee = 0, dk = 0;
        uint2 rr = make_uint2(0u, 0u);
        if (li < n) {
            const uint32_t k = list[li];   // its count's successor k + 1 is at most the closing zero
            pos = block_offs[k / kScanBlock] + inblock[k];
            cnt = block_offs[(k + 1u) / kScanBlock] + inblock[k + 1u] - pos;
            rr = rect_sorted[a + k];
            ee = COMPACT ? rr.y : order[a + k];
            if (WIDE) dk = depth_key[ee] - kmin;
        }
        const uint32_t m = __ballot_sync(kFull, cnt > 0u);
        if (m)
            emit_warp_segmented<COMPACT, WIDE>(m, rr, ee, pos, dk, s_tb, s_tx, done, keys, values, pair_cap,
                                               overflow);
    }
}

// Tile ranges of the sorted pair keys.  A CTA takes the 256 tiles
// [256 h, 256 h + 256); their keys form one run [L, R) of the sorted array,
// which the sort's second pass already located (its digit is t >> 8: L and R
// are that digit's base and the next one's), else two searches find it.  The
// CTA samples kRangeSample keys of the run into shared memory, and each thread's
// lower bound of its tile searches the sample first and the keys between two
// samples after, about 5 dependent reads instead of a search of the whole
// array.  Tiles with pairs in this slice that are not done form the active
// list.  A tile with at least kHeavyTile pairs goes in as its strips of pixel
// rows, so that several warps share its long list: strips of the tiles with
// at least kLongestTile pairs from the front (count n_active[0]; four 4-row
// strips for a list of at least fine_min pairs, else two 8-row strips), the
// others' two 8-row strips from the middle downward (count
// n_active[3]).  The remaining tiles go in whole from the back (count
// n_active[1]).  The blend's dynamic scheduler takes the three regions in
// that order, so the longest lists start first and the short ones fill the
// tail.
// KS: words per key (1: 32-bit tile keys; 2: the high words of 64-bit
// (tile, depth) keys, `keys` pointing at the first key's high word).
template <int KS>
__device__ inline uint64_t lower_bound_u32(const uint32_t* __restrict__ keys, uint64_t lo, uint64_t hi, uint32_t t) {
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (keys[KS * mid] < t) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// keys sampled per run of 256 tiles before the exact search (ranges stage
// 0.0724 / 0.0703 / 0.0697 ms per 8-view launch set at 1024 / 512 / 256; 2048:
// 0.082): the sample's loads weigh more than the longer search they save
#ifndef TIGAS_RANGE_SAMPLE
#define TIGAS_RANGE_SAMPLE 256
#endif
constexpr int kRangeSample = TIGAS_RANGE_SAMPLE;
template <int KS>
__global__ void __launch_bounds__(256)
k_ranges_active(const uint32_t* __restrict__ keys, uint64_t n_cap, const uint64_t* d_n, uint2* __restrict__ ranges,
                uint32_t n_tiles, const uint32_t* __restrict__ done, uint32_t* __restrict__ active,
                uint32_t* __restrict__ n_active, uint32_t* __restrict__ overflow,
                const uint32_t* __restrict__ hi_bases, uint32_t* __restrict__ strips, uint32_t fine_min) {
    __shared__ uint32_t s_sample[kRangeSample];
    __shared__ uint32_t s_lo[256];
    __shared__ uint64_t s_run[2];
    uint64_t n = d_n ? *d_n : n_cap;
    if (n > n_cap) n = n_cap;
    const uint32_t t0 = blockIdx.x * 256u, t = t0 + threadIdx.x;
    if (t < n_tiles) {
        // the previous blend is over: what it marked as seen now is seen before this slice
        const uint32_t w = strips[t];
        if (w & kStripSeenNow) strips[t] = (w & ~kStripSeenNow) | kStripSeen;
    }
    if (t == 0 && n > 0 && keys[KS * (n - 1)] >= n_tiles) atomicOr(overflow, 2u);
    if (threadIdx.x < 2) {
        uint64_t x;
        if (hi_bases) {
            const uint32_t h = blockIdx.x + threadIdx.x;   // h <= 256: tile ids have at most 16 bits
            x = h < 256u ? hi_bases[h] : n;
            if (x > n) x = n;
        } else {
            x = lower_bound_u32<KS>(keys, 0, n, t0 + 256u * threadIdx.x);
        }
        s_run[threadIdx.x] = x;
    }
    __syncthreads();
    const uint64_t L = s_run[0], R = s_run[1] > L ? s_run[1] : L, span = R - L;
    for (int k = threadIdx.x; k < kRangeSample; k += 256)
        s_sample[k] = span ? keys[KS * (L + (uint64_t)k * span / kRangeSample)] : 0xFFFFFFFFu;
    __syncthreads();
    {
        // first sample >= t, then the keys after the sample before it
        int lo = 0, hi = kRangeSample;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_sample[mid] < t) lo = mid + 1; else hi = mid;
        }
        const uint64_t a = lo == 0 ? L : L + (uint64_t)(lo - 1) * span / kRangeSample + 1;
        const uint64_t b = lo == kRangeSample ? R : L + (uint64_t)lo * span / kRangeSample;
        s_lo[threadIdx.x] = (uint32_t)lower_bound_u32<KS>(keys, a, b, t);
    }
    __syncthreads();
    bool act = false, heavy = false, longest = false;
    uint32_t lens = 0;
    if (t < n_tiles) {
        const uint32_t lo = s_lo[threadIdx.x];
        const uint32_t hi = threadIdx.x < 255 ? s_lo[threadIdx.x + 1] : (uint32_t)R;
        ranges[t] = make_uint2(lo, hi);
        act = hi > lo && !tile_done(done, t);
        lens = hi - lo;
        heavy = act && lens >= kHeavyTile;
        longest = heavy && lens >= kLongestTile;
    }
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    // strips of the longest lists from the front, of the other long lists from the
    // middle (6 n_tiles) down, so that the blend starts the longest work first
    const uint32_t mx = __ballot_sync(kFull, longest);
    const uint32_t mh = __ballot_sync(kFull, heavy && !longest);
    const uint32_t ml = __ballot_sync(kFull, act && !heavy);
    if (mx) {
        // four 4-row strips for a list of at least fine_min pairs, else two 8-row ones
        const uint32_t rows = longest && lens >= fine_min ? 4u : 8u;
        const uint32_t ns = longest ? 16u / rows : 0u;
        uint32_t incl = ns;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        uint32_t base = 0;
        if (lane == 31) base = atomicAdd(&n_active[0], incl);
        base = __shfl_sync(kFull, base, 31);
        if (longest) {
            const uint32_t at = base + incl - ns;
            for (uint32_t s = 0; s < ns; ++s) active[at + s] = t | (strip_code(rows, s) << kStripShift);
        }
    }
    if (mh) {
        uint32_t base = 0;
        if (lane == __ffs(mh) - 1) base = atomicAdd(&n_active[3], 2u * (uint32_t)__popc(mh));
        base = __shfl_sync(kFull, base, __ffs(mh) - 1);
        if (heavy && !longest) {
            const uint32_t at = base + 2u * (uint32_t)__popc(mh & below);
#pragma unroll
            for (uint32_t s = 0; s < 2u; ++s)
                active[6u * n_tiles - 1u - (at + s)] = t | (strip_code(8, s) << kStripShift);
        }
    }
    if (ml) {
        uint32_t base = 0;
        if (lane == __ffs(ml) - 1) base = atomicAdd(&n_active[1], (uint32_t)__popc(ml));
        base = __shfl_sync(kFull, base, __ffs(ml) - 1);
        if (act && !heavy) active[kActivePerTile * n_tiles - 1u - (base + __popc(ml & below))] = t;
    }
}

}  // namespace

Status launch_init_slices(uint32_t total_tiles, uint32_t* done, uint32_t* strips, uint64_t* totals, int n_totals,
                          const uint32_t* word_src, uint32_t* word_dst, cudaStream_t st) {
    if (n_totals > 256) return {TIGAS_ERR_INVALID, "too many slice totals"};
    const uint32_t n = total_tiles > (uint32_t)n_totals ? total_tiles : (uint32_t)n_totals;
    if (n == 0) return {};
    k_init_slices<<<(n + 255) / 256, 256, 0, st>>>(total_tiles, done, strips,
                                                   reinterpret_cast<unsigned long long*>(totals), n_totals, word_src,
                                                   word_dst);
    TIGAS_LAUNCHED();
    return {};
}

Status launch_fill_unseen(const ViewParams* views, int V, uint32_t total_tiles, const uint32_t* strips,
                          const float* bg, cudaStream_t st) {
    if (total_tiles == 0) return {};
    k_fill_unseen<<<(total_tiles + 7) / 8, 256, 0, st>>>(views, V, total_tiles, strips, bg[0], bg[1], bg[2]);
    TIGAS_LAUNCHED();
    return {};
}

Status launch_running_sat(const ViewParams* views, int V, const uint32_t* done, uint32_t* sat, uint32_t* slice_zero,
                          int n_zero, uint32_t* sort_zero, int n_sort_zero, cudaStream_t st) {
    if (n_zero > 1024) return {TIGAS_ERR_INVALID, "too many words to clear"};
    k_running_sat<<<V, 1024, 0, st>>>(views, done, sat, slice_zero, n_zero, sort_zero, sort_zero ? n_sort_zero : 0);
    TIGAS_LAUNCHED();
    return {};
}

Status launch_count_slice(const uint2* rect_sorted, uint64_t a, uint64_t b, const ViewParams* views, int V,
                          const uint32_t* sat, uint32_t* inblock, uint32_t* sums, bool compact, uint32_t* list,
                          uint32_t* n_list, uint64_t list_cap, cudaStream_t st) {
    if (b <= a) return {};
    if (list && !n_list) return {TIGAS_ERR_INVALID, "an entry list needs its counter"};
    const uint32_t lc = (uint32_t)(list_cap < 0xFFFFFFFFull ? list_cap : 0xFFFFFFFFull);
    const unsigned grid = (unsigned)((b - a + 1 + kScanBlock - 1) / kScanBlock);
    // a slice of few blocks (less than two per SM) takes 1024 threads per block,
    // 4 rectangles each, so that its few CTAs hold more warps
    const bool big = grid < (unsigned)TIGAS_COUNT_BIG * (unsigned)kSmCount;
    if (compact) {
        if (big)
            k_count_slice<true, 1024><<<grid, 1024, 0, st>>>(rect_sorted, a, b, views, V, sat, inblock, sums, list,
                                                             n_list, lc);
        else
            k_count_slice<true, 256><<<grid, 256, 0, st>>>(rect_sorted, a, b, views, V, sat, inblock, sums, list,
                                                           n_list, lc);
    } else {
        if (big)
            k_count_slice<false, 1024><<<grid, 1024, 0, st>>>(rect_sorted, a, b, views, V, sat, inblock, sums, list,
                                                              n_list, lc);
        else
            k_count_slice<false, 256><<<grid, 256, 0, st>>>(rect_sorted, a, b, views, V, sat, inblock, sums, list,
                                                            n_list, lc);
    }
    TIGAS_LAUNCHED();
    return {};
}

Status launch_emit_slice(const uint32_t* order, const uint2* rect_sorted, uint64_t a, uint64_t b,
                         const uint32_t* inblock, const uint32_t* block_offs, const ViewParams* views, int V,
                         const uint32_t* done,
                         uint32_t* keys, uint32_t* values, uint64_t pair_cap, uint32_t* overflow, bool compact,
                         const uint32_t* wide_depth, const uint32_t* key_range, const uint32_t* list,
                         const uint32_t* n_list, uint64_t list_cap, cudaStream_t st) {
    if (b <= a) return {};
    if (wide_depth && (!key_range || (reinterpret_cast<uintptr_t>(keys) & 7u)))
        return {TIGAS_ERR_INVALID, "wide emit needs the key range and 8-byte aligned keys"};
    if (list) {
        if (!n_list) return {TIGAS_ERR_INVALID, "an entry list needs its counter"};
        const uint32_t lc = (uint32_t)(list_cap < 0xFFFFFFFFull ? list_cap : 0xFFFFFFFFull);
        // persistent warps over the list, at most TIGAS_LIST_CTAS CTAs per SM
        const uint64_t most = (b - a + kEmitThreads - 1) / kEmitThreads;
        const unsigned grid = (unsigned)(most < (uint64_t)TIGAS_LIST_CTAS * kSmCount ? most : TIGAS_LIST_CTAS * kSmCount);
#define TIGAS_EMIT_LIST(CC, WW)                                                                                 \
    k_emit_list<CC, WW><<<grid, kEmitThreads, 0, st>>>(order, rect_sorted, a, inblock, block_offs, list, n_list, \
                                                       lc, views, V, done, keys, values, pair_cap, overflow,     \
                                                       wide_depth, key_range)
        if (compact) {
            if (wide_depth) TIGAS_EMIT_LIST(true, true);
            else TIGAS_EMIT_LIST(true, false);
        } else {
            if (wide_depth) TIGAS_EMIT_LIST(false, true);
            else TIGAS_EMIT_LIST(false, false);
        }
#undef TIGAS_EMIT_LIST
        TIGAS_LAUNCHED();
        return {};
    }
    // entries per lane: the largest J in {1, 2, 4, 8} that still leaves about
    // 4 waves of 8 CTAs per SM (slices with many pairs per entry want the warps)
    const uint64_t n = b - a;
    int J = 1;
    while (J < 8 && n >= (uint64_t)(2 * J) * kEmitThreads * kSmCount * 8 * TIGAS_EMIT_WAVES) J *= 2;
    const unsigned grid = (unsigned)((n + (uint64_t)J * kEmitThreads - 1) / ((uint64_t)J * kEmitThreads));
#define TIGAS_EMIT2(CC, JJ)                                                                                       \
    do {                                                                                                          \
        if (wide_depth)                                                                                           \
            k_emit_slice<CC, JJ, true><<<grid, kEmitThreads, 0, st>>>(order, rect_sorted, a, b, inblock,           \
                                                                      block_offs, views, V, done, keys, values,   \
                                                                      pair_cap, overflow, wide_depth, key_range); \
        else                                                                                                      \
            k_emit_slice<CC, JJ, false><<<grid, kEmitThreads, 0, st>>>(order, rect_sorted, a, b, inblock,          \
                                                                       block_offs, views, V, done, keys, values,  \
                                                                       pair_cap, overflow, nullptr, nullptr);     \
    } while (0)
#define TIGAS_EMIT(JJ)                \
    do {                              \
        if (compact)                  \
            TIGAS_EMIT2(true, JJ);    \
        else                          \
            TIGAS_EMIT2(false, JJ);   \
    } while (0)
    switch (J) {
        case 1: TIGAS_EMIT(1); break;
        case 2: TIGAS_EMIT(2); break;
        case 4: TIGAS_EMIT(4); break;
        default: TIGAS_EMIT(8); break;
    }
#undef TIGAS_EMIT
#undef TIGAS_EMIT2
    TIGAS_LAUNCHED();
    return {};
}

Status launch_ranges_active(const uint32_t* keys, uint64_t n_cap, const uint64_t* d_n, uint2* ranges,
                            uint32_t n_tiles, const uint32_t* done, uint32_t* active, uint32_t* n_active,
                            uint32_t* overflow, const uint32_t* hi_bases, uint32_t* strips, bool wide,
                            uint32_t fine_min, cudaStream_t st) {
    if (n_tiles == 0) return {};
    static_assert(kActivePerTile == 7, "4 + 2 + 1 items per tile at most, one region each");
    if (hi_bases && n_tiles > 65536u) return {TIGAS_ERR_INVALID, "second-pass digit bases need tile ids of 16 bits"};
    if (wide)   // the tile is the high word of each 64-bit key
        k_ranges_active<2><<<(n_tiles + 255) / 256, 256, 0, st>>>(keys + 1, n_cap, d_n, ranges, n_tiles, done,
                                                                  active, n_active, overflow, hi_bases, strips,
                                                                  fine_min);
    else
        k_ranges_active<1><<<(n_tiles + 255) / 256, 256, 0, st>>>(keys, n_cap, d_n, ranges, n_tiles, done, active,
                                                                  n_active, overflow, hi_bases, strips,
                                                                  fine_min);
    TIGAS_LAUNCHED();
    return {};
}

}  // namespace tigas
