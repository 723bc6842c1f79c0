// Launch interface of the depth-sliced schedule (see sliced.cu).
#pragma once

#include "common.cuh"

namespace tigas {

#ifndef TIGAS_HEAVY_TILE
#define TIGAS_HEAVY_TILE 128
#endif
constexpr uint32_t kHeavyTile = TIGAS_HEAVY_TILE;   // pairs of a slice that make a tile "long"
#ifndef TIGAS_LONGEST_TILE
#define TIGAS_LONGEST_TILE 512
#endif
constexpr uint32_t kLongestTile = TIGAS_LONGEST_TILE;   // long tiles whose strips the blend starts first
// A long tile is composited as strips of pixel rows, each a separate item of
// the active list: two strips of 8 rows, or, for the longest tiles of a slice
// whose tail their serial compositing sets, four strips of 4 rows.
// Active-list items: a tile id (whole tile) or tile id | code << kStripShift,
// code 1 + s for 8-row strip s (rows 8 s .. 8 s + 7), code 3 + s for 4-row
// strip s (rows 4 s .. 4 s + 3).
constexpr int kStripShift = 28;
constexpr uint32_t kCode8 = 1u, kCode4 = 3u;
__host__ __device__ constexpr uint32_t strip_code(uint32_t rows, uint32_t s) { return (rows == 8 ? kCode8 : kCode4) + s; }
// Strip-word bits.  Bits kRowShift + r: pixel row r of the tile has stopped
// (set by the strips that finish; the tile is done once all 16 are set, so
// tiles split into 8-row strips in one slice and 4-row strips in another
// stay consistent).  kStripSeen: a slice before the current one blended the
// tile, so its pixels carry (C, T) in the state.  A blend marks the tiles it
// visits with kStripSeenNow instead, never with kStripSeen: the strips of one
// tile run in the same slice on different warps, and a strip that finished
// first must not make a sibling that starts later take its first visit for a
// later one (and read state nobody wrote).  The next slice's ranges kernel,
// which runs after that blend and before the next, turns kStripSeenNow into
// kStripSeen.
constexpr uint32_t kStripSeen = 0x10u;
constexpr uint32_t kStripSeenNow = 0x20u;
constexpr int kRowShift = 8;
constexpr uint32_t kRowsAll = 0xFFFFu << kRowShift;
// The active list: 4-row strips from the front, 8-row strips from the
// middle down, whole tiles from the back (kActivePerTile words per tile).
constexpr uint32_t kActivePerTile = 7;
constexpr uint32_t kTileMask = (1u << kStripShift) - 1u;

// Clears the per-tile done bits (total_tiles bits) and strip words (row bits:
// the tile's pixel rows that stopped; kStripSeen / kStripSeenNow: the tile was
// blended and its pixels carry (C, T) in `state`; a tile's first blend starts
// from (0, 1) instead), and totals[0 .. n_totals) (at most 256).  No pixel is
// written.  Also copies *word_src to *word_dst when word_src is not null (a
// word the caller reads back with the launch set's other results, instead of
// a device-to-host copy in the middle of the launch set).
Status launch_init_slices(uint32_t total_tiles, uint32_t* done, uint32_t* strips, uint64_t* totals, int n_totals,
                          const uint32_t* word_src, uint32_t* word_dst, cudaStream_t st);

// After the last slice: the background in the outputs of every tile that no
// slice blended (kStripSeen and kStripSeenNow clear).
Status launch_fill_unseen(const ViewParams* views, int V, uint32_t total_tiles, const uint32_t* strips,
                          const float* bg, cudaStream_t st);

// Per view, the summed-area table of tiles not done: sat[sat_base + y (TX+1) + x]
// = not-done tiles in columns [0, x) of rows [0, y).  Also clears
// slice_zero[0 .. n_zero) (at most 1024 words: the slice's active-list counts
// and blend work counter, which the ranges and blend launches expect zeroed)
// and sort_zero[0 .. n_sort_zero) (null: none; the scratch words the slice's
// pair sort expects zeroed, radix_zero_words).
Status launch_running_sat(const ViewParams* views, int V, const uint32_t* done, uint32_t* sat, uint32_t* slice_zero,
                          int n_zero, uint32_t* sort_zero, int n_sort_zero, cudaStream_t st);

// count(k): not-done tiles in the rectangle of depth-ordered entry k, k in
// [a, b) (four reads of the running-tile table), and count(b) = 0.  Writes
// inblock[k - a] = the sum of count over the entries before k in k's block
// (kScanBlock consecutive entries; b - a + 1 values), and sums[j] = block j's
// total.  compact: rectangles in the compact form (SplatArrays::compact_rect).
// list (or null): appends k - a of every entry with count(k) > 0 at
// list[atomicAdd(n_list, ...)] (*n_list zero on entry; slots past list_cap
// are counted but not written).
Status launch_count_slice(const uint2* rect_sorted, uint64_t a, uint64_t b, const ViewParams* views, int V,
                          const uint32_t* sat, uint32_t* inblock, uint32_t* sums, bool compact, uint32_t* list,
                          uint32_t* n_list, uint64_t list_cap, cudaStream_t st);

// (tile, entry) pairs of entries [a, b) for tiles not done, entry k's at
// block_offs[(k - a) / kScanBlock] + inblock[k - a] (block_offs: the exclusive
// scan of the count kernel's block sums).  The entry of k is order[k], or the
// second word of a compact rectangle (order may then be null).
// wide_depth (the depth keys in entry order, key_range[0] the smallest kept
// one): keys holds 64-bit keys (tile << 32 | depth key - key_range[0]), for a
// slice whose entries are not in depth order; null: 32-bit tile keys.
// list (or null): visit only the min(*n_list, list_cap) entries the count
// kernel listed (the same pairs, fewer entries read).
Status launch_emit_slice(const uint32_t* order, const uint2* rect_sorted, uint64_t a, uint64_t b,
                         const uint32_t* inblock, const uint32_t* block_offs, const ViewParams* views, int V,
                         const uint32_t* done, uint32_t* keys, uint32_t* values, uint64_t pair_cap,
                         uint32_t* overflow, bool compact, const uint32_t* wide_depth, const uint32_t* key_range,
                         const uint32_t* list, const uint32_t* n_list, uint64_t list_cap, cudaStream_t st);

// Tile ranges of the slice's sorted keys, and the list of tiles with pairs
// that are not done, in three regions of `active` (kActivePerTile n_tiles
// items): the strips of each tile with >= kLongestTile pairs from the front
// (n_active[0] items; four 4-row strips for a tile of at least fine_min
// pairs, else two 8-row strips; 0xFFFFFFFF: never 4-row), the two 8-row
// strips of the other tiles with >= kHeavyTile pairs from active[6 n_tiles -
// 1] downward (n_active[3]), and the remaining tiles whole from the back
// (active[7 n_tiles - 1 - k], n_active[1]).  The three counts must be zero on
// entry (launch_running_sat clears them).  Also turns every strip word's
// kStripSeenNow into kStripSeen (the blend before this one is over).
// The key count is min(*d_n, n_cap) when d_n is given, else n_cap.
// hi_bases: null, or 256 words whose word h is the first position of a key
// whose tile t has t >> 8 == h (the digit bases of the pass over the tile's
// high byte in the sort that produced `keys`); n_tiles <= 65536.
// wide: keys holds 64-bit (tile << 32 | depth) keys.
Status launch_ranges_active(const uint32_t* keys, uint64_t n_cap, const uint64_t* d_n, uint2* ranges,
                            uint32_t n_tiles, const uint32_t* done, uint32_t* active, uint32_t* n_active,
                            uint32_t* overflow, const uint32_t* hi_bases, uint32_t* strips, bool wide,
                            uint32_t fine_min, cudaStream_t st);

// Blend of the active tiles of one slice: persistent CTAs take tiles from the
// active list, composite the slice's entries onto each pixel's carried state,
// store the state and the outputs, and mark tiles whose pixels all stopped.
// ctas_per_sm: persistent CTAs per SM (0 or more than fit: as many as fit).
// batch: list entries a warp stages at a time, 16 or 32.
struct SliceBlendArgs {
    const uint32_t* active;
    const uint32_t* n_active;   // [longest strips, whole tiles, (work counter), other strips]
    uint32_t* work_counter;     // zero on entry (launch_running_sat clears it)
    float4* state;              // per pixel (C.rgb, T), T negated once the pixel stopped; valid for the
                                // tiles whose strip word has kStripSeen (or kStripSeenNow)
    const uint64_t* pix_base;   // per view
    uint32_t* done;             // per-tile bitmap
    uint32_t* strips;           // per tile: row bits of the rows whose pixels all stopped, kStripSeenNow
                                // once this slice blended it, kStripSeen once an earlier one did
    uint32_t active_cap;        // capacity of `active` (kActivePerTile x all tiles of the launch set)
};
Status launch_blend_slice(const uint2* ranges, const uint32_t* values, const SplatArrays& sp,
                          const ViewParams* views, int V, uint32_t n_entries, const float* bg,
                          unsigned long long* counters, const SliceBlendArgs& sl, int ctas_per_sm, int batch,
                          cudaStream_t st);

}  // namespace tigas
