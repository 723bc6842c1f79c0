// Launch interface of the hot-path kernels (all stream-ordered, no host sync).
#pragma once

#include "common.cuh"

namespace tigas {

// a0 / K7: activate raw attributes and pack them into the resident layout.
Status launch_scene_pack(const float* means, const float* log_scales, const float* quats,
                         const float* opacity_logits, const float* sh, uint32_t n, int sh_degree,
                         int storage, uint4* chunks, cudaStream_t st);

// K1: per-Gaussian preprocess for V views (Gaussian attributes read once).
// views: device array of V ViewParams.  n_visible: device counters [V], and
// out.key_range: [min, max] of the kept depth keys; both set to their start
// values here (zero, [0xFFFFFFFF, 0]) unless counters_set says the caller
// already did.
Status launch_preprocess(const SceneView& scene, const ViewParams* views, int V, const SplatArrays& out,
                         uint32_t* n_visible, cudaStream_t st, bool counters_set = false);

// K2: exclusive scan of u32 counts.  out[k] = sum_{k' < k} in[order ? order[k'] : k'],
// total64 = full sum (u64).  tmp: scratch of scan_tmp_words(n) words.
size_t scan_tmp_words(uint64_t n);
// total_zeroed: *total64 is already zero (no clearing launch).
Status launch_scan_u32(const uint32_t* in, const uint32_t* order, uint32_t* out, uint64_t n,
                       uint64_t* total64, uint32_t* tmp, cudaStream_t st, bool total_zeroed = false);
// Entries per block of the sliced count kernel, whose blocks' sums this scan
// turns into block offsets (also the scan's own tile).
constexpr uint32_t kScanBlock = 4096;

// K3: duplicate-and-key emit.  For each k < n_entries with e = order ? order[k] : k
// and tiles[e] > 0, write the tiles of rect[e] (row-major) at offsets[k]..:
//   32-bit keys: key = tile_base(view) + ty * TX + tx
//   64-bit keys: key = (tile id << 32) | depth_key[e]
// value = e.  Writes beyond pair_cap are dropped and set *overflow.
Status launch_emit_u32(const uint32_t* order, const uint32_t* offsets, const SplatArrays& sp,
                       const ViewParams* views, int V, uint32_t n_per_view, uint64_t n_entries,
                       uint32_t* keys, uint32_t* values, uint64_t pair_cap, uint32_t* overflow,
                       cudaStream_t st);
Status launch_emit_u64(const uint32_t* offsets, const SplatArrays& sp, const ViewParams* views, int V,
                       uint32_t n_per_view, uint64_t n_entries, uint64_t* keys, uint32_t* values,
                       uint64_t pair_cap, uint32_t* overflow, cudaStream_t st);

// K4: stable LSD radix sort of (key, value) pairs over key bits [begin, end).
// The element count is min(*d_n, n_cap) when d_n is given, else n_cap.
// values_in == nullptr means values 0..n-1.  keys_alt/values_alt are the
// ping-pong buffers; the sorted result lands in (keys_out, values_out).
// tmp: radix_tmp_words(n_cap) words.  flags (optional device word): the sort
// ORs kSortTimeoutFlag into it when a look-back wait ran out (the result is
// then not to be trusted); without flags the bit goes to a word of tmp.
// A pass whose digit is the same for every key is skipped on the device.
// ex (optional; the fields other than tmp_zeroed for 32-bit keys only):
//   key_range: device [kmin, kmax] of the keys other than 0xFFFFFFFF; digits
//     are taken from k - kmin (0xFFFFFFFF -> kmax - kmin + 1), the same order,
//     so keys spanning less than 2^24 need three passes; keys_out then holds
//     the mapped keys (the first pass stores them, later passes read them);
//   pay_in / pay_alt / pay_out: an 8-byte payload per key moved with it;
//   near_split (with key_range, after launch_near_split wrote key_range[2..3]
//     and *d_near): a partial sort.  The keys below the threshold (the near
//     ones, *d_near of them) end up in full order at the front; the others
//     (the far ones, and 0xFFFFFFFF) follow in input order.  The first pass
//     runs over every key and moves the far ones to the output buffers; the
//     later passes run over the near ones only.  The near keys' digits are
//     taken in base 255 for the first pass (m = k - kmin = 255 q + r: r, then
//     q's bytes), so that digit 255 of the first pass is the far keys' alone.
// With a payload, values_in, values_alt and values_out may all be null: no
// value stream is read or written (the payload identifies each key).
constexpr uint32_t kSortTimeoutFlag = 16u;
struct SortExtras {
    const uint32_t* key_range = nullptr;
    const uint2* pay_in = nullptr;
    uint2* pay_alt = nullptr;
    uint2* pay_out = nullptr;
    bool near_split = false;
    const uint64_t* d_near = nullptr;
    // the threshold came from a sample of the keys: the sort writes *d_near
    // itself (the keys below the threshold) and sets the overflow bit of its
    // flags if fewer than near_target are (the caller renders again)
    bool near_sampled = false;
    uint64_t near_target = 0;
    // (any key width) tmp's first radix_zero_words(passes) words are already
    // zero: the sort clears nothing itself (no memset in the launch sequence)
    bool tmp_zeroed = false;
};
// Threshold of a partial depth sort: the smallest bin boundary thr (bins of
// (k - kmin) >> s, at most kSplitBins of them over [kmin, kmax]) below which
// at least `target` of the n keys lie (all kept keys when fewer), from a
// histogram of the keys.  key_range: [kmin, kmax, thr, split flag]; writes
// key_range[2] = thr, key_range[3] = 1 and *d_near = the keys below thr.
// hist: kSplitBins + 1 words, zero on entry (the last word counts finished
// CTAs).  keys 16-byte aligned.  Also clears sort_zero[0 .. n_sort_zero)
// (null: none; the scratch words the depth sort expects zeroed).
// sample > 1: the histogram of every sample-th group of 4 keys places the
// threshold, with a margin of 1 % of the sampled keys above the target's share
// of them; *d_near is then left to the sort (SortExtras::near_sampled), which
// counts the near keys exactly and flags a shortfall.
constexpr int kSplitBins = 2048;
Status launch_near_split(const uint32_t* keys, uint64_t n, uint32_t* key_range, uint64_t target, uint32_t* hist,
                         uint64_t* d_near, uint32_t* sort_zero, int n_sort_zero, int sample, cudaStream_t st);
size_t radix_tmp_words(uint64_t n_cap);
// Device word of tmp holding how many passes the last one-sweep sort using
// tmp ran (valid once it completed; inputs of 2^30 keys or more leave it 0).
const uint32_t* radix_active_passes(const uint32_t* tmp);
// Device words of tmp holding, for digit d of pass `pass` of the last
// one-sweep sort using tmp, how many keys have a smaller digit in that pass
// (256 words; valid once it completed; inputs of 2^30 keys or more do not
// write them).
const uint32_t* radix_digit_bases(const uint32_t* tmp, int pass);
// Words at the start of tmp that a sort of `passes` passes expects zeroed
// (it clears them itself unless SortExtras::tmp_zeroed says they are).
size_t radix_zero_words(int passes);
template <typename K>
Status radix_sort(const K* keys_in, const uint32_t* values_in, K* keys_alt, uint32_t* values_alt,
                  K* keys_out, uint32_t* values_out, uint64_t n_cap, const uint64_t* d_n, int begin_bit,
                  int end_bit, uint32_t* tmp, cudaStream_t st, int* passes_out, uint32_t* flags = nullptr,
                  const SortExtras* ex = nullptr);

// Test hook: one radix-sort scatter CTA whose look-back waits on a chunk that
// no CTA publishes; *timed_out tells whether it recorded the timeout flag.
// Synchronous; allocates its own buffer of debug_lookback_words() words.
Status debug_lookback_timeout(int spin_limit, bool* timed_out);
// The same probe enqueued on st in buf (debug_lookback_words() words, 16-byte
// aligned, no other requirement: it initialises what it reads); the timeout
// flag is ORed into *flags (null: a word of buf).
size_t debug_lookback_words();
Status debug_lookback_enqueue(int spin_limit, uint32_t* buf, uint32_t* flags, cudaStream_t st);

// K5: tile ranges from sorted keys (tile = key >> shift), binary search per
// tile.  ranges: n_tiles uint2.  A key outside [0, n_tiles) sets *overflow bit 2.
template <typename K>
Status launch_ranges(const K* keys, uint64_t n_cap, const uint64_t* d_n, int shift, uint2* ranges,
                     uint32_t n_tiles, uint32_t* overflow, cudaStream_t st);

// K6: per-tile front-to-back blend of every view's tiles (grid = total_tiles).
// values hold entry indices < n_entries.  bg: host RGB.
// counters: optional device [evals, fetched, blends]: list entries evaluated per
// pixel up to its stop, entries staged into shared memory, entries blended.
Status launch_blend(const uint2* ranges, const uint32_t* values, const SplatArrays& sp,
                    const ViewParams* views, int V, uint32_t total_tiles, uint32_t n_entries,
                    const float* bg, unsigned long long* counters, cudaStream_t st);

}  // namespace tigas
