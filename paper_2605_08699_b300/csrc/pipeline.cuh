// Frame pipeline: scenes, workspace arenas, camera setup and the stream-ordered
// sequence K1 -> (depth sort) -> K2 -> K3 -> K4 -> K5 -> K6.
#pragma once

#include <cstddef>
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace tigas {

struct Scene {
    SceneView view;            // device layout
    uint4* chunks = nullptr;   // owned allocation
    size_t bytes = 0;
    std::atomic<int> refs{1};  // caller reference + in-flight users
    uint64_t id = 0;           // unique for the process: a freed scene's address can be reused, its id cannot
};

void scene_acquire(Scene* s);
void scene_release(Scene* s);

// Resident bytes of a scene of n Gaussians in the given storage.
size_t scene_bytes_for(uint64_t n, int storage);
// New scene (one reference) from raw attribute arrays in device memory:
// activate and pack on st, then synchronize st.
Status scene_create(const float* means, const float* log_scales, const float* quats, const float* logits,
                    const float* sh, uint32_t n, int sh_degree, int storage, const float bg[3], cudaStream_t st,
                    Scene** out);

// ------------------------------------------------------------ PLY models
// A 3DGS vertex record maps to 59 raw fields in scene-description order:
// x y z | scale_0..2 | rot_0..3 | opacity | SH coefficient k, channel c at
// 11 + 3k + c (f_dc_c is k = 0; f_rest_{c*M+j} is k = j + 1, M = (d+1)^2 - 1).
constexpr int kPlyFields = 59;
enum PlyType : uint8_t { kPlyI8, kPlyU8, kPlyI16, kPlyU16, kPlyI32, kPlyU32, kPlyF32, kPlyF64, kPlyAbsent = 0xFF };
enum PlyFormat { kPlyBinaryLE = 0, kPlyBinaryBE = 1, kPlyAscii = 2 };

struct PlyLayout {
    uint64_t n = 0;                  // vertex count
    uint64_t body_offset = 0;        // byte offset of the vertex block (binary) or of the data (ascii)
    uint64_t skip_lines = 0;         // ascii: lines of elements that precede the vertex element
    uint64_t file_bytes = 0;
    int format = kPlyBinaryLE;
    int sh_degree = 0;               // from the count of f_rest_* properties (0, 9, 24, 45)
    uint32_t row_bytes = 0;          // bytes of one binary vertex record
    std::vector<uint8_t> prop_type;  // vertex properties in file order
    std::vector<uint32_t> prop_offset;
    int32_t field_prop[kPlyFields];  // vertex property feeding each field, -1 = absent (zero)
};

// Parse the header of a 3DGS PLY file (no body read beyond a size check).
Status ply_probe(const char* path, PlyLayout* out);
// Decode the vertex block into raw attribute arrays in device memory
// (means[n][3], log_scales[n][3], quats[n][4], logits[n], sh[n][48]); synchronizes st.
Status ply_decode(const char* path, const PlyLayout& lay, float* means, float* log_scales, float* quats,
                  float* logits, float* sh, cudaStream_t st);
// probe + decode + scene_create.
Status scene_load_ply(const char* path, int storage, const float bg[3], Scene** out);

// ------------------------------------------------------- quality metrics
// Bilinear RGBA8 resample (w x h -> W x H), exact fixed-point arithmetic.
Status launch_resample(const uint8_t* src, int w, int h, uint8_t* dst, int W, int H, cudaStream_t st);
// Device scratch for launch_quality; its first two words receive the SSIM sum
// over window positions and channels (double) and the squared error (u64).
size_t quality_tmp_bytes(int W, int H);
Status launch_quality(const uint8_t* a, const uint8_t* b, int W, int H, void* tmp, float* map, cudaStream_t st);
struct RenderContext;
Status resample_rgba8(RenderContext& ctx, const uint8_t* src, int w, int h, uint8_t* dst, int W, int H,
                      cudaStream_t st);
Status image_quality(RenderContext& ctx, const uint8_t* a, const uint8_t* b, int W, int H, float* map,
                     double* ssim, double* psnr, cudaStream_t st);

// Grow-only device buffer handed out in 256-byte aligned slices.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    uint64_t gen = 0;               // bumped whenever base is freed (captured graphs hold pointers)
    bool over = false;              // a take went past cap since the last reset (nothing may launch)
    Status reserve(size_t bytes);   // call only when no work uses the arena
    void reset() {
        used = 0;
        over = false;
    }
    template <typename T>
    T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        if (used > cap) over = true;
        return reinterpret_cast<T*>(base + off);
    }
    void release();
};

// The values a sliced launch set starts from, laid out contiguously so that
// one host-to-device copy from the context's pinned staging sets them all
// (each copy or memset node in a launch set's graph costs a step of its own).
struct LaunchHeader {
    ViewParams views[kMaxViews];
    uint64_t pix_base[kMaxViews];   // first pixel of each view in the per-pixel state
    uint32_t flags[2];              // [overflow and timeout flags, passes of the depth sort]: zero
    uint64_t near;                  // entries in full depth order (a partial depth sort): zero; read back
                                    // with the flags
    uint32_t visible[kMaxViews];    // kept entries per view: zero
    uint32_t key_range[4];          // [min, max] of the kept depth keys: [0xFFFFFFFF, 0]; a partial depth
                                    // sort's threshold and flag: zero
    uint32_t split_hist[kSplitBins + 1];   // the threshold's depth histogram and finished-CTA count: zero
};
static_assert(offsetof(LaunchHeader, near) == offsetof(LaunchHeader, flags) + 8,
              "the flags and the near count are read back in one copy");

// Camera setup for one view (host, FP64 -> FP32): R = R_y(az) R_x(el),
// W = R^T, limits of the EWA guard band.  tile_base: first global tile id.
ViewParams make_view(const tigas_pose& pose, const tigas_intrinsics& k, int width, int height,
                     uint32_t tile_base);

enum Stage { kStPreprocess, kStDepthSort, kStScan, kStEmit, kStPairSort, kStRanges, kStBlend, kNumStages };
constexpr int kMaxSlices = 16;   // depth slices of the sliced schedule (and event pairs per stage)

// Process-wide stage timing (tigas_profile_*).
extern std::atomic<uint32_t> g_profile;   // bit s: time stage s (0: off)
void profile_accumulate(const float* ms, const int* used, float frame_ms);
void profile_read(double* ms, uint64_t* calls, bool reset);

struct FrameResult {
    uint64_t pairs = 0;
    uint32_t total_tiles = 0;
    int sort_passes = 0;
    // device pointers valid until the context is reused
    const uint32_t* values = nullptr;    // sorted pair values (entries)
    const uint2* ranges = nullptr;
    SplatArrays splats{};
    uint32_t* d_visible = nullptr;
    unsigned long long* d_counters = nullptr;   // [evals, fetched, blends] when requested
    int graph_slices = 0;                       // replayed graph: pairs = sum of ctx.h_total[0..slices)
    bool direct_static = false;                 // fixed-capacity launch set run directly, not from a graph
    bool near_split = false;                    // partial depth sort: ctx.h_flags[2..3] hold its near count
    uint64_t entries = 0;                       // (Gaussian, view) entries of the launch set
};

// Render state of one in-flight frame or launch set: stream, arenas, pinned staging.
struct RenderContext {
    cudaEvent_t ev_start[kNumStages][kMaxSlices] = {};
    cudaEvent_t ev_stop[kNumStages][kMaxSlices] = {};
    int ev_count[kNumStages] = {};     // start/stop pairs recorded per stage this frame
    uint32_t* h_misc = nullptr;        // pinned readback of per-view counts
    cudaStream_t stream = nullptr;     // own stream (used when the caller passes none)
    cudaStream_t copy_stream = nullptr;  // device-to-host copies of asynchronous launch sets
    cudaEvent_t ev_rendered = nullptr;   // end of a launch set's device work (copies wait on it)
    Arena fixed;                       // per-entry buffers
    Arena pairs;                       // per-pair buffers
    Arena jpeg;                        // frame encoder buffers
    uint64_t* h_total = nullptr;       // pinned readback of P
    uint32_t* h_flags = nullptr;       // pinned readback of the flags and a partial depth sort's near count
    LaunchHeader* h_header = nullptr;  // pinned staging of a launch set's header (views and counters)
    std::vector<uint8_t*> dev_staging; // device frames for host outputs
    std::vector<size_t> staging_bytes;
    // captured sliced launch sets, keyed by their shape
    struct Graph {
        std::vector<int64_t> key;
        cudaGraphExec_t exec = nullptr;
        uint64_t cap = 0;
        uint64_t launches = 0;
        int ev_count[kNumStages] = {};
        int slices = 0;
        uint64_t fixed_gen = 0, pairs_gen = 0;
        FrameResult res;
    };
    std::vector<Graph> graphs;
    // launch-set shapes seen once (captured on their second appearance)
    std::vector<std::vector<int64_t>> seen_keys;
    // largest slice pair count seen, per unit of view scale (pair_scale), for each
    // schedule (slices, first-slice fraction) the context has rendered: a schedule
    // of fewer slices has larger ones, and a context serves every launch-set size
    std::vector<std::pair<uint32_t, double>> slice_ratios;
    double& slice_ratio(int n_slices, int first_slice_inv);
    Status init();
    void destroy();
};

struct FrameRequest {
    int V = 1;
    ViewParams views[kMaxViews];       // out pointers must be device pointers (or null)
    int sort_mode = TIGAS_SORT_DEPTH_FIRST;
    int n_slices = 8;                    // sliced schedule: geometric depth slices
    int first_slice_inv = 64;            // the nearest slice holds 1/first_slice_inv of the entries
    int blend_ctas_per_sm = 0;           // persistent blend CTAs per SM (0: as many as fit)
    int blend_batch = 32;                // list entries a blend warp stages at a time (16 or 32)
    bool want_counters = false;          // count blend evaluations / fetched entries
    bool want_q = false;
};

// After the stream is synchronised: add this frame's stage times (profiling on).
void collect_profile(RenderContext& ctx);

// Run the whole hot path for req.V views of one scene on stream st.  Reads P
// back once (after the scan) to size the pair buffers exactly.  Returns after
// enqueuing the blend and the flag readback; the caller synchronises.
Status render_frame(Scene* scene, FrameRequest& req, RenderContext& ctx, cudaStream_t st, FrameResult* res);

// The depth-sliced schedule.  static_cap == 0: exact (host reads back counts);
// static_cap > 0: device-side counts and fixed pair capacity, capturable in a
// CUDA graph (workspace reserved beforehand, see sliced_workspace).
// slice_pairs (host, n_slices entries, exact mode only): pairs per slice.
Status render_frame_sliced(Scene* scene, FrameRequest& req, RenderContext& ctx, cudaStream_t st, FrameResult* res,
                           uint64_t static_cap, uint64_t* slice_pairs);
Status sliced_workspace(const Scene* scene, FrameRequest& req, uint64_t pair_cap, size_t* fixed_bytes,
                        size_t* pair_bytes);
// Write the launch set's view table and pixel offsets to the pinned staging
// buffer the (captured) host-to-device copy reads.
void sliced_stage_views(const Scene* scene, FrameRequest& req, RenderContext& ctx);

// Render req through a CUDA graph of the static sliced schedule, capturing it
// on first use of a shape (that first frame is rendered exactly).  *rendered
// is false when graphs cannot serve this request (caller renders exactly).
Status render_sliced_graph(Scene* scene, FrameRequest& req, RenderContext& ctx, cudaStream_t st, FrameResult* res,
                           bool* rendered);
extern std::atomic<bool> g_use_graphs;
extern std::atomic<uint64_t> g_exact_rerenders;   // fixed-capacity launch sets rendered again exactly
// Schedule parameters of a launch set (tigas_set_schedule / tigas_autotune).
struct Schedule {
    int n_slices = 8;
    int first_slice_inv = 64;
    int blend_ctas_per_sm = 0;
    int blend_batch = 32;
    int views_per_set = 0;   // the server's launch sets hold at most this many views (0: no cap)
};
// Launch sets are grouped by view count into the classes 1, 2, 3-4, 5-8,
// 9-16, 17-32 and 33-64 views, each with its own schedule: fixed per-slice
// costs weigh more in a small launch set, so fewer slices suit it.
constexpr int kScheduleClasses = 7;
int schedule_class(int n_views);
Schedule current_schedule(int n_views);
void set_schedule(const Schedule& s);                  // every class
void set_schedule_for(int n_views, const Schedule& s);   // the class of n_views
void drop_graphs(RenderContext& ctx);
// Idle contexts drop their graphs, the shapes they have seen and the learned
// slice capacity.
void forget_launch_sets();
// Pair-count scale of a launch set: sum over views of n (1 + 3 sqrt(W H / 1080p))^2 / 16.
double pair_scale(const Scene* scene, const FrameRequest& req);

// Context pool used by the synchronous entry points.
RenderContext* acquire_context(Status* err);
void release_context(RenderContext* ctx);
// Destroy the pooled contexts no call holds (arenas, graphs, staging, pinned
// buffers); later calls create new ones.
void release_idle_contexts();

bool is_device_pointer(const void* p);
// Baseline JPEG of one RGBA8 frame (host or device in/out), synchronous on st.
Status jpeg_encode(RenderContext& ctx, const uint8_t* rgba, int W, int H, int quality, int restart, uint8_t* out,
                   uint64_t cap, uint64_t* out_len, cudaStream_t st);

}  // namespace tigas
