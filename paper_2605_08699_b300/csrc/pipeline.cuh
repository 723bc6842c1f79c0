// Frame pipeline: scenes, workspace arenas, camera setup and the stream-ordered
// sequence K1 -> (depth sort) -> K2 -> K3 -> K4 -> K5 -> K6.
#pragma once

#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace tigas {

struct Scene {
    SceneView view;            // device layout
    uint4* chunks = nullptr;   // owned allocation
    size_t bytes = 0;
    std::atomic<int> refs{1};  // caller reference + in-flight users
};

void scene_acquire(Scene* s);
void scene_release(Scene* s);

// Grow-only device buffer handed out in 256-byte aligned slices.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    Status reserve(size_t bytes);   // call only when no work uses the arena
    void reset() { used = 0; }
    template <typename T>
    T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        return reinterpret_cast<T*>(base + off);
    }
    void release();
};

// Camera setup for one view (host, FP64 -> FP32): R = R_y(az) R_x(el),
// W = R^T, limits of the EWA guard band.  tile_base: first global tile id.
ViewParams make_view(const tigas_pose& pose, const tigas_intrinsics& k, int width, int height,
                     uint32_t tile_base);

enum Stage { kStPreprocess, kStDepthSort, kStScan, kStEmit, kStPairSort, kStRanges, kStBlend, kNumStages };
constexpr int kMaxSlices = 16;   // depth slices of the sliced schedule (and event pairs per stage)

// Process-wide stage timing (tigas_profile_*).
extern std::atomic<bool> g_profile;
void profile_accumulate(const float* ms, const int* used, float frame_ms);
void profile_read(double* ms, uint64_t* calls, bool reset);

// Render state of one in-flight frame or launch set: stream, arenas, pinned staging.
struct RenderContext {
    cudaEvent_t ev_start[kNumStages][kMaxSlices] = {};
    cudaEvent_t ev_stop[kNumStages][kMaxSlices] = {};
    int ev_count[kNumStages] = {};     // start/stop pairs recorded per stage this frame
    uint32_t* h_misc = nullptr;        // pinned readback of per-view counts
    cudaStream_t stream = nullptr;     // own stream (used when the caller passes none)
    Arena fixed;                       // per-entry buffers
    Arena pairs;                       // per-pair buffers
    uint64_t* h_total = nullptr;       // pinned readback of P
    uint32_t* h_flags = nullptr;       // pinned readback of overflow flags
    ViewParams* h_views = nullptr;     // pinned view table
    std::vector<uint8_t*> dev_staging; // device frames for host outputs
    std::vector<size_t> staging_bytes;
    Status init();
    void destroy();
};

struct FrameRequest {
    int V = 1;
    ViewParams views[kMaxViews];       // out pointers must be device pointers (or null)
    int sort_mode = TIGAS_SORT_DEPTH_FIRST;
    int n_slices = 8;                    // sliced schedule: geometric depth slices
    bool want_counters = false;          // count blend evaluations / fetched entries
    bool want_q = false;
};

struct FrameResult {
    uint64_t pairs = 0;
    uint32_t total_tiles = 0;
    int sort_passes = 0;
    // device pointers valid until the context is reused
    const uint32_t* values = nullptr;    // sorted pair values (entries)
    const uint2* ranges = nullptr;
    SplatArrays splats{};
    uint32_t* d_visible = nullptr;
    unsigned long long* d_counters = nullptr;   // [evals, fetched] when requested
};

// After the stream is synchronised: add this frame's stage times (profiling on).
void collect_profile(RenderContext& ctx);

// Run the whole hot path for req.V views of one scene on stream st.  Reads P
// back once (after the scan) to size the pair buffers exactly.  Returns after
// enqueuing the blend and the flag readback; the caller synchronises.
Status render_frame(Scene* scene, FrameRequest& req, RenderContext& ctx, cudaStream_t st, FrameResult* res);

// Context pool used by the synchronous entry points.
RenderContext* acquire_context(Status* err);
void release_context(RenderContext* ctx);

bool is_device_pointer(const void* p);

}  // namespace tigas
