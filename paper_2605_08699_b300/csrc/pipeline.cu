// Frame pipeline orchestration (host side of the hot path).
#include "pipeline.cuh"
#include "sliced.cuh"

#include <cmath>
#include <cstring>

namespace tigas {

std::atomic<uint64_t> g_launches{0};
std::atomic<uint64_t> g_exact_rerenders{0};
std::atomic<uint32_t> g_profile{0u};
std::atomic<bool> g_use_graphs{true};

namespace {
std::mutex g_sched_mu;
// Defaults, the autotuner's picks for 3M Gaussians at 1080p: one view in 3
// slices (the first holding 1/16 of the entries), two in 4, three or four in
// 5, more in 6 (the first holding 1/64).
Schedule g_sched[kScheduleClasses] = {Schedule{3, 16, 0, 32, 0}, Schedule{4, 64, 0, 32, 0}, Schedule{5, 64, 0, 32, 0},
                                      Schedule{6, 64, 0, 32, 0},  Schedule{6, 64, 0, 32, 0}, Schedule{6, 64, 0, 32, 0},
                                      Schedule{6, 64, 0, 32, 0}};
}  // namespace

int schedule_class(int n_views) {
    int c = 0;
    while (c + 1 < kScheduleClasses && (1 << c) < n_views) ++c;
    return c;
}

Schedule current_schedule(int n_views) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    return g_sched[schedule_class(n_views)];
}

void set_schedule(const Schedule& s) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    for (Schedule& c : g_sched) c = s;
}

void set_schedule_for(int n_views, const Schedule& s) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    g_sched[schedule_class(n_views)] = s;
}

namespace {
std::mutex g_prof_mu;
double g_stage_ms[kNumStages + 1] = {};
uint64_t g_stage_calls[kNumStages + 1] = {};
}  // namespace

void profile_accumulate(const float* ms, const int* used, float frame_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int k = 0; k < kNumStages; ++k)
        if (used[k]) {
            g_stage_ms[k] += ms[k];
            g_stage_calls[k] += 1;
        }
    g_stage_ms[kNumStages] += frame_ms;
    g_stage_calls[kNumStages] += 1;
}

void profile_read(double* ms, uint64_t* calls, bool reset) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int k = 0; k <= kNumStages; ++k) {
        if (ms) ms[k] = g_stage_ms[k];
        if (calls) calls[k] = g_stage_calls[k];
        if (reset) {
            g_stage_ms[k] = 0;
            g_stage_calls[k] = 0;
        }
    }
}

void collect_profile(RenderContext& ctx) {
    float ms[kNumStages] = {};
    cudaEvent_t first = nullptr, last = nullptr;
    for (int k = 0; k < kNumStages; ++k) {
        for (int r = 0; r < ctx.ev_count[k]; ++r) {
            float t = 0;
            if (cudaEventElapsedTime(&t, ctx.ev_start[k][r], ctx.ev_stop[k][r]) != cudaSuccess) {
                cudaGetLastError();
                t = 0;
            }
            ms[k] += t;
        }
    }
    // frame span: the preprocess start to the last blend stop
    if (ctx.ev_count[kStPreprocess] > 0) first = ctx.ev_start[kStPreprocess][0];
    if (ctx.ev_count[kStBlend] > 0) last = ctx.ev_stop[kStBlend][ctx.ev_count[kStBlend] - 1];
    bool any = false;
    for (int k = 0; k < kNumStages; ++k) any |= ctx.ev_count[k] > 0;
    if (!any) return;
    float frame = 0;
    if (first && last && cudaEventElapsedTime(&frame, first, last) != cudaSuccess) {
        cudaGetLastError();
        frame = 0;
    }
    profile_accumulate(ms, ctx.ev_count, frame);
    for (int k = 0; k < kNumStages; ++k) ctx.ev_count[k] = 0;
}

// ------------------------------------------------------------------ scene

void scene_acquire(Scene* s) { s->refs.fetch_add(1, std::memory_order_relaxed); }

void scene_release(Scene* s) {
    if (s->refs.fetch_sub(1, std::memory_order_acq_rel) == 1) {
        if (s->chunks) cudaFree(s->chunks);
        delete s;
    }
}

// ------------------------------------------------------- allocation faults

namespace {
std::atomic<bool> g_inject_armed{false};
std::mutex g_inject_mu;
int64_t g_inject_skip[2] = {0, 0};   // allocations of the kind still to pass
int64_t g_inject_fail[2] = {0, 0};   // then this many fail

bool injected_failure(int kind) {
    if (!g_inject_armed.load(std::memory_order_acquire)) return false;
    std::lock_guard<std::mutex> lk(g_inject_mu);
    if (g_inject_fail[kind] <= 0) return false;
    if (g_inject_skip[kind] > 0) {
        --g_inject_skip[kind];
        return false;
    }
    --g_inject_fail[kind];
    return true;
}
}  // namespace

void inject_alloc_failures(int kind, int64_t nth, int64_t count) {
    std::lock_guard<std::mutex> lk(g_inject_mu);
    g_inject_skip[kind] = nth > 0 ? nth - 1 : 0;
    g_inject_fail[kind] = nth > 0 ? count : 0;
    g_inject_armed.store(g_inject_fail[0] > 0 || g_inject_fail[1] > 0, std::memory_order_release);
}

cudaError_t device_alloc(void** p, size_t bytes) {
    if (injected_failure(0)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t pinned_alloc(void** p, size_t bytes) {
    if (injected_failure(1)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

// ------------------------------------------------------------------ arena

Status Arena::reserve(size_t bytes) {
    if (bytes <= cap) return {};
    if (base) {
        cudaFree(base);
        base = nullptr;
        cap = 0;
        ++gen;   // whatever was captured against the old buffer is stale, even if the next allocation fails
    }
    size_t want = bytes + bytes / 4 + (1 << 20);
    cudaError_t e = device_alloc(&base, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        base = nullptr;
        e = device_alloc(&base, bytes);   // retry without headroom
        if (e != cudaSuccess) {
            cudaGetLastError();
            base = nullptr;
            return {TIGAS_ERR_OOM, "workspace allocation of " + std::to_string(bytes) + " bytes failed"};
        }
        want = bytes;
    }
    cap = want;
    used = 0;
    ++gen;
    return {};
}

void Arena::release() {
    if (base) {
        cudaFree(base);
        ++gen;
    }
    base = nullptr;
    cap = used = 0;
}

// ----------------------------------------------------------------- camera

ViewParams make_view(const tigas_pose& pose, const tigas_intrinsics& k, int width, int height, uint32_t tile_base) {
    ViewParams v{};
    const double ca = std::cos(pose.azimuth), sa = std::sin(pose.azimuth);
    const double ce = std::cos(pose.elevation), se = std::sin(pose.elevation);
    // R = R_y(az) R_x(el); columns: camera right, down, forward in world
    const double R[9] = {ca, sa * se, sa * ce,
                         0.0, ce, -se,
                         -sa, ca * se, ca * ce};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) v.Rt[3 * r + c] = (float)R[3 * c + r];
    for (int c = 0; c < 3; ++c) v.campos[c] = (float)pose.t[c];
    v.fx = (float)k.fx; v.fy = (float)k.fy; v.cx = (float)k.cx; v.cy = (float)k.cy;
    v.limx = (float)(1.3 * width / (2.0 * k.fx));
    v.limy = (float)(1.3 * height / (2.0 * k.fy));
    v.W = width; v.H = height;
    v.TX = (width + kTile - 1) / kTile;
    v.TY = (height + kTile - 1) / kTile;
    v.tile_base = tile_base;
    return v;
}

// ---------------------------------------------------------------- context

Status RenderContext::init() {
    TIGAS_CUDA_TRY(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    TIGAS_CUDA_TRY(cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking));
    TIGAS_CUDA_TRY(cudaEventCreateWithFlags(&ev_rendered, cudaEventDisableTiming));
    TIGAS_CUDA_TRY(pinned_alloc(&h_total, sizeof(uint64_t) * (kMaxSlices + 2)));
    TIGAS_CUDA_TRY(pinned_alloc(&h_flags, sizeof(uint32_t) * 4));
    TIGAS_CUDA_TRY(pinned_alloc(&h_header, sizeof(LaunchHeader)));
    std::memset(h_header, 0, sizeof(LaunchHeader));
    h_header->key_range[0] = 0xFFFFFFFFu;
    TIGAS_CUDA_TRY(pinned_alloc(&h_misc, sizeof(uint32_t) * kMaxViews));
    for (int k = 0; k < kNumStages; ++k)
        for (int r = 0; r < kMaxSlices; ++r) {
            TIGAS_CUDA_TRY(cudaEventCreate(&ev_start[k][r]));
            TIGAS_CUDA_TRY(cudaEventCreate(&ev_stop[k][r]));
        }
    return {};
}

void drop_graphs(RenderContext& ctx);

void RenderContext::destroy() {
    drop_graphs(*this);
    fixed.release();
    pairs.release();
    jpeg.release();
    for (auto* p : dev_staging)
        if (p) cudaFree(p);
    dev_staging.clear();
    staging_bytes.clear();
    if (h_total) cudaFreeHost(h_total);
    if (h_flags) cudaFreeHost(h_flags);
    if (h_header) cudaFreeHost(h_header);
    if (stream) cudaStreamDestroy(stream);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    if (ev_rendered) cudaEventDestroy(ev_rendered);
    copy_stream = nullptr;
    ev_rendered = nullptr;
    for (int k = 0; k < kNumStages; ++k)
        for (int r = 0; r < kMaxSlices; ++r) {
            if (ev_start[k][r]) cudaEventDestroy(ev_start[k][r]);
            if (ev_stop[k][r]) cudaEventDestroy(ev_stop[k][r]);
            ev_start[k][r] = ev_stop[k][r] = nullptr;
        }
    if (h_misc) cudaFreeHost(h_misc);
    h_misc = nullptr;
    h_total = nullptr; h_flags = nullptr; h_header = nullptr; stream = nullptr;
}

namespace {
std::mutex g_pool_mu;
std::vector<RenderContext*> g_pool;
}  // namespace

RenderContext* acquire_context(Status* err) {
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool.empty()) {
            RenderContext* c = g_pool.back();
            g_pool.pop_back();
            return c;
        }
    }
    auto* c = new RenderContext();
    Status s = c->init();
    if (!s.ok()) {
        c->destroy();
        delete c;
        if (err) *err = s;
        return nullptr;
    }
    return c;
}

void release_context(RenderContext* ctx) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    g_pool.push_back(ctx);
}

void release_idle_contexts() {
    std::vector<RenderContext*> idle;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        idle.swap(g_pool);
    }
    for (RenderContext* c : idle) {
        // idle contexts have no work queued; wait anyway before freeing what their streams used
        if (c->stream) cudaStreamSynchronize(c->stream);
        if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
        c->destroy();
        delete c;
    }
}

void forget_launch_sets() {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (RenderContext* c : g_pool) {
        drop_graphs(*c);
        c->seen_keys.clear();
        c->slice_ratios.clear();
    }
}

double& RenderContext::slice_ratio(int n_slices, int first_slice_inv) {
    const uint32_t key = ((uint32_t)n_slices << 16) | ((uint32_t)first_slice_inv & 0xFFFFu);
    for (auto& r : slice_ratios)
        if (r.first == key) return r.second;
    if (slice_ratios.size() >= 64) slice_ratios.erase(slice_ratios.begin());
    slice_ratios.emplace_back(key, 0.0);
    return slice_ratios.back().second;
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// -------------------------------------------------------------- pipeline

namespace {
// Stage timing: a start and a stop event per stage repetition.
struct Marker {
    RenderContext& ctx;
    cudaStream_t st;
    uint32_t stages;   // bit s: record stage s
    Status operator()(Stage sg, bool begin) {
        if (!((stages >> sg) & 1u)) return {};
        const int r = ctx.ev_count[sg];
        if (r >= kMaxSlices) return {};
        cudaEvent_t ev = begin ? ctx.ev_start[sg][r] : ctx.ev_stop[sg][r];
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        TIGAS_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        // inside a capture a plain record only orders work; an external record
        // node records the event each time the graph runs
        if (cs == cudaStreamCaptureStatusActive)
            TIGAS_CUDA_TRY(cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
        else
            TIGAS_CUDA_TRY(cudaEventRecord(ev, st));
        if (!begin) ctx.ev_count[sg] = r + 1;
        return {};
    }
};
}  // namespace

Status render_frame(Scene* scene, FrameRequest& req, RenderContext& ctx, cudaStream_t st, FrameResult* res) {
    if (req.sort_mode == TIGAS_SORT_SLICED) return render_frame_sliced(scene, req, ctx, st, res, 0, nullptr);
    for (int k = 0; k < kNumStages; ++k) ctx.ev_count[k] = 0;
    Marker mark{ctx, st, g_profile.load(std::memory_order_relaxed)};
    const int V = req.V;
    const uint32_t n = scene->view.n;
    const uint64_t E = (uint64_t)V * n;
    if (E >= 0xFFFFFFFFull) return {TIGAS_ERR_INVALID, "views x Gaussians exceeds 2^32 entries"};
    uint32_t total_tiles = 0;
    for (int v = 0; v < V; ++v) {
        req.views[v].tile_base = total_tiles;
        total_tiles += (uint32_t)(req.views[v].TX * req.views[v].TY);
    }
    const int tile_bits = total_tiles <= 1 ? 1 : 32 - __builtin_clz(total_tiles - 1);
    const bool full64 = req.sort_mode == TIGAS_SORT_FULL64;

    // ---- per-entry workspace
    const size_t presort_words = full64 ? 0 : radix_tmp_words(E);
    const size_t scan_words = scan_tmp_words(E);
    const size_t tmp_words = presort_words > scan_words ? presort_words : scan_words;
    size_t fixed_bytes = sizeof(ViewParams) * kMaxViews + 64 * 256;
    fixed_bytes += E * (16 + 16 + 4 + 4 + 4 + 8 + (req.want_q ? 4 : 0));
    fixed_bytes += full64 ? 0 : E * 4 * 4;                 // depth-sort ping-pong + result
    fixed_bytes += E * 4;                                  // offsets
    fixed_bytes += tmp_words * 4;
    fixed_bytes += sizeof(uint2) * (size_t)total_tiles;
    TIGAS_TRY(ctx.fixed.reserve(fixed_bytes));
    ctx.fixed.reset();
    ViewParams* d_views = ctx.fixed.take<ViewParams>(kMaxViews);
    uint64_t* d_total = ctx.fixed.take<uint64_t>(2);
    unsigned long long* d_counters = ctx.fixed.take<unsigned long long>(4);
    uint32_t* d_flags = ctx.fixed.take<uint32_t>(2);
    uint32_t* d_visible = ctx.fixed.take<uint32_t>(kMaxViews);
    SplatArrays sp{};
    sp.geom = ctx.fixed.take<float4>(E);
    sp.appear = ctx.fixed.take<float4>(E);
    sp.blue = ctx.fixed.take<float>(E);
    sp.depth_key = ctx.fixed.take<uint32_t>(E);
    sp.tiles = ctx.fixed.take<uint32_t>(E);
    sp.rect = ctx.fixed.take<uint2>(E);
    sp.q_dbg = req.want_q ? ctx.fixed.take<float>(E) : nullptr;
    uint32_t* offsets = ctx.fixed.take<uint32_t>(E);
    uint32_t *pk_alt = nullptr, *pv_alt = nullptr, *pk = nullptr, *order = nullptr;
    if (!full64) {
        pk_alt = ctx.fixed.take<uint32_t>(E);
        pv_alt = ctx.fixed.take<uint32_t>(E);
        pk = ctx.fixed.take<uint32_t>(E);
        order = ctx.fixed.take<uint32_t>(E);
    }
    uint32_t* tmp = ctx.fixed.take<uint32_t>(tmp_words);
    uint2* ranges = ctx.fixed.take<uint2>(total_tiles);
    if (ctx.fixed.over) return {TIGAS_ERR_CUDA, "workspace layout exceeds its reservation"};

    std::memcpy(ctx.h_header->views, req.views, sizeof(ViewParams) * V);
    TIGAS_CUDA_TRY(cudaMemcpyAsync(d_views, ctx.h_header->views, sizeof(ViewParams) * V, cudaMemcpyHostToDevice, st));
    TIGAS_CUDA_TRY(cudaMemsetAsync(d_flags, 0, sizeof(uint32_t) * 2, st));
    if (sp.q_dbg) TIGAS_CUDA_TRY(cudaMemsetAsync(sp.q_dbg, 0, E * 4, st));
    if (req.want_counters) TIGAS_CUDA_TRY(cudaMemsetAsync(d_counters, 0, sizeof(unsigned long long) * 4, st));

    // K1
    TIGAS_TRY(mark(kStPreprocess, true));
    TIGAS_TRY(launch_preprocess(scene->view, d_views, V, sp, d_visible, st));
    TIGAS_TRY(mark(kStPreprocess, false));

    // depth digits first (one key per entry), or nothing here (FULL64)
    if (!full64) {
        int passes = 0;
        TIGAS_TRY(mark(kStDepthSort, true));
        TIGAS_TRY(radix_sort<uint32_t>(sp.depth_key, nullptr, pk_alt, pv_alt, pk, order, E, nullptr, 0, 32, tmp, st,
                                       &passes, d_flags));
        TIGAS_TRY(mark(kStDepthSort, false));
    }
    // K2: pair offsets in emit order
    TIGAS_TRY(mark(kStScan, true));
    TIGAS_TRY(launch_scan_u32(sp.tiles, order, offsets, E, d_total, tmp, st));
    TIGAS_TRY(mark(kStScan, false));
    TIGAS_CUDA_TRY(cudaMemcpyAsync(ctx.h_total, d_total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
    const uint64_t P = ctx.h_total[0];
    if (P >= 0xFFFFFFFFull) return {TIGAS_ERR_OVERFLOW, "pair count exceeds 2^32"};

    // ---- per-pair workspace
    const size_t kb = full64 ? 8 : 4;
    const size_t sort_words = radix_tmp_words(P);
    size_t pair_bytes = P * (kb * 3 + 4 * 3) + sort_words * 4 + 3 * 256 * 4 + 16 * 256;
    TIGAS_TRY(ctx.pairs.reserve(pair_bytes));
    ctx.pairs.reset();
    void* keys_a = ctx.pairs.take<uint8_t>(P * kb);
    void* keys_b = ctx.pairs.take<uint8_t>(P * kb);
    void* keys_c = ctx.pairs.take<uint8_t>(P * kb);
    uint32_t* vals_a = ctx.pairs.take<uint32_t>(P);
    uint32_t* vals_b = ctx.pairs.take<uint32_t>(P);
    uint32_t* vals_c = ctx.pairs.take<uint32_t>(P);
    uint32_t* stmp = ctx.pairs.take<uint32_t>(sort_words);
    if (ctx.fixed.over || ctx.pairs.over) return {TIGAS_ERR_CUDA, "workspace layout exceeds its reservation"};

    int passes = 0;
    if (!full64) {
        // K3 in depth order, K4 on the tile digits only
        TIGAS_TRY(mark(kStEmit, true));
        TIGAS_TRY(launch_emit_u32(order, offsets, sp, d_views, V, n, E, (uint32_t*)keys_a, vals_a, P, d_flags, st));
        TIGAS_TRY(mark(kStEmit, false));
        TIGAS_TRY(mark(kStPairSort, true));
        TIGAS_TRY(radix_sort<uint32_t>((uint32_t*)keys_a, vals_a, (uint32_t*)keys_b, vals_b, (uint32_t*)keys_c, vals_c,
                                       P, nullptr, 0, tile_bits, stmp, st, &passes, d_flags));
        TIGAS_TRY(mark(kStPairSort, false));
        TIGAS_TRY(mark(kStRanges, true));
        TIGAS_TRY(launch_ranges<uint32_t>((uint32_t*)keys_c, P, nullptr, 0, ranges, total_tiles, d_flags, st));
        TIGAS_TRY(mark(kStRanges, false));
    } else {
        // K3 in index order with 64-bit (tile | depth) keys, K4 on all significant bits
        TIGAS_TRY(mark(kStEmit, true));
        TIGAS_TRY(launch_emit_u64(offsets, sp, d_views, V, n, E, (uint64_t*)keys_a, vals_a, P, d_flags, st));
        TIGAS_TRY(mark(kStEmit, false));
        TIGAS_TRY(mark(kStPairSort, true));
        TIGAS_TRY(radix_sort<uint64_t>((uint64_t*)keys_a, vals_a, (uint64_t*)keys_b, vals_b, (uint64_t*)keys_c, vals_c,
                                       P, nullptr, 0, 32 + tile_bits, stmp, st, &passes, d_flags));
        TIGAS_TRY(mark(kStPairSort, false));
        TIGAS_TRY(mark(kStRanges, true));
        TIGAS_TRY(launch_ranges<uint64_t>((uint64_t*)keys_c, P, nullptr, 32, ranges, total_tiles, d_flags, st));
        TIGAS_TRY(mark(kStRanges, false));
    }
    // K6
    TIGAS_TRY(mark(kStBlend, true));
    TIGAS_TRY(launch_blend(ranges, vals_c, sp, d_views, V, total_tiles, (uint32_t)E, scene->view.bg,
                           req.want_counters ? d_counters : nullptr, st));
    TIGAS_TRY(mark(kStBlend, false));
    TIGAS_CUDA_TRY(cudaMemcpyAsync(ctx.h_flags, d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));

    if (res) {
        res->pairs = P;
        res->total_tiles = total_tiles;
        res->sort_passes = passes;
        res->values = vals_c;
        res->ranges = ranges;
        res->splats = sp;
        res->d_visible = d_visible;
        res->d_counters = req.want_counters ? d_counters : nullptr;
    }
    return {};
}

// Depth-sliced schedule: same kernels per slice, only for tiles with a pixel
// still running; pixel state carried across slices (see sliced.cu).
//
// Two ways to run it:
//  - exact (static_cap == 0): the number of kept entries is read back once and
//    the slices cut the kept entries; every slice's pair count is read back
//    to size its buffers exactly (one host round trip per slice);
//  - static (static_cap > 0): slices cut all entries (culled ones sort last
//    and emit nothing), every kernel takes its counts from device memory and
//    pair buffers have the fixed capacity static_cap; nothing waits on the
//    host, so the launch sequence can be captured in a CUDA graph.  A slice
//    with more pairs than the capacity sets the overflow flag (the caller
//    re-renders exactly).  The arenas must already be reserved
//    (sliced_workspace gives the sizes).
namespace {

struct SlicedLayout {
    int V = 0, S = 0, tile_bits = 0;
    uint64_t E = 0, total_pix = 0;
    uint32_t total_tiles = 0, done_words = 0, total_sat = 0;
    uint64_t pix_base[kMaxViews] = {};
    size_t tmp_words = 0, fixed_bytes = 0;
};

SlicedLayout sliced_layout(const Scene* scene, FrameRequest& req) {
    SlicedLayout L;
    L.V = req.V;
    L.E = (uint64_t)req.V * scene->view.n;
    L.S = req.n_slices < 1 ? 1 : (req.n_slices > kMaxSlices ? kMaxSlices : req.n_slices);
    for (int v = 0; v < L.V; ++v) {
        req.views[v].tile_base = L.total_tiles;
        L.total_tiles += (uint32_t)(req.views[v].TX * req.views[v].TY);
        req.views[v].sat_base = L.total_sat;
        L.total_sat += (uint32_t)((req.views[v].TX + 1) * (req.views[v].TY + 1));
        L.pix_base[v] = L.total_pix;
        L.total_pix += (uint64_t)req.views[v].W * req.views[v].H;
    }
    L.tile_bits = L.total_tiles <= 1 ? 1 : 32 - __builtin_clz(L.total_tiles - 1);
    L.done_words = (L.total_tiles + 31) / 32;
    const size_t presort_words = radix_tmp_words(L.E);
    const size_t scan_words = scan_tmp_words(L.E + 1);
    L.tmp_words = presort_words > scan_words ? presort_words : scan_words;
    const uint64_t E = L.E;
    size_t b = sizeof(LaunchHeader) + 96 * 256;
    b += E * (16 + 16 + 4 + 4 + 4 + 8 + (req.want_q ? 4 : 0));
    b += E * 4 * 4 + (E + 1) * 4 + E * 8 * 2;             // depth sort buffers, in-block offsets, rects (2)
    b += ((E + 1 + kScanBlock - 1) / kScanBlock) * 4 * 2; // block sums of the counts and their offsets
    b += L.tmp_words * 4;
    b += (sizeof(uint2) + 4 * kActivePerTile + 4) * (size_t)L.total_tiles + L.done_words * 4;   // ranges, active, strips
    b += (size_t)L.total_sat * 4;                                                   // running-tile tables
    b += L.total_pix * 16 + sizeof(uint64_t) * kMaxViews * 2;
    L.fixed_bytes = b;
    return L;
}

// wide: room for 64-bit keys (a partial depth sort's last slice)
size_t pair_bytes_for(uint64_t P, bool wide) { return P * (wide ? 36 : 24) + radix_tmp_words(P) * 4 + 16 * 256; }

// A fixed-capacity launch set of three or more slices sorts by depth only the
// entries before its last slice (and a margin): the last slice holds most of
// the entries but few pairs, since most tiles have stopped by then, and its
// pairs are sorted by (tile, depth) instead.  Frames are the same; only the
// work differs.
#ifndef TIGAS_LIST_FROM
#define TIGAS_LIST_FROM 6   // in eighths of the slice count: the first slice emitting from a list
#endif
#ifndef TIGAS_FINE_FROM
#define TIGAS_FINE_FROM 6   // in eighths of the slice count: the first slice whose long lists take 4-row strips
#endif
#ifndef TIGAS_SPLIT_SAMPLE
#define TIGAS_SPLIT_SAMPLE 64   // the depth threshold's sample: every n-th group of four keys
#endif
#ifndef TIGAS_NEAR_SPLIT
#define TIGAS_NEAR_SPLIT 3   // fewest slices of a launch set with a partial depth sort
#endif
bool near_split_on(const SlicedLayout& L) { return L.S >= TIGAS_NEAR_SPLIT; }

// End of slice i of S over K entries: K / F ... K, geometric.
uint64_t slice_end(int i, int S, int F, uint64_t K) {
    if (i == S - 1) return K;
    const double f = S == 1 ? 1.0 : std::pow((double)F, (double)(i - (S - 1)) / (double)(S - 1));
    return (uint64_t)std::ceil(f * (double)K);
}

}  // namespace

void sliced_stage_views(const Scene* scene, FrameRequest& req, RenderContext& ctx) {
    SlicedLayout L = sliced_layout(scene, req);
    std::memcpy(ctx.h_header->views, req.views, sizeof(ViewParams) * L.V);
    std::memcpy(ctx.h_header->pix_base, L.pix_base, sizeof(uint64_t) * L.V);
}

Status sliced_workspace(const Scene* scene, FrameRequest& req, uint64_t pair_cap, size_t* fixed_bytes,
                        size_t* pair_bytes) {
    SlicedLayout L = sliced_layout(scene, req);
    *fixed_bytes = L.fixed_bytes;
    *pair_bytes = pair_bytes_for(pair_cap, near_split_on(L));
    return {};
}

Status render_frame_sliced(Scene* scene, FrameRequest& req, RenderContext& ctx, cudaStream_t st, FrameResult* res,
                           uint64_t static_cap, uint64_t* slice_pairs) {
    for (int k = 0; k < kNumStages; ++k) ctx.ev_count[k] = 0;
    Marker mark{ctx, st, g_profile.load(std::memory_order_relaxed)};
    const bool stat = static_cap > 0;
    const uint32_t n = scene->view.n;
    if ((uint64_t)req.V * n >= 0xFFFFFFFFull) return {TIGAS_ERR_INVALID, "views x Gaussians exceeds 2^32 entries"};
    const SlicedLayout L = sliced_layout(scene, req);
    const int V = L.V, S = L.S;
    const uint64_t E = L.E;
    const uint32_t total_tiles = L.total_tiles;
    // a partial depth sort (fixed capacity only: the exact path's slice ends
    // need the kept count, read back after the sort)
    const bool split = stat && near_split_on(L) && slice_end(S - 2, S, req.first_slice_inv, E) > 0;

    if (stat) {
        if (ctx.fixed.cap < L.fixed_bytes || ctx.pairs.cap < pair_bytes_for(static_cap, near_split_on(L)))
            return {TIGAS_ERR_INVALID, "static sliced schedule needs its workspace reserved first"};
    } else {
        TIGAS_TRY(ctx.fixed.reserve(L.fixed_bytes));
    }
    ctx.fixed.reset();
    LaunchHeader* d_hdr = ctx.fixed.take<LaunchHeader>(1);
    ViewParams* d_views = d_hdr->views;
    uint64_t* d_pix_base = d_hdr->pix_base;
    uint32_t* d_flags = d_hdr->flags;
    uint32_t* d_visible = d_hdr->visible;
    uint64_t* d_total = ctx.fixed.take<uint64_t>(kMaxSlices + 2);
    unsigned long long* d_counters = ctx.fixed.take<unsigned long long>(4);
    // [longest tiles, short tiles, work counter, long tiles, listed entries]
    uint32_t* d_misc = ctx.fixed.take<uint32_t>(8);
    SplatArrays sp{};
    sp.geom = ctx.fixed.take<float4>(E);
    sp.appear = ctx.fixed.take<float4>(E);
    sp.blue = ctx.fixed.take<float>(E);
    sp.depth_key = ctx.fixed.take<uint32_t>(E);
    sp.tiles = ctx.fixed.take<uint32_t>(E);
    sp.rect = ctx.fixed.take<uint2>(E);
    sp.q_dbg = req.want_q ? ctx.fixed.take<float>(E) : nullptr;
    uint32_t* pk_alt = ctx.fixed.take<uint32_t>(E);
    uint32_t* pv_alt = ctx.fixed.take<uint32_t>(E);
    uint32_t* pk = ctx.fixed.take<uint32_t>(E);
    uint32_t* order = ctx.fixed.take<uint32_t>(E);
    uint32_t* inblock = ctx.fixed.take<uint32_t>(E + 1);   // each entry's pair offset within its count block
    uint32_t* count_sums = ctx.fixed.take<uint32_t>((E + 1 + kScanBlock - 1) / kScanBlock);
    uint32_t* block_offs = ctx.fixed.take<uint32_t>((E + 1 + kScanBlock - 1) / kScanBlock);
    uint2* rect_sorted = ctx.fixed.take<uint2>(E);
    uint2* rect_alt = ctx.fixed.take<uint2>(E);
    sp.key_range = d_hdr->key_range;
    sp.tight_rect = req.want_q ? 0 : 1;   // debug frames report the method's 3-sigma rectangles
    // compact rectangles carry their entry through the depth sort (no value stream)
    bool compact = !req.want_q && V <= kCompactViews;
    for (int v = 0; v < V; ++v)
        compact = compact && req.views[v].TX <= kCompactTiles && req.views[v].TY <= kCompactTiles;
    sp.compact_rect = compact ? 1 : 0;
    uint32_t* tmp = ctx.fixed.take<uint32_t>(L.tmp_words);
    uint2* ranges = ctx.fixed.take<uint2>(total_tiles);
    uint32_t* active = ctx.fixed.take<uint32_t>(kActivePerTile * (size_t)total_tiles);
    uint32_t* strips = ctx.fixed.take<uint32_t>(total_tiles);
    uint32_t* sat = ctx.fixed.take<uint32_t>(L.total_sat);
    uint32_t* done = ctx.fixed.take<uint32_t>(L.done_words);
    float4* state = ctx.fixed.take<float4>(L.total_pix);
    if (ctx.fixed.over) return {TIGAS_ERR_CUDA, "sliced workspace layout exceeds its reservation"};

    // host -> device in one copy from the pinned staging: the view table, the views'
    // pixel offsets and the counters' start values (flags, kept entries, key range)
    sliced_stage_views(scene, req, ctx);
    TIGAS_CUDA_TRY(cudaMemcpyAsync(d_hdr, ctx.h_header, sizeof(LaunchHeader), cudaMemcpyHostToDevice, st));
    if (sp.q_dbg) TIGAS_CUDA_TRY(cudaMemsetAsync(sp.q_dbg, 0, E * 4, st));
    if (req.want_counters) TIGAS_CUDA_TRY(cudaMemsetAsync(d_counters, 0, sizeof(unsigned long long) * 4, st));

    TIGAS_TRY(mark(kStPreprocess, true));
    TIGAS_TRY(launch_preprocess(scene->view, d_views, V, sp, d_visible, st, /*counters_set=*/true));
    TIGAS_TRY(mark(kStPreprocess, false));
    TIGAS_TRY(mark(kStDepthSort, true));
    // depth order of every entry; its packed rectangle travels with it (no gather
    // afterwards), and digits count from the smallest kept depth key, so depths
    // spanning less than 2^24 key steps skip the fourth pass on the device.
    // Split: only the entries before the last slice need their order (the
    // last slice's pairs are sorted by (tile, depth)), so the passes after the
    // first run over the entries below a threshold that covers them.
    SortExtras dex;
    dex.key_range = sp.key_range;
    dex.pay_in = sp.rect;
    dex.pay_alt = rect_alt;
    dex.pay_out = rect_sorted;
    if (split) {
        // (also clears the depth sort's scratch words: no memset before it)
        // the threshold from a sample of the keys (TIGAS_SPLIT_SAMPLE: every n-th group of
        // four), the near count from the sort's own first histogram (depth sort 0.563 ->
        // 0.558 ms against reading every key; every 16th group: 0.560)
        const uint64_t target = slice_end(S - 2, S, req.first_slice_inv, E);
        TIGAS_TRY(launch_near_split(sp.depth_key, E, sp.key_range, target, d_hdr->split_hist, &d_hdr->near, tmp,
                                    (int)radix_zero_words(4), TIGAS_SPLIT_SAMPLE, st));
        dex.near_split = true;
        dex.d_near = &d_hdr->near;
        dex.tmp_zeroed = true;
        dex.near_sampled = TIGAS_SPLIT_SAMPLE > 1;
        dex.near_target = target;
    }
    TIGAS_TRY(radix_sort<uint32_t>(sp.depth_key, nullptr, pk_alt, compact ? nullptr : pv_alt, pk,
                                   compact ? nullptr : order, E, nullptr, 0, 32, tmp, st, nullptr, d_flags, &dex));
    TIGAS_TRY(mark(kStDepthSort, false));
    // also clears the done and strip bits and the slice totals (empty slices count 0),
    // and keeps the passes the depth sort ran in d_flags[1] (read back with the flags
    // at the end; the slices' scans reuse tmp)
    TIGAS_TRY(launch_init_slices(total_tiles, done, strips, d_total, kMaxSlices + 2, radix_active_passes(tmp),
                                 d_flags + 1, st));

    // entries the slices cut: kept ones only (exact), or all (static; culled
    // ones sort after every kept one and have empty rectangles)
    uint64_t K = E;
    if (!stat) {
        TIGAS_CUDA_TRY(cudaMemcpyAsync(ctx.h_misc, d_visible, sizeof(uint32_t) * V, cudaMemcpyDeviceToHost, st));
        TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
        K = 0;
        for (int v = 0; v < V; ++v) K += ctx.h_misc[v];
    }

    // geometric slice ends: K / first_slice_inv ... K
    uint64_t ends[kMaxSlices];
    for (int i = 0; i < S; ++i) ends[i] = slice_end(i, S, req.first_slice_inv, K);
    uint64_t total_pairs = 0;
    int passes = 0;
    uint64_t a = 0;
    SliceBlendArgs sl{active, d_misc, d_misc + 2, state, d_pix_base, done, strips, kActivePerTile * total_tiles};
    // the last quarter of the slices cut their longest lists (kLongestTile pairs or
    // more) into 4-row strips: measured per item, the first slices keep most warps
    // busy until their end, while a late slice ends with the serial compositing of
    // its few longest 8-row strips (8-view launch set, 7 slices: 3.405 ms with 8-row
    // strips only, 3.378 with 4-row strips from slice 5, 3.399 from slice 3)
    const int fine_from = (S * TIGAS_FINE_FROM) / 8;
    // the last quarter of the slices emit from a list of their entries with pairs
    // (8-view launch set, 7 slices: emit 0.272 -> 0.243 ms, the counts' list
    // 0.242 -> 0.250 ms; from slice 3 on: 0.240 and 0.254)
    const int list_from = (S * TIGAS_LIST_FROM) / 8;
    if (stat) {
        // pair buffers for the fixed capacity, taken once
        ctx.pairs.reset();
    }
    uint32_t *keys_a = nullptr, *keys_b = nullptr, *keys_c = nullptr, *vals_a = nullptr, *vals_b = nullptr,
             *vals_c = nullptr, *stmp = nullptr;
    // split: key buffers of 64-bit keys (the last slice's)
    const uint64_t kw = split ? 2 : 1;
    auto take_pairs = [&](uint64_t cap) {
        ctx.pairs.reset();
        keys_a = ctx.pairs.take<uint32_t>(kw * cap);
        keys_b = ctx.pairs.take<uint32_t>(kw * cap);
        keys_c = ctx.pairs.take<uint32_t>(kw * cap);
        vals_a = ctx.pairs.take<uint32_t>(cap);
        vals_b = ctx.pairs.take<uint32_t>(cap);
        vals_c = ctx.pairs.take<uint32_t>(cap);
        stmp = ctx.pairs.take<uint32_t>(radix_tmp_words(cap));
    };
    if (stat) {
        take_pairs(static_cap);
        if (ctx.pairs.over) return {TIGAS_ERR_CUDA, "pair workspace layout exceeds its reservation"};
    }
    for (int i = 0; i < S; ++i) {
        const uint64_t b = ends[i] > a ? ends[i] : a;
        if (slice_pairs) slice_pairs[i] = 0;
        if (b == a) continue;
        uint64_t* d_P = d_total + i;
        TIGAS_TRY(mark(kStScan, true));
        // the last slice of a split: its entries are in depth order only up to
        // the threshold, so its pairs carry (tile, depth) keys
        const bool wide = split && i == S - 1;
        const int pair_passes = ((wide ? 32 : 0) + L.tile_bits + 7) / 8;
        // also clears the slice's active-list counts and blend work counter (d_misc[0..3])
        // and, with fixed capacities (the pair buffers already taken), the pair sort's
        // scratch words, so that the sort runs no memset
        TIGAS_TRY(launch_running_sat(d_views, V, done, sat, d_misc, 5, stat ? stmp : nullptr,
                                     (int)radix_zero_words(pair_passes), st));
        // a late slice lists its entries with pairs (at most one per pair, so the list
        // fits a pair buffer that the sort fills only later) and emits from the list
        uint32_t* list = stat && i >= list_from ? vals_c : nullptr;
        // the count kernel writes each entry's prefix within its block of kScanBlock
        // entries and the blocks' sums; the scan of the sums gives the blocks'
        // offsets and the slice total (*d_P; the closing zero count puts the total at b)
        TIGAS_TRY(launch_count_slice(rect_sorted, a, b, d_views, V, sat, inblock, count_sums, compact, list,
                                     d_misc + 4, static_cap, st));
        TIGAS_TRY(launch_scan_u32(count_sums, nullptr, block_offs, (b - a + 1 + kScanBlock - 1) / kScanBlock, d_P,
                                  tmp, st));
        TIGAS_TRY(mark(kStScan, false));
        uint64_t cap = static_cap;
        if (!stat) {
            TIGAS_CUDA_TRY(cudaMemcpyAsync(ctx.h_total, d_P, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
            TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
            const uint64_t P = ctx.h_total[0];
            if (P >= 0xFFFFFFFFull) return {TIGAS_ERR_OVERFLOW, "pair count exceeds 2^32"};
            if (slice_pairs) slice_pairs[i] = P;
            if (P == 0) {
                a = b;
                continue;
            }
            total_pairs += P;
            TIGAS_TRY(ctx.pairs.reserve(pair_bytes_for(P, false)));
            take_pairs(P);
            if (ctx.pairs.over) return {TIGAS_ERR_CUDA, "pair workspace layout exceeds its reservation"};
            cap = P;
        }
        TIGAS_TRY(mark(kStEmit, true));
        TIGAS_TRY(launch_emit_slice(compact ? nullptr : order, rect_sorted, a, b, inblock, block_offs, d_views, V,
                                    done, keys_a, vals_a, cap, d_flags, compact, wide ? sp.depth_key : nullptr,
                                    sp.key_range, list, d_misc + 4, static_cap, st));
        TIGAS_TRY(mark(kStEmit, false));
        TIGAS_TRY(mark(kStPairSort, true));
        SortExtras pex;
        pex.tmp_zeroed = stat;
        if (wide)
            TIGAS_TRY(radix_sort<uint64_t>(reinterpret_cast<uint64_t*>(keys_a), vals_a,
                                           reinterpret_cast<uint64_t*>(keys_b), vals_b,
                                           reinterpret_cast<uint64_t*>(keys_c), vals_c, cap, d_P, 0,
                                           32 + L.tile_bits, stmp, st, nullptr, d_flags, &pex));
        else
            TIGAS_TRY(radix_sort<uint32_t>(keys_a, vals_a, keys_b, vals_b, keys_c, vals_c, cap, stat ? d_P : nullptr,
                                           0, L.tile_bits, stmp, st, &passes, d_flags, &pex));
        TIGAS_TRY(mark(kStPairSort, false));
        TIGAS_TRY(mark(kStRanges, true));
        // the pass over the tile's high byte (the second of a one-sweep sort of 9 to 16
        // key bits; the sixth of 64-bit keys): its digit bases bound each run of 256 tiles
        const uint32_t* hi_bases = cap < (1ull << 30) && L.tile_bits > 8 && L.tile_bits <= 16
                                       ? radix_digit_bases(stmp, wide ? 5 : 1)
                                       : nullptr;
        TIGAS_TRY(launch_ranges_active(keys_c, cap, stat ? d_P : nullptr, ranges, total_tiles, done, active, d_misc,
                                       d_flags, hi_bases, strips, wide,
                                       i >= fine_from ? kLongestTile : 0xFFFFFFFFu, st));
        TIGAS_TRY(mark(kStRanges, false));
        TIGAS_TRY(mark(kStBlend, true));
        TIGAS_TRY(launch_blend_slice(ranges, vals_c, sp, d_views, V, (uint32_t)E, scene->view.bg,
                                     req.want_counters ? d_counters : nullptr, sl, req.blend_ctas_per_sm,
                                     req.blend_batch, st));
        TIGAS_TRY(mark(kStBlend, false));
        a = b;
    }
    // the background of every tile no slice blended
    TIGAS_TRY(launch_fill_unseen(d_views, V, total_tiles, strips, scene->view.bg, st));
    // the flags and the near count of a partial depth sort
    TIGAS_CUDA_TRY(cudaMemcpyAsync(ctx.h_flags, d_flags, sizeof(uint32_t) * 4, cudaMemcpyDeviceToHost, st));
    if (stat) TIGAS_CUDA_TRY(cudaMemcpyAsync(ctx.h_total, d_total, sizeof(uint64_t) * S, cudaMemcpyDeviceToHost, st));
    if (res) {
        res->pairs = total_pairs;   // static: read ctx.h_total after the stream completes
        res->total_tiles = total_tiles;
        res->sort_passes = passes;
        res->values = nullptr;
        res->ranges = nullptr;
        res->splats = sp;
        res->d_visible = d_visible;
        res->d_counters = req.want_counters ? d_counters : nullptr;
        res->near_split = split;
        res->entries = E;
    }
    return {};
}


// ------------------------------------------------------------- CUDA graphs

namespace {
// Captured graphs hold the scene's device pointers: the key names the scene by
// its id, never by its address (a freed scene's address may come back).
std::vector<int64_t> graph_key(const Scene* scene, const FrameRequest& req) {
    std::vector<int64_t> k = {(int64_t)scene->id, scene->view.storage, req.V, req.n_slices,
                              req.first_slice_inv, req.blend_ctas_per_sm, req.blend_batch, req.want_counters ? 1 : 0,
                              (int64_t)g_profile.load()};
    for (int v = 0; v < req.V; ++v) {
        k.push_back(req.views[v].W);
        k.push_back(req.views[v].H);
    }
    return k;
}
}  // namespace

Status render_sliced_graph(Scene* scene, FrameRequest& req, RenderContext& ctx, cudaStream_t st, FrameResult* res,
                           bool* rendered) {
    *rendered = false;
    if (req.want_q) return {};
    const std::vector<int64_t> key = graph_key(scene, req);
    RenderContext::Graph* g = nullptr;
    for (auto& e : ctx.graphs)
        if (e.key == key) g = &e;
    if (g && (g->fixed_gen != ctx.fixed.gen || g->pairs_gen != ctx.pairs.gen)) {
        drop_graphs(ctx);   // an arena moved since the capture
        g = nullptr;
    }
    if (g) {
        sliced_stage_views(scene, req, ctx);
        TIGAS_CUDA_TRY(cudaGraphLaunch(g->exec, st));
        g_launches.fetch_add(g->launches, std::memory_order_relaxed);
        for (int k = 0; k < kNumStages; ++k) ctx.ev_count[k] = g->ev_count[k];
        if (res) {
            *res = g->res;
            res->graph_slices = g->slices;
        }
        *rendered = true;
        return {};
    }
    const double scale = pair_scale(scene, req);
    bool seen = false;
    for (auto& k : ctx.seen_keys) seen = seen || k == key;
    if (!seen) {
        // first launch set of this shape: no capture (shapes that do not repeat,
        // as in a server's mixed-resolution batches, would pay it every time)
        if (ctx.seen_keys.size() >= 64) ctx.seen_keys.erase(ctx.seen_keys.begin());
        ctx.seen_keys.push_back(key);
        const double ratio = ctx.slice_ratio(req.n_slices, req.first_slice_inv);
        if (ratio > 0.0) {
            // fixed capacity from the largest slice seen so far under this schedule: no
            // host round trips; an overflow is caught after the stream completes and
            // rendered exactly
            const uint64_t cap = (uint64_t)(1.5 * ratio * scale) + 65536;
            size_t fb = 0, pb = 0;
            TIGAS_TRY(sliced_workspace(scene, req, cap, &fb, &pb));
            TIGAS_TRY(ctx.fixed.reserve(fb));
            TIGAS_TRY(ctx.pairs.reserve(pb));
            TIGAS_TRY(render_frame_sliced(scene, req, ctx, st, res, cap, nullptr));
            if (res) {
                res->graph_slices = req.n_slices < 1 ? 1 : (req.n_slices > kMaxSlices ? kMaxSlices : req.n_slices);
                res->direct_static = true;
            }
            *rendered = true;
            return {};
        }
    }
    // render exactly and learn the slices' pair counts; capture when the shape repeats
    uint64_t sp[kMaxSlices] = {};
    TIGAS_TRY(render_frame_sliced(scene, req, ctx, st, res, 0, sp));
    TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
    *rendered = true;
    int exact_counts[kNumStages];
    for (int k = 0; k < kNumStages; ++k) exact_counts[k] = ctx.ev_count[k];
    if (ctx.h_flags[0] != 0) return {};
    uint64_t mx = 0;
    for (int i = 0; i < kMaxSlices; ++i) mx = sp[i] > mx ? sp[i] : mx;
    {
        double& ratio = ctx.slice_ratio(req.n_slices, req.first_slice_inv);
        if (scale > 0.0 && (double)mx / scale > ratio) ratio = (double)mx / scale;
    }
    if (!seen) return {};
    const uint64_t cap = mx + mx / 2 + 65536;
    size_t fb = 0, pb = 0;
    TIGAS_TRY(sliced_workspace(scene, req, cap, &fb, &pb));
    TIGAS_TRY(ctx.fixed.reserve(fb));
    TIGAS_TRY(ctx.pairs.reserve(pb));
    // capture on the context's own stream
    const uint64_t l0 = g_launches.load();
    TIGAS_CUDA_TRY(cudaStreamBeginCapture(ctx.stream, cudaStreamCaptureModeThreadLocal));
    FrameResult tmp_res;
    Status s = render_frame_sliced(scene, req, ctx, ctx.stream, &tmp_res, cap, nullptr);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx.stream, &graph);
    const uint64_t captured = g_launches.load() - l0;
    g_launches.fetch_sub(captured, std::memory_order_relaxed);   // captured, not run
    if (!s.ok()) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return {TIGAS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e)};
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return {TIGAS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)};
    RenderContext::Graph entry;
    entry.key = key;
    entry.exec = exec;
    entry.cap = cap;
    entry.launches = captured;
    entry.slices = req.n_slices < 1 ? 1 : (req.n_slices > kMaxSlices ? kMaxSlices : req.n_slices);
    entry.fixed_gen = ctx.fixed.gen;
    entry.pairs_gen = ctx.pairs.gen;
    entry.res = tmp_res;
    for (int k = 0; k < kNumStages; ++k) entry.ev_count[k] = ctx.ev_count[k];
    // nothing of the capture ran: the exact frame's events are the ones to read
    for (int k = 0; k < kNumStages; ++k) ctx.ev_count[k] = exact_counts[k];
    if (ctx.graphs.size() >= 8) {
        cudaGraphExecDestroy(ctx.graphs.front().exec);
        ctx.graphs.erase(ctx.graphs.begin());
    }
    ctx.graphs.push_back(entry);
    return {};
}

double pair_scale(const Scene* scene, const FrameRequest& req) {
    double s = 0.0;
    for (int v = 0; v < req.V; ++v) {
        const double f = std::sqrt((double)req.views[v].W * req.views[v].H / (1920.0 * 1080.0));
        s += (1.0 + 3.0 * f) * (1.0 + 3.0 * f) / 16.0;
    }
    return s * (double)scene->view.n;
}

void drop_graphs(RenderContext& ctx) {
    for (auto& g : ctx.graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    ctx.graphs.clear();
}

}  // namespace tigas
