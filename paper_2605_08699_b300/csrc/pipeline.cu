// Frame pipeline orchestration (host side of the hot path).
#include "pipeline.cuh"
#include "sliced.cuh"

#include <cmath>
#include <cstring>

namespace tigas {

std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_profile{false};

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

// ------------------------------------------------------------------ arena

Status Arena::reserve(size_t bytes) {
    if (bytes <= cap) return {};
    if (base) {
        cudaFree(base);
        base = nullptr;
        cap = 0;
    }
    size_t want = bytes + bytes / 4 + (1 << 20);
    cudaError_t e = cudaMalloc(&base, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        base = nullptr;
        e = cudaMalloc(&base, bytes);   // retry without headroom
        if (e != cudaSuccess) {
            cudaGetLastError();
            base = nullptr;
            return {TIGAS_ERR_OOM, "workspace allocation of " + std::to_string(bytes) + " bytes failed"};
        }
        want = bytes;
    }
    cap = want;
    used = 0;
    return {};
}

void Arena::release() {
    if (base) cudaFree(base);
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
    TIGAS_CUDA_TRY(cudaMallocHost(&h_total, sizeof(uint64_t) * 2));
    TIGAS_CUDA_TRY(cudaMallocHost(&h_flags, sizeof(uint32_t) * 2));
    TIGAS_CUDA_TRY(cudaMallocHost(&h_views, (sizeof(ViewParams) + sizeof(uint64_t)) * kMaxViews));
    TIGAS_CUDA_TRY(cudaMallocHost(&h_misc, sizeof(uint32_t) * kMaxViews));
    for (int k = 0; k < kNumStages; ++k)
        for (int r = 0; r < kMaxSlices; ++r) {
            TIGAS_CUDA_TRY(cudaEventCreate(&ev_start[k][r]));
            TIGAS_CUDA_TRY(cudaEventCreate(&ev_stop[k][r]));
        }
    return {};
}

void RenderContext::destroy() {
    fixed.release();
    pairs.release();
    for (auto* p : dev_staging)
        if (p) cudaFree(p);
    dev_staging.clear();
    staging_bytes.clear();
    if (h_total) cudaFreeHost(h_total);
    if (h_flags) cudaFreeHost(h_flags);
    if (h_views) cudaFreeHost(h_views);
    if (stream) cudaStreamDestroy(stream);
    for (int k = 0; k < kNumStages; ++k)
        for (int r = 0; r < kMaxSlices; ++r) {
            if (ev_start[k][r]) cudaEventDestroy(ev_start[k][r]);
            if (ev_stop[k][r]) cudaEventDestroy(ev_stop[k][r]);
            ev_start[k][r] = ev_stop[k][r] = nullptr;
        }
    if (h_misc) cudaFreeHost(h_misc);
    h_misc = nullptr;
    h_total = nullptr; h_flags = nullptr; h_views = nullptr; stream = nullptr;
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
    bool on;
    Status operator()(Stage sg, bool begin) {
        if (!on) return {};
        const int r = ctx.ev_count[sg];
        if (r >= kMaxSlices) return {};
        TIGAS_CUDA_TRY(cudaEventRecord(begin ? ctx.ev_start[sg][r] : ctx.ev_stop[sg][r], st));
        if (!begin) ctx.ev_count[sg] = r + 1;
        return {};
    }
};
}  // namespace

Status render_frame_sliced(Scene* scene, FrameRequest& req, RenderContext& ctx, cudaStream_t st, FrameResult* res);

Status render_frame(Scene* scene, FrameRequest& req, RenderContext& ctx, cudaStream_t st, FrameResult* res) {
    if (req.sort_mode == TIGAS_SORT_SLICED) return render_frame_sliced(scene, req, ctx, st, res);
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

    std::memcpy(ctx.h_views, req.views, sizeof(ViewParams) * V);
    TIGAS_CUDA_TRY(cudaMemcpyAsync(d_views, ctx.h_views, sizeof(ViewParams) * V, cudaMemcpyHostToDevice, st));
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
Status render_frame_sliced(Scene* scene, FrameRequest& req, RenderContext& ctx, cudaStream_t st, FrameResult* res) {
    for (int k = 0; k < kNumStages; ++k) ctx.ev_count[k] = 0;
    Marker mark{ctx, st, g_profile.load(std::memory_order_relaxed)};
    const int V = req.V;
    const uint32_t n = scene->view.n;
    const uint64_t E = (uint64_t)V * n;
    if (E >= 0xFFFFFFFFull) return {TIGAS_ERR_INVALID, "views x Gaussians exceeds 2^32 entries"};
    const int S = req.n_slices < 1 ? 1 : (req.n_slices > kMaxSlices ? kMaxSlices : req.n_slices);
    uint32_t total_tiles = 0;
    uint64_t pix_base_h[kMaxViews];
    uint64_t total_pix = 0;
    for (int v = 0; v < V; ++v) {
        req.views[v].tile_base = total_tiles;
        total_tiles += (uint32_t)(req.views[v].TX * req.views[v].TY);
        pix_base_h[v] = total_pix;
        total_pix += (uint64_t)req.views[v].W * req.views[v].H;
    }
    const int tile_bits = total_tiles <= 1 ? 1 : 32 - __builtin_clz(total_tiles - 1);
    const uint32_t done_words = (total_tiles + 31) / 32;

    // ---- per-entry and per-pixel workspace
    const size_t presort_words = radix_tmp_words(E);
    const size_t scan_words = scan_tmp_words(E + 1);
    const size_t tmp_words = presort_words > scan_words ? presort_words : scan_words;
    size_t fixed_bytes = sizeof(ViewParams) * kMaxViews + 80 * 256;
    fixed_bytes += E * (16 + 16 + 4 + 4 + 4 + 8 + (req.want_q ? 4 : 0));
    fixed_bytes += E * 4 * 4 + E * 4 * 2 + 8 + E * 8;     // depth sort buffers, counts, offsets, rects
    fixed_bytes += tmp_words * 4;
    fixed_bytes += (sizeof(uint2) + 4) * (size_t)total_tiles + done_words * 4;
    fixed_bytes += total_pix * 16 + sizeof(uint64_t) * kMaxViews;
    TIGAS_TRY(ctx.fixed.reserve(fixed_bytes));
    ctx.fixed.reset();
    ViewParams* d_views = ctx.fixed.take<ViewParams>(kMaxViews);
    uint64_t* d_total = ctx.fixed.take<uint64_t>(2);
    unsigned long long* d_counters = ctx.fixed.take<unsigned long long>(4);
    uint32_t* d_flags = ctx.fixed.take<uint32_t>(2);
    uint32_t* d_visible = ctx.fixed.take<uint32_t>(kMaxViews);
    uint32_t* d_misc = ctx.fixed.take<uint32_t>(4);       // [n_active, work counter]
    uint64_t* d_pix_base = ctx.fixed.take<uint64_t>(kMaxViews);
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
    uint32_t* counts = ctx.fixed.take<uint32_t>(E + 1);
    uint32_t* offsets = ctx.fixed.take<uint32_t>(E + 1);
    uint2* rect_sorted = ctx.fixed.take<uint2>(E);
    uint32_t* tmp = ctx.fixed.take<uint32_t>(tmp_words);
    uint2* ranges = ctx.fixed.take<uint2>(total_tiles);
    uint32_t* active = ctx.fixed.take<uint32_t>(total_tiles);
    uint32_t* done = ctx.fixed.take<uint32_t>(done_words);
    float4* state = ctx.fixed.take<float4>(total_pix);

    std::memcpy(ctx.h_views, req.views, sizeof(ViewParams) * V);
    TIGAS_CUDA_TRY(cudaMemcpyAsync(d_views, ctx.h_views, sizeof(ViewParams) * V, cudaMemcpyHostToDevice, st));
    std::memcpy(reinterpret_cast<char*>(ctx.h_views) + sizeof(ViewParams) * V, pix_base_h, sizeof(uint64_t) * V);
    TIGAS_CUDA_TRY(cudaMemcpyAsync(d_pix_base, reinterpret_cast<char*>(ctx.h_views) + sizeof(ViewParams) * V,
                                   sizeof(uint64_t) * V, cudaMemcpyHostToDevice, st));
    TIGAS_CUDA_TRY(cudaMemsetAsync(d_flags, 0, sizeof(uint32_t) * 2, st));
    TIGAS_CUDA_TRY(cudaMemsetAsync(done, 0, done_words * 4, st));
    if (sp.q_dbg) TIGAS_CUDA_TRY(cudaMemsetAsync(sp.q_dbg, 0, E * 4, st));
    if (req.want_counters) TIGAS_CUDA_TRY(cudaMemsetAsync(d_counters, 0, sizeof(unsigned long long) * 4, st));

    TIGAS_TRY(mark(kStPreprocess, true));
    TIGAS_TRY(launch_preprocess(scene->view, d_views, V, sp, d_visible, st));
    TIGAS_TRY(mark(kStPreprocess, false));
    TIGAS_TRY(mark(kStDepthSort, true));
    TIGAS_TRY(radix_sort<uint32_t>(sp.depth_key, nullptr, pk_alt, pv_alt, pk, order, E, nullptr, 0, 32, tmp, st,
                                   nullptr, d_flags));
    TIGAS_TRY(mark(kStDepthSort, false));
    TIGAS_TRY(launch_init_state(d_views, V, total_tiles, d_pix_base, state, scene->view.bg, st));
    // kept entries: culled ones (depth key 0xFFFFFFFF) sort after all kept ones
    TIGAS_CUDA_TRY(cudaMemcpyAsync(ctx.h_misc, d_visible, sizeof(uint32_t) * V, cudaMemcpyDeviceToHost, st));
    TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
    uint64_t K = 0;
    for (int v = 0; v < V; ++v) K += ctx.h_misc[v];
    TIGAS_TRY(mark(kStScan, true));
    TIGAS_TRY(launch_permute_rects(order, K, sp, n, rect_sorted, st));
    TIGAS_TRY(mark(kStScan, false));

    // geometric slice ends: K / 64 ... K
    uint64_t ends[kMaxSlices];
    for (int i = 0; i < S; ++i) {
        const double f = S == 1 ? 1.0 : std::pow(64.0, (double)(i - (S - 1)) / (double)(S - 1));
        ends[i] = i == S - 1 ? K : (uint64_t)std::ceil(f * (double)K);
    }
    uint64_t total_pairs = 0;
    int passes = 0;
    uint64_t a = 0;
    SliceBlendArgs sl{active, d_misc, d_misc + 1, state, d_pix_base, done};
    for (int i = 0; i < S; ++i) {
        const uint64_t b = ends[i] > a ? ends[i] : a;
        if (b == a) continue;
        TIGAS_TRY(mark(kStScan, true));
        TIGAS_TRY(launch_count_slice(rect_sorted, a, b, d_views, V, done, counts, st));
        // one extra zero count makes offsets[b - a] the slice total
        TIGAS_CUDA_TRY(cudaMemsetAsync(counts + (b - a), 0, sizeof(uint32_t), st));
        TIGAS_TRY(launch_scan_u32(counts, nullptr, offsets, b - a + 1, d_total, tmp, st));
        TIGAS_TRY(mark(kStScan, false));
        TIGAS_CUDA_TRY(cudaMemcpyAsync(ctx.h_total, d_total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
        const uint64_t P = ctx.h_total[0];
        if (P >= 0xFFFFFFFFull) return {TIGAS_ERR_OVERFLOW, "pair count exceeds 2^32"};
        if (P > 0) {
            total_pairs += P;
            const size_t sort_words = radix_tmp_words(P);
            TIGAS_TRY(ctx.pairs.reserve(P * 24 + sort_words * 4 + 8 * 256));
            ctx.pairs.reset();
            uint32_t* keys_a = ctx.pairs.take<uint32_t>(P);
            uint32_t* keys_b = ctx.pairs.take<uint32_t>(P);
            uint32_t* keys_c = ctx.pairs.take<uint32_t>(P);
            uint32_t* vals_a = ctx.pairs.take<uint32_t>(P);
            uint32_t* vals_b = ctx.pairs.take<uint32_t>(P);
            uint32_t* vals_c = ctx.pairs.take<uint32_t>(P);
            uint32_t* stmp = ctx.pairs.take<uint32_t>(sort_words);
            TIGAS_TRY(mark(kStEmit, true));
            TIGAS_TRY(launch_emit_slice(order, rect_sorted, a, b, offsets, d_views, V, done, keys_a, vals_a, P, d_flags,
                                        st));
            TIGAS_TRY(mark(kStEmit, false));
            TIGAS_TRY(mark(kStPairSort, true));
            TIGAS_TRY(radix_sort<uint32_t>(keys_a, vals_a, keys_b, vals_b, keys_c, vals_c, P, nullptr, 0, tile_bits,
                                           stmp, st, &passes, d_flags));
            TIGAS_TRY(mark(kStPairSort, false));
            TIGAS_TRY(mark(kStRanges, true));
            TIGAS_TRY(launch_ranges_active(keys_c, P, ranges, total_tiles, done, active, d_misc, d_flags, st));
            TIGAS_TRY(mark(kStRanges, false));
            TIGAS_TRY(mark(kStBlend, true));
            TIGAS_TRY(launch_blend_slice(ranges, vals_c, sp, d_views, V, (uint32_t)E, scene->view.bg,
                                         req.want_counters ? d_counters : nullptr, sl, st));
            TIGAS_TRY(mark(kStBlend, false));
        }
        a = b;
    }
    TIGAS_CUDA_TRY(cudaMemcpyAsync(ctx.h_flags, d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    if (res) {
        res->pairs = total_pairs;
        res->total_tiles = total_tiles;
        res->sort_passes = passes;
        res->values = nullptr;
        res->ranges = nullptr;
        res->splats = sp;
        res->d_visible = d_visible;
        res->d_counters = req.want_counters ? d_counters : nullptr;
    }
    return {};
}

}  // namespace tigas
