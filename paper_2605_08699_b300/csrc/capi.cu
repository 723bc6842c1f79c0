// C ABI entry points (include/tigas.h): argument validation, host/device
// buffer handling and error reporting around the frame pipeline.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pipeline.cuh"

#define TIGAS_API extern "C" __attribute__((visibility("default")))

namespace tigas {

namespace {
thread_local std::string t_last_error;
}

void set_error(const std::string& msg) { t_last_error = msg; }
const char* last_error() { return t_last_error.c_str(); }

tigas_status fail(const Status& s) {
    set_error(s.msg);
    return s.code;
}
tigas_status fail(tigas_status code, const std::string& msg) {
    set_error(msg);
    return code;
}

Status validate_view(const tigas_pose* pose, const tigas_intrinsics* k, int w, int h) {
    if (!pose || !k) return {TIGAS_ERR_INVALID, "null pose or intrinsics"};
    if (!std::isfinite(pose->azimuth) || !std::isfinite(pose->elevation) || !std::isfinite(pose->t[0]) ||
        !std::isfinite(pose->t[1]) || !std::isfinite(pose->t[2]))
        return {TIGAS_ERR_INVALID, "non-finite pose"};
    if (!(std::isfinite(k->fx) && std::isfinite(k->fy) && std::isfinite(k->cx) && std::isfinite(k->cy)) ||
        !(k->fx > 0) || !(k->fy > 0))
        return {TIGAS_ERR_INVALID, "intrinsics must be finite with fx, fy > 0"};
    if (w < 1 || h < 1 || w > kMaxDim || h > kMaxDim) return {TIGAS_ERR_INVALID, "width/height out of 1..8192"};
    return {};
}

// Device buffer for a host output, grown on demand (one slot per output).
Status staging(RenderContext& ctx, int slot, size_t bytes, uint8_t** out) {
    if ((int)ctx.dev_staging.size() <= slot) {
        ctx.dev_staging.resize(slot + 1, nullptr);
        ctx.staging_bytes.resize(slot + 1, 0);
    }
    if (ctx.staging_bytes[slot] < bytes) {
        if (ctx.dev_staging[slot]) cudaFree(ctx.dev_staging[slot]);
        ctx.dev_staging[slot] = nullptr;
        ctx.staging_bytes[slot] = 0;
        TIGAS_CUDA_TRY(device_alloc(&ctx.dev_staging[slot], bytes));
        ctx.staging_bytes[slot] = bytes;
    }
    *out = ctx.dev_staging[slot];
    return {};
}

struct ContextGuard {
    RenderContext* ctx = nullptr;
    ~ContextGuard() {
        if (ctx) release_context(ctx);
    }
};

struct SceneGuard {
    Scene* s = nullptr;
    explicit SceneGuard(Scene* sc) : s(sc) {
        if (s) scene_acquire(s);
    }
    ~SceneGuard() {
        if (s) scene_release(s);
    }
};

// A launch set between its submission and its completion.
struct PendingRender {
    Scene* scene = nullptr;
    int V = 0;
    int sort_mode = TIGAS_SORT_SLICED;
    FrameRequest req;
    FrameResult res;
    std::vector<uint8_t*> host8;
    std::vector<float*> host32;
    std::vector<int> ws, hs;
};

// Validate and enqueue V views on st (host outputs go through device staging
// and are copied back on st).  Returns with the work in flight.
// copy_st: stream for the device-to-host copies of host outputs (it waits for
// the launch set; null: st itself).
Status submit_render(RenderContext& ctx, Scene* scene, int V, const tigas_pose* poses, const tigas_intrinsics* intrs,
                     const int* ws, const int* hs, uint8_t* const* outs8, float* const* outs32, cudaStream_t st,
                     int sort_mode, bool want_stats, bool want_q, PendingRender& p, cudaStream_t copy_st = nullptr) {
    if (!scene) return {TIGAS_ERR_INVALID, "null scene"};
    if (V < 1 || V > kMaxViews) return {TIGAS_ERR_INVALID, "n_views out of 1..64"};
    if (sort_mode != TIGAS_SORT_DEPTH_FIRST && sort_mode != TIGAS_SORT_FULL64 && sort_mode != TIGAS_SORT_SLICED)
        return {TIGAS_ERR_INVALID, "unknown sort mode"};
    for (int v = 0; v < V; ++v) TIGAS_TRY(validate_view(&poses[v], &intrs[v], ws[v], hs[v]));
    p.scene = scene;
    p.V = V;
    p.sort_mode = sort_mode;
    p.ws.assign(ws, ws + V);
    p.hs.assign(hs, hs + V);
    FrameRequest& req = p.req;
    req.V = V;
    req.sort_mode = sort_mode;
    const Schedule sched = current_schedule(V);
    req.n_slices = sched.n_slices;
    req.first_slice_inv = sched.first_slice_inv;
    req.blend_ctas_per_sm = sched.blend_ctas_per_sm;
    req.blend_batch = sched.blend_batch;
    req.want_q = want_q;
    req.want_counters = want_stats;
    p.host8.assign(V, nullptr);
    p.host32.assign(V, nullptr);
    for (int v = 0; v < V; ++v) {
        req.views[v] = make_view(poses[v], intrs[v], ws[v], hs[v], 0);
        const size_t px = (size_t)ws[v] * hs[v];
        uint8_t* o8 = outs8 ? outs8[v] : nullptr;
        float* o32 = outs32 ? outs32[v] : nullptr;
        if (o8 && !is_device_pointer(o8)) {
            p.host8[v] = o8;
            TIGAS_TRY(staging(ctx, 2 * v, px * 4, &o8));
        }
        if (o32 && !is_device_pointer(o32)) {
            p.host32[v] = o32;
            uint8_t* q = nullptr;
            TIGAS_TRY(staging(ctx, 2 * v + 1, px * 16, &q));
            o32 = reinterpret_cast<float*>(q);
        }
        req.views[v].out_rgba8 = o8;
        req.views[v].out_rgba_f32 = o32;
    }
    bool done = false;
    const bool try_graph = sort_mode == TIGAS_SORT_SLICED && !want_q && g_use_graphs.load();
    if (try_graph) TIGAS_TRY(render_sliced_graph(scene, req, ctx, st, &p.res, &done));
    if (!done) TIGAS_TRY(render_frame(scene, req, ctx, st, &p.res));
    cudaStream_t cs = st;
    if (copy_st) {
        TIGAS_CUDA_TRY(cudaEventRecord(ctx.ev_rendered, st));
        TIGAS_CUDA_TRY(cudaStreamWaitEvent(copy_st, ctx.ev_rendered, 0));
        cs = copy_st;
    }
    for (int v = 0; v < V; ++v) {
        const size_t px = (size_t)ws[v] * hs[v];
        if (p.host8[v])
            TIGAS_CUDA_TRY(cudaMemcpyAsync(p.host8[v], req.views[v].out_rgba8, px * 4, cudaMemcpyDeviceToHost, cs));
        if (p.host32[v])
            TIGAS_CUDA_TRY(
                cudaMemcpyAsync(p.host32[v], req.views[v].out_rgba_f32, px * 16, cudaMemcpyDeviceToHost, cs));
    }
    return {};
}

// After the submitted work completed: timing, and an exact re-render when a
// fixed-capacity launch set outgrew its pair buffers.
Status finish_render(RenderContext& ctx, cudaStream_t st, PendingRender& p) {
    FrameResult& res = p.res;
    collect_profile(ctx);
    if (res.graph_slices > 0) {
        if (ctx.h_flags[0] & 1u) {
            // a slice outgrew the fixed pair capacity: render this frame exactly;
            // a graph is captured again (with the new counts) on the next call,
            // a direct launch set takes a larger capacity next time
            if (res.direct_static)
                ctx.slice_ratio(p.req.n_slices, p.req.first_slice_inv) *= 2.0;
            else
                drop_graphs(ctx);
            g_exact_rerenders.fetch_add(1, std::memory_order_relaxed);
            TIGAS_TRY(render_frame(p.scene, p.req, ctx, st, &res));
            for (int v = 0; v < p.V; ++v) {
                const size_t px = (size_t)p.ws[v] * p.hs[v];
                if (p.host8[v])
                    TIGAS_CUDA_TRY(
                        cudaMemcpyAsync(p.host8[v], p.req.views[v].out_rgba8, px * 4, cudaMemcpyDeviceToHost, st));
                if (p.host32[v])
                    TIGAS_CUDA_TRY(cudaMemcpyAsync(p.host32[v], p.req.views[v].out_rgba_f32, px * 16,
                                                   cudaMemcpyDeviceToHost, st));
            }
            TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
            collect_profile(ctx);
        } else {
            uint64_t P = 0, mx = 0;
            for (int i = 0; i < res.graph_slices; ++i) {
                P += ctx.h_total[i];
                mx = ctx.h_total[i] > mx ? ctx.h_total[i] : mx;
            }
            res.pairs = P;
            const double scale = pair_scale(p.scene, p.req);
            double& ratio = ctx.slice_ratio(p.req.n_slices, p.req.first_slice_inv);
            if (scale > 0.0 && (double)mx / scale > ratio) ratio = (double)mx / scale;
        }
    }
    if (ctx.h_flags[0] & 1u) return {TIGAS_ERR_OVERFLOW, "pair buffer overflow"};
    if (ctx.h_flags[0] & 2u) return {TIGAS_ERR_CUDA, "tile id out of range in sorted keys"};
    if (ctx.h_flags[0] & kSortTimeoutFlag) return {TIGAS_ERR_TIMEOUT, "radix sort look-back wait ran out"};
    return {};
}

// Render V views synchronously; outputs may be host or device.  dbg_pairs
// (optional) receives the launch set's pair count; stats turns on the
// instrumented kernels.
Status do_render(Scene* scene, int V, const tigas_pose* poses, const tigas_intrinsics* intrs, const int* ws,
                 const int* hs, uint8_t* const* outs8, float* const* outs32, cudaStream_t user_st, int sort_mode,
                 tigas_frame_stats* stats, tigas_debug_frame* dbg, uint64_t* dbg_pairs) {
    if (dbg && sort_mode == TIGAS_SORT_SLICED && (dbg->values || dbg->ranges))
        return {TIGAS_ERR_INVALID, "the sliced schedule builds no whole tile lists: pass values = ranges = NULL"};
    if (!scene) return {TIGAS_ERR_INVALID, "null scene"};
    if (V < 1 || V > kMaxViews) return {TIGAS_ERR_INVALID, "n_views out of 1..64"};
    for (int v = 0; v < V; ++v) TIGAS_TRY(validate_view(&poses[v], &intrs[v], ws[v], hs[v]));
    Status err;
    ContextGuard g;
    g.ctx = acquire_context(&err);
    if (!g.ctx) return err;
    RenderContext& ctx = *g.ctx;
    cudaStream_t st = user_st ? user_st : ctx.stream;
    PendingRender p;
    TIGAS_TRY(submit_render(ctx, scene, V, poses, intrs, ws, hs, outs8, outs32, st, sort_mode, stats != nullptr,
                            dbg != nullptr, p));
    TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
    TIGAS_TRY(finish_render(ctx, st, p));
    FrameResult& res = p.res;
    if (dbg_pairs && !dbg) *dbg_pairs = res.pairs;   // the pair count alone, without instrumented kernels

    if (stats) {
        uint32_t vis[kMaxViews];
        TIGAS_CUDA_TRY(cudaMemcpy(vis, res.d_visible, sizeof(uint32_t) * V, cudaMemcpyDeviceToHost));
        uint64_t nv = 0;
        for (int v = 0; v < V; ++v) nv += vis[v];
        stats->n_visible = nv;
        stats->n_pairs = res.pairs;
        stats->n_tiles = res.total_tiles;
        stats->sort_passes = (uint32_t)res.sort_passes;
        unsigned long long cnt[3] = {0, 0, 0};
        if (res.d_counters) TIGAS_CUDA_TRY(cudaMemcpy(cnt, res.d_counters, sizeof(cnt), cudaMemcpyDeviceToHost));
        stats->blend_evals = cnt[0];
        stats->blend_fetched = cnt[1];
        stats->blend_contribs = cnt[2];
        stats->depth_sort_passes = sort_mode == TIGAS_SORT_SLICED ? ctx.h_flags[1] : 0u;
        const uint64_t near = res.near_split ? (uint64_t)ctx.h_flags[2] | ((uint64_t)ctx.h_flags[3] << 32)
                                             : res.entries;
        stats->depth_sort_near = sort_mode == TIGAS_SORT_SLICED ? (uint32_t)near : 0u;
    }
    if (dbg) {
        const uint32_t n = scene->view.n;
        if (dbg_pairs) *dbg_pairs = res.pairs;
        std::vector<uint32_t> tiles(n), dkey(n);
        std::vector<uint2> rect(n);
        std::vector<float4> geom(n);
        std::vector<float> q(n);
        TIGAS_CUDA_TRY(cudaMemcpy(tiles.data(), res.splats.tiles, n * 4ull, cudaMemcpyDeviceToHost));
        TIGAS_CUDA_TRY(cudaMemcpy(dkey.data(), res.splats.depth_key, n * 4ull, cudaMemcpyDeviceToHost));
        TIGAS_CUDA_TRY(cudaMemcpy(rect.data(), res.splats.rect, n * 8ull, cudaMemcpyDeviceToHost));
        TIGAS_CUDA_TRY(cudaMemcpy(geom.data(), res.splats.geom, n * 16ull, cudaMemcpyDeviceToHost));
        TIGAS_CUDA_TRY(cudaMemcpy(q.data(), res.splats.q_dbg, n * 4ull, cudaMemcpyDeviceToHost));
        for (uint32_t i = 0; i < n; ++i) {
            const bool vis = tiles[i] > 0;
            if (dbg->visible) dbg->visible[i] = vis ? 1 : 0;
            if (dbg->radius) dbg->radius[i] = vis ? (int32_t)ceilf(q[i]) : 0;
            if (dbg->rect) {
                int32_t* r = dbg->rect + 4 * (size_t)i;
                if (vis) {
                    r[0] = rect[i].x & 0x3FF; r[1] = rect[i].y & 0x3FF;
                    r[2] = (rect[i].x >> 10) & 0x3FF; r[3] = (rect[i].y >> 10) & 0x3FF;
                } else {
                    r[0] = r[1] = r[2] = r[3] = 0;
                }
            }
            if (dbg->depth) {
                float d;
                std::memcpy(&d, &dkey[i], 4);
                dbg->depth[i] = vis ? d : 0.0f;
            }
            if (dbg->uv) {
                dbg->uv[2 * (size_t)i] = vis ? geom[i].x : 0.0f;
                dbg->uv[2 * (size_t)i + 1] = vis ? geom[i].y : 0.0f;
            }
            if (dbg->q) dbg->q[i] = q[i];
        }
        if (dbg->values && res.values && res.pairs <= dbg->pair_capacity && res.pairs)
            TIGAS_CUDA_TRY(cudaMemcpy(dbg->values, res.values, res.pairs * 4, cudaMemcpyDeviceToHost));
        if (dbg->ranges && res.ranges)
            TIGAS_CUDA_TRY(cudaMemcpy(dbg->ranges, res.ranges, (size_t)res.total_tiles * 8, cudaMemcpyDeviceToHost));
    }
    return {};
}

}  // namespace tigas

using namespace tigas;

TIGAS_API const char* tigas_last_error(void) { return last_error(); }
TIGAS_API tigas_status tigas_set_graphs(int enable) {
    g_use_graphs.store(enable != 0);
    forget_launch_sets();
    return TIGAS_OK;
}

namespace {
Status check_schedule(const tigas_schedule* s) {
    if (!s) return {TIGAS_ERR_INVALID, "null schedule"};
    if (s->n_slices < 1 || s->n_slices > kMaxSlices) return {TIGAS_ERR_INVALID, "n_slices out of 1..16"};
    if (s->first_slice_inv < 1 || s->first_slice_inv > 4096) return {TIGAS_ERR_INVALID, "first_slice_inv out of 1..4096"};
    if (s->blend_ctas_per_sm < 0 || s->blend_ctas_per_sm > 64) return {TIGAS_ERR_INVALID, "blend_ctas_per_sm out of 0..64"};
    if (s->blend_batch != 0 && s->blend_batch != 16 && s->blend_batch != 32)
        return {TIGAS_ERR_INVALID, "blend_batch must be 0, 16 or 32"};
    if (s->views_per_set < 0 || s->views_per_set > kMaxViews) return {TIGAS_ERR_INVALID, "views_per_set out of 0..64"};
    return {};
}
}  // namespace

namespace {
Schedule to_schedule(const tigas_schedule* s) {
    return Schedule{s->n_slices, s->first_slice_inv, s->blend_ctas_per_sm, s->blend_batch ? s->blend_batch : 32,
                    s->views_per_set};
}
void from_schedule(const Schedule& c, tigas_schedule* s) {
    s->n_slices = c.n_slices;
    s->first_slice_inv = c.first_slice_inv;
    s->blend_ctas_per_sm = c.blend_ctas_per_sm;
    s->blend_batch = c.blend_batch;
    s->views_per_set = c.views_per_set;
}
}  // namespace

TIGAS_API tigas_status tigas_set_schedule(const tigas_schedule* s) {
    Status c = check_schedule(s);
    if (!c.ok()) return fail(c);
    set_schedule(to_schedule(s));
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_set_schedule_for_views(int n_views, const tigas_schedule* s) {
    if (n_views < 1 || n_views > kMaxViews) return fail(TIGAS_ERR_INVALID, "n_views out of 1..64");
    Status c = check_schedule(s);
    if (!c.ok()) return fail(c);
    set_schedule_for(n_views, to_schedule(s));
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_get_schedule(int n_views, tigas_schedule* s) {
    if (!s) return fail(TIGAS_ERR_INVALID, "null schedule");
    if (n_views < 1 || n_views > kMaxViews) return fail(TIGAS_ERR_INVALID, "n_views out of 1..64");
    from_schedule(current_schedule(n_views), s);
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_autotune(tigas_scene* scene, int n_sets, int n_views, const tigas_pose* poses,
                                      const tigas_intrinsics* intrs, const int* widths, const int* heights,
                                      uint8_t* const* outs_rgba8, int iters, tigas_schedule* best,
                                      double* best_ms) {
    if (!scene || !poses || !intrs || !widths || !heights || !outs_rgba8) return fail(TIGAS_ERR_INVALID, "null argument");
    if (n_views < 1 || n_views > kMaxViews) return fail(TIGAS_ERR_INVALID, "n_views out of 1..64");
    if (n_sets < 1 || n_sets > 1024) return fail(TIGAS_ERR_INVALID, "n_sets out of 1..1024");
    if (iters < 1 || iters > 100) return fail(TIGAS_ERR_INVALID, "iters out of 1..100");
    for (int v = 0; v < n_views; ++v)
        if (!outs_rgba8[v] || !is_device_pointer(outs_rgba8[v]))
            return fail(TIGAS_ERR_INVALID, "autotune outputs must be device buffers");
    Scene* sc = reinterpret_cast<Scene*>(scene);
    SceneGuard sg(sc);
    // every class's schedule, restored on failure (the call sets only the classes it times)
    Schedule saved[kScheduleClasses];
    for (int c = 0; c < kScheduleClasses; ++c) saved[c] = current_schedule(1 << c);
    const Schedule own = current_schedule(n_views);
    static const int kSlices[] = {1, 2, 3, 4, 5, 6, 7, 8, 12};
    static const int kFirst[] = {8, 16, 32, 64, 128, 256};
    static const int kCtas[] = {0, 4};
    static const int kBatch[] = {32, 16};
    std::vector<Schedule> cands;
    for (int ns : kSlices)
        for (int fi : kFirst) {
            if (ns == 1 && fi != kFirst[0]) continue;   // one slice holds every entry whatever the first fraction
            for (int ct : kCtas)
                for (int wb : kBatch) cands.push_back(Schedule{ns, fi, ct, wb, own.views_per_set});
        }
    std::vector<std::vector<double>> times(cands.size());
    int next_set = 0;
    // the next pose set's views [v0, v0 + m) as one launch set; returns host ms
    // device time of a launch set: events on the render stream around its work (the
    // measure that back-to-back launch sets run at; host time adds the launch and the wait)
    struct Timing {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Timing() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } tm;
    {
        cudaError_t e = cudaEventCreate(&tm.e0);
        if (e == cudaSuccess) e = cudaEventCreate(&tm.e1);
        if (e != cudaSuccess) return fail(TIGAS_ERR_CUDA, std::string("autotune events: ") + cudaGetErrorString(e));
    }
    auto render_part = [&](int v0, int m, double* ms) -> Status {
        const size_t off = (size_t)next_set * n_views + v0;
        Status err;
        ContextGuard g;
        g.ctx = acquire_context(&err);
        if (!g.ctx) return err;
        RenderContext& ctx = *g.ctx;
        PendingRender p;
        TIGAS_CUDA_TRY(cudaEventRecord(tm.e0, ctx.stream));
        TIGAS_TRY(submit_render(ctx, sc, m, poses + off, intrs + off, widths + v0, heights + v0, outs_rgba8 + v0,
                                nullptr, ctx.stream, TIGAS_SORT_SLICED, false, false, p));
        TIGAS_CUDA_TRY(cudaEventRecord(tm.e1, ctx.stream));
        TIGAS_CUDA_TRY(cudaStreamSynchronize(ctx.stream));
        TIGAS_TRY(finish_render(ctx, ctx.stream, p));
        float f = 0.0f;
        TIGAS_CUDA_TRY(cudaEventElapsedTime(&f, tm.e0, tm.e1));
        *ms = f;
        return {};
    };
    // one launch set of all views (the next pose set) under schedule c; untimed ones
    // warm up (a shape's first launch set runs directly, the second is captured)
    auto run = [&](size_t c, bool timed) -> Status {
        set_schedule_for(n_views, cands[c]);
        double ms = 0.0;
        Status s = render_part(0, n_views, &ms);
        next_set = (next_set + 1) % n_sets;
        if (timed) times[c].push_back(ms);
        return s;
    };
    auto median = [](std::vector<double> t) {
        std::sort(t.begin(), t.end());
        return t.empty() ? 1e300 : t[t.size() / 2];
    };
    auto restore = [&]() {
        for (int c = 0; c < kScheduleClasses; ++c) set_schedule_for(1 << c, saved[c]);
    };
    auto give_up = [&](const Status& s) {
        restore();
        return fail(s);
    };
    // first pass: every candidate, two untimed then `iters` timed launch sets
    for (size_t c = 0; c < cands.size(); ++c)
        for (int it = 0; it < iters + 2; ++it) {
            Status s = run(c, it >= 2);
            if (!s.ok()) return give_up(s);
        }
    // second pass: the four fastest again, interleaved so that drift hits them alike
    std::vector<size_t> order(cands.size());
    for (size_t c = 0; c < cands.size(); ++c) order[c] = c;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return median(times[a]) < median(times[b]); });
    order.resize(std::min<size_t>(4, order.size()));
    for (size_t c : order) times[c].clear();
    for (int round = 0; round < 2 * iters + 1; ++round)
        for (size_t c : order) {
            Status s = run(c, true);
            if (!s.ok()) return give_up(s);
        }
    Schedule win = own;
    double win_ms = 1e300;
    for (size_t c : order) {
        const double m = median(times[c]);
        if (m < win_ms) {
            win_ms = m;
            win = cands[c];
        }
    }
    // views per launch set under the winning schedule: the pose set's views as
    // n_views / m launch sets of m (each taking the winner too), time per view
    int win_m = n_views;
    double win_per_view = 1e300;
    for (int m = n_views; m >= 1; m /= 2) {
        if (n_views % m != 0) continue;
        restore();
        set_schedule_for(m, win);
        std::vector<double> per_view;
        for (int round = 0; round < 2 * iters + 3; ++round) {
            double total = 0.0;
            for (int v0 = 0; v0 < n_views; v0 += m) {
                double ms = 0.0;
                Status s = render_part(v0, m, &ms);
                if (!s.ok()) return give_up(s);
                total += ms;
            }
            next_set = (next_set + 1) % n_sets;
            if (round >= 2) per_view.push_back(total / n_views);
        }
        const double med = median(per_view);
        if (med < win_per_view) {
            win_per_view = med;
            win_m = m;
        }
        if (m == 1) break;
    }
    // the class of n_views takes the winner and the views per launch set; a smaller
    // winning launch set size takes the winner too (it was timed with it)
    restore();
    if (win_m < n_views) {
        Schedule w = win;
        w.views_per_set = current_schedule(win_m).views_per_set;
        set_schedule_for(win_m, w);
    }
    win.views_per_set = win_m;
    set_schedule_for(n_views, win);
    if (best) from_schedule(win, best);
    if (best_ms) *best_ms = win_ms;
    return TIGAS_OK;
}

TIGAS_API uint64_t tigas_exact_rerenders(void) { return g_exact_rerenders.load(); }

TIGAS_API tigas_status tigas_jpeg_encode(const uint8_t* rgba, int width, int height, int quality, int restart_mcus,
                                         uint8_t* out, uint64_t out_capacity, uint64_t* out_len, void* cuda_stream) {
    if (!rgba || !out || !out_len) return fail(TIGAS_ERR_INVALID, "null argument");
    Status err;
    ContextGuard g;
    g.ctx = acquire_context(&err);
    if (!g.ctx) return fail(err);
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : g.ctx->stream;
    Status s = jpeg_encode(*g.ctx, rgba, width, height, quality, restart_mcus, out, out_capacity, out_len, st);
    return s.ok() ? TIGAS_OK : fail(s);
}

TIGAS_API tigas_status tigas_resample_rgba8(const uint8_t* src, int w, int h, uint8_t* dst, int width, int height,
                                            void* cuda_stream) {
    Status err;
    ContextGuard g;
    g.ctx = acquire_context(&err);
    if (!g.ctx) return fail(err);
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : g.ctx->stream;
    Status s = resample_rgba8(*g.ctx, src, w, h, dst, width, height, st);
    return s.ok() ? TIGAS_OK : fail(s);
}

TIGAS_API tigas_status tigas_image_quality(const uint8_t* a, const uint8_t* b, int width, int height, float* out_map,
                                           double* out_ssim, double* out_psnr, void* cuda_stream) {
    Status err;
    ContextGuard g;
    g.ctx = acquire_context(&err);
    if (!g.ctx) return fail(err);
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : g.ctx->stream;
    Status s = image_quality(*g.ctx, a, b, width, height, out_map, out_ssim, out_psnr, st);
    return s.ok() ? TIGAS_OK : fail(s);
}

TIGAS_API tigas_status tigas_debug_fail_alloc(int kind, int64_t nth, int64_t count) {
    set_error("");
    if (kind != 0 && kind != 1) return fail(TIGAS_ERR_INVALID, "kind must be 0 (device) or 1 (pinned host)");
    if (nth < 0 || count < 0 || (nth > 0 && count < 1)) return fail(TIGAS_ERR_INVALID, "nth >= 0, count >= 1");
    inject_alloc_failures(kind, nth, count);
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_release_workspace(void) {
    set_error("");
    release_idle_contexts();
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_debug_sort_wait_timeout(int spin_limit) {
    bool timed_out = false;
    Status s = debug_lookback_timeout(spin_limit, &timed_out);
    if (!s.ok()) return fail(s);
    if (timed_out) return fail(TIGAS_ERR_TIMEOUT, "radix sort look-back wait ran out");
    return TIGAS_OK;
}

TIGAS_API const char* tigas_version(void) { return "tigas-b300 0.1 (sm_103a)"; }
TIGAS_API uint64_t tigas_kernel_launches(void) { return g_launches.load(); }

TIGAS_API tigas_status tigas_profile_enable(int enable) {
    g_profile.store(enable != 0 ? (1u << kNumStages) - 1u : 0u);
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_profile_stages(uint32_t mask) {
    if (mask >> kNumStages) return fail(TIGAS_ERR_INVALID, "stage mask has bits past the last stage");
    g_profile.store(mask);
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_profile_read(double* ms, uint64_t* calls, int reset) {
    profile_read(ms, calls, reset != 0);
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_scene_load(const tigas_scene_desc* d, tigas_scene** out) {
    set_error("");
    if (!d || !out) return fail(TIGAS_ERR_INVALID, "null argument");
    *out = nullptr;
    if (d->n < 1 || d->n > (1ull << 27)) return fail(TIGAS_ERR_INVALID, "n out of 1..2^27");
    if (d->sh_degree < 0 || d->sh_degree > 3) return fail(TIGAS_ERR_INVALID, "sh_degree out of 0..3");
    if (d->storage != TIGAS_STORAGE_FP32 && d->storage != TIGAS_STORAGE_FP16)
        return fail(TIGAS_ERR_INVALID, "unknown storage");
    if (!d->means || !d->log_scales || !d->quats || !d->opacity_logits || !d->sh)
        return fail(TIGAS_ERR_INVALID, "null attribute array");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(d->background[c])) return fail(TIGAS_ERR_INVALID, "non-finite background");
    const uint32_t n = (uint32_t)d->n;
    const float *m = d->means, *ls = d->log_scales, *q = d->quats, *op = d->opacity_logits, *sh = d->sh;
    float* staging_buf = nullptr;
    auto finish = [&](const Status& st) -> tigas_status {
        if (staging_buf) cudaFree(staging_buf);
        return st.ok() ? TIGAS_OK : fail(st);
    };
    if (!d->inputs_on_device) {
        const size_t words = (size_t)n * (3 + 3 + 4 + 1 + 48);
        cudaError_t e = device_alloc(&staging_buf, words * 4);
        if (e != cudaSuccess) {
            cudaGetLastError();
            staging_buf = nullptr;
            return finish({TIGAS_ERR_OOM, "staging allocation failed"});
        }
        float* p = staging_buf;
        const float* src[5] = {m, ls, q, op, sh};
        const size_t len[5] = {3ull * n, 3ull * n, 4ull * n, 1ull * n, 48ull * n};
        const float** dst[5] = {&m, &ls, &q, &op, &sh};
        for (int k = 0; k < 5; ++k) {
            e = cudaMemcpy(p, src[k], len[k] * 4, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return finish({TIGAS_ERR_CUDA, cudaGetErrorString(e)});
            *dst[k] = p;
            p += len[k];
        }
    }
    Scene* s = nullptr;
    Status st = scene_create(m, ls, q, op, sh, n, d->sh_degree, d->storage, d->background, 0, &s);
    if (st.ok()) *out = reinterpret_cast<tigas_scene*>(s);
    return finish(st);
}

TIGAS_API tigas_status tigas_scene_free(tigas_scene* scene) {
    if (!scene) return fail(TIGAS_ERR_INVALID, "null scene");
    scene_release(reinterpret_cast<Scene*>(scene));
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_scene_bytes(const tigas_scene* scene, uint64_t* out) {
    if (!scene || !out) return fail(TIGAS_ERR_INVALID, "null argument");
    *out = reinterpret_cast<const Scene*>(scene)->bytes;
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_render_ex(tigas_scene* scene, const tigas_pose* pose, const tigas_intrinsics* intr,
                                       int width, int height, uint8_t* out_rgba8, float* out_rgba_f32,
                                       void* cuda_stream, int sort_mode, tigas_frame_stats* stats) {
    set_error("");
    if (!out_rgba8 && !out_rgba_f32) return fail(TIGAS_ERR_INVALID, "no output buffer");
    SceneGuard sg(reinterpret_cast<Scene*>(scene));
    Status st = do_render(sg.s, 1, pose, intr, &width, &height, &out_rgba8, &out_rgba_f32, (cudaStream_t)cuda_stream,
                          sort_mode, stats, nullptr, nullptr);
    return st.ok() ? TIGAS_OK : fail(st);
}

TIGAS_API tigas_status tigas_render(tigas_scene* scene, const tigas_pose* pose, const tigas_intrinsics* intr,
                                    int width, int height, uint8_t* out_rgba8) {
    if (!out_rgba8) return fail(TIGAS_ERR_INVALID, "null output");
    return tigas_render_ex(scene, pose, intr, width, height, out_rgba8, nullptr, nullptr, TIGAS_SORT_SLICED, nullptr);
}

TIGAS_API tigas_status tigas_render_batch(tigas_scene* scene, int n_views, const tigas_pose* poses,
                                          const tigas_intrinsics* intrs, const int* widths, const int* heights,
                                          uint8_t* const* outs, void* cuda_stream) {
    set_error("");
    if (!poses || !intrs || !widths || !heights || !outs) return fail(TIGAS_ERR_INVALID, "null argument");
    if (n_views < 1 || n_views > kMaxViews) return fail(TIGAS_ERR_INVALID, "n_views out of 1..64");
    for (int v = 0; v < n_views; ++v)
        if (!outs[v]) return fail(TIGAS_ERR_INVALID, "null output buffer");
    SceneGuard sg(reinterpret_cast<Scene*>(scene));
    Status st = do_render(sg.s, n_views, poses, intrs, widths, heights, outs, nullptr, (cudaStream_t)cuda_stream,
                          TIGAS_SORT_SLICED, nullptr, nullptr, nullptr);
    return st.ok() ? TIGAS_OK : fail(st);
}

TIGAS_API tigas_status tigas_render_batch_ex(tigas_scene* scene, int n_views, const tigas_pose* poses,
                                             const tigas_intrinsics* intrs, const int* widths, const int* heights,
                                             uint8_t* const* outs, void* cuda_stream, int sort_mode,
                                             tigas_frame_stats* stats) {
    set_error("");
    if (!poses || !intrs || !widths || !heights || !outs) return fail(TIGAS_ERR_INVALID, "null argument");
    if (n_views < 1 || n_views > kMaxViews) return fail(TIGAS_ERR_INVALID, "n_views out of 1..64");
    for (int v = 0; v < n_views; ++v)
        if (!outs[v]) return fail(TIGAS_ERR_INVALID, "null output buffer");
    SceneGuard sg(reinterpret_cast<Scene*>(scene));
    Status st = do_render(sg.s, n_views, poses, intrs, widths, heights, outs, nullptr, (cudaStream_t)cuda_stream,
                          sort_mode, stats, nullptr, nullptr);
    return st.ok() ? TIGAS_OK : fail(st);
}

struct tigas_ticket {
    RenderContext* ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t submitted = nullptr;
    PendingRender p;
};

TIGAS_API tigas_status tigas_render_batch_async(tigas_scene* scene, int n_views, const tigas_pose* poses,
                                                const tigas_intrinsics* intrs, const int* widths, const int* heights,
                                                uint8_t* const* outs, void* cuda_stream, tigas_ticket** out_ticket) {
    set_error("");
    if (!out_ticket) return fail(TIGAS_ERR_INVALID, "null ticket output");
    *out_ticket = nullptr;
    if (!scene || !poses || !intrs || !widths || !heights || !outs) return fail(TIGAS_ERR_INVALID, "null argument");
    if (n_views < 1 || n_views > kMaxViews) return fail(TIGAS_ERR_INVALID, "n_views out of 1..64");
    for (int v = 0; v < n_views; ++v)
        if (!outs[v]) return fail(TIGAS_ERR_INVALID, "null output buffer");
    Status err;
    RenderContext* ctx = acquire_context(&err);
    if (!ctx) return fail(err);
    auto* t = new tigas_ticket();
    t->ctx = ctx;
    t->st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    Scene* sc = reinterpret_cast<Scene*>(scene);
    scene_acquire(sc);
    t->p.scene = sc;
    // host outputs are copied back on the context's copy stream, so the copies
    // of this launch set overlap the next one's device work
    Status s = submit_render(*ctx, sc, n_views, poses, intrs, widths, heights, outs, nullptr, t->st,
                             TIGAS_SORT_SLICED, false, false, t->p, ctx->copy_stream);
    if (s.ok()) {
        cudaError_t e = cudaEventCreateWithFlags(&t->submitted, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(t->submitted, ctx->copy_stream);
        if (e != cudaSuccess) s = {TIGAS_ERR_CUDA, cudaGetErrorString(e)};
    }
    if (!s.ok()) {
        cudaStreamSynchronize(t->st);   // nothing of this launch set may still use the context
        cudaStreamSynchronize(ctx->copy_stream);
        if (t->submitted) cudaEventDestroy(t->submitted);
        scene_release(sc);
        release_context(ctx);
        delete t;
        return fail(s);
    }
    *out_ticket = t;
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_render_wait(tigas_ticket* t) {
    set_error("");
    if (!t) return fail(TIGAS_ERR_INVALID, "null ticket");
    Status s;
    cudaError_t e = cudaEventSynchronize(t->submitted);
    if (e != cudaSuccess) s = {TIGAS_ERR_CUDA, cudaGetErrorString(e)};
    if (s.ok()) s = finish_render(*t->ctx, t->st, t->p);
    if (!s.ok()) {
        cudaStreamSynchronize(t->st);
        cudaStreamSynchronize(t->ctx->copy_stream);
    }
    cudaEventDestroy(t->submitted);
    scene_release(t->p.scene);
    release_context(t->ctx);
    delete t;
    return s.ok() ? TIGAS_OK : fail(s);
}

TIGAS_API tigas_status tigas_debug_render(tigas_scene* scene, const tigas_pose* pose, const tigas_intrinsics* intr,
                                          int width, int height, int sort_mode, tigas_debug_frame* out,
                                          uint64_t* out_pairs) {
    set_error("");
    if (!out) return fail(TIGAS_ERR_INVALID, "null debug output");
    SceneGuard sg(reinterpret_cast<Scene*>(scene));
    float* f32 = out->rgba_f32;
    uint8_t* none = nullptr;
    Status st = do_render(sg.s, 1, pose, intr, &width, &height, &none, f32 ? &f32 : nullptr, nullptr, sort_mode,
                          nullptr, out, out_pairs);
    return st.ok() ? TIGAS_OK : fail(st);
}

TIGAS_API tigas_status tigas_sort_pairs_u64(const uint64_t* keys_in, const uint32_t* values_in, uint64_t* keys_out,
                                            uint32_t* values_out, uint64_t n, int begin_bit, int end_bit,
                                            void* cuda_stream) {
    set_error("");
    if (n > 0 && (!keys_in || !values_in || !keys_out || !values_out)) return fail(TIGAS_ERR_INVALID, "null buffer");
    if (begin_bit < 0 || end_bit > 64 || begin_bit >= end_bit) return fail(TIGAS_ERR_INVALID, "bad bit range");
    if (n >= 0xFFFFFFFFull) return fail(TIGAS_ERR_INVALID, "n too large");
    if (n == 0) return TIGAS_OK;
    if (keys_in == keys_out || values_in == values_out) return fail(TIGAS_ERR_INVALID, "in and out must differ");
    Status err;
    ContextGuard g;
    g.ctx = acquire_context(&err);
    if (!g.ctx) return fail(err);
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : g.ctx->stream;
    const size_t words = radix_tmp_words(n);
    Status s = g.ctx->pairs.reserve(n * 12 + words * 4 + 8192);
    if (!s.ok()) return fail(s);
    g.ctx->pairs.reset();
    uint64_t* ka = g.ctx->pairs.take<uint64_t>(n);
    uint32_t* va = g.ctx->pairs.take<uint32_t>(n);
    uint32_t* tmp = g.ctx->pairs.take<uint32_t>(words);
    uint32_t* d_flags = g.ctx->pairs.take<uint32_t>(1);
    cudaError_t e = cudaMemsetAsync(d_flags, 0, 4, st);
    if (e != cudaSuccess) return fail(TIGAS_ERR_CUDA, cudaGetErrorString(e));
    s = radix_sort<uint64_t>(keys_in, values_in, ka, va, keys_out, values_out, n, nullptr, begin_bit, end_bit, tmp, st,
                             nullptr, d_flags);
    if (!s.ok()) return fail(s);
    e = cudaMemcpyAsync(g.ctx->h_flags, d_flags, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(TIGAS_ERR_CUDA, cudaGetErrorString(e));
    if (g.ctx->h_flags[0] & kSortTimeoutFlag) return fail(TIGAS_ERR_TIMEOUT, "radix sort look-back wait ran out");
    return TIGAS_OK;
}
