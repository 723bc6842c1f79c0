// Serving loop: continuous batching of per-client render requests.
//
// The paper's backend serves every pose request as an isolated, stateless
// render task (Sec. 4.2) from scenes kept resident on the GPU and shared by
// all clients (Sec. 5.1 "Dynamic Multi-Model Runtime").  Here requests queue
// on the host; `max_inflight` worker slots, each with its own stream and
// persistent workspace, pull batches of up to `max_batch` queued requests of
// one scene (mixed resolutions) and render each batch as one fused launch set.
// A slot takes new work as soon as its previous batch is done and the
// admission budget (predicted workspace bytes of all batches in flight) has
// room, so requests that arrive while others are on the GPU join the next
// launch set and their work overlaps on the device with the other slots'.
// A queued request is superseded by a newer one of the same client.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "pipeline.cuh"

#define TIGAS_API extern "C" __attribute__((visibility("default")))

namespace tigas {

tigas_status fail(const Status& s);
tigas_status fail(tigas_status code, const std::string& msg);
Status validate_view(const tigas_pose* pose, const tigas_intrinsics* k, int w, int h);
Status do_render(Scene* scene, int V, const tigas_pose* poses, const tigas_intrinsics* intrs, const int* ws,
                 const int* hs, uint8_t* const* outs8, float* const* outs32, cudaStream_t user_st, int sort_mode,
                 tigas_frame_stats* stats, tigas_debug_frame* dbg, uint64_t* dbg_pairs);

namespace {

double now_us() {
    using namespace std::chrono;
    return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

struct Request {
    uint64_t ticket;
    uint64_t client;
    Scene* scene;
    tigas_pose pose;
    tigas_intrinsics intr;
    int w, h;
    uint8_t* out;
    double submit_us;
    bool superseded = false;
};

constexpr size_t kQueueCap = 1 << 16;

}  // namespace

struct Server {
    tigas_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work;   // queue changed / budget freed / stop
    std::condition_variable cv_done;   // completions available
    std::deque<Request> queue;
    std::unordered_map<uint64_t, uint64_t> queued_ticket_of_client;
    std::deque<tigas_completion> done;
    std::vector<std::thread> workers;
    uint64_t next_ticket = 1;
    uint64_t inflight_bytes = 0;
    int busy = 0;
    uint64_t batches_done = 0;
    bool stop = false;
    bool cancel = false;
    // pairs per Gaussian at 1920x1080, learned from finished frames
    double pairs_per_gaussian_1080 = 20.0;

    uint64_t predict_bytes(const Request& r) {
        const double f = std::sqrt((double)r.w * r.h / (1920.0 * 1080.0));
        // rectangle tiles scale roughly like (a f + 1)^2 with the radius in tiles
        const double a = std::max(0.0, std::sqrt(pairs_per_gaussian_1080) - 1.0);
        const double pairs = (double)r.scene->view.n * (a * f + 1.0) * (a * f + 1.0);
        return (uint64_t)(pairs * 24.0 + (double)r.scene->view.n * 96.0 + (double)r.w * r.h * 4.0);
    }

    void complete(const Request& r, int status, double admit, double t_done) {
        tigas_completion c{};
        c.ticket = r.ticket;
        c.client_id = r.client;
        c.status = status;
        c.width = r.w;
        c.height = r.h;
        c.submit_us = r.submit_us;
        c.admit_us = admit;
        c.done_us = t_done;
        done.push_back(c);
        scene_release(r.scene);
    }

    void worker() {
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            cv_work.wait(lk, [&] { return stop || !queue.empty(); });
            if (queue.empty()) {
                if (stop) return;
                continue;
            }
            // a launch set holds at most max_batch views, and no more than the tuned
            // views per launch set of the schedule of max_batch-view launch sets
            const int vps = current_schedule(cfg.max_batch).views_per_set;
            const int cap = vps > 0 && vps < cfg.max_batch ? vps : cfg.max_batch;
            if (cfg.batch_window_us > 0 && (int)queue.size() < cap && !stop) {
                // give a partial batch a short window to fill
                cv_work.wait_for(lk, std::chrono::microseconds(cfg.batch_window_us),
                                 [&] { return stop || (int)queue.size() >= cap; });
                if (queue.empty()) continue;
            }
            // form a batch: the oldest request's scene, oldest first, within budget
            Scene* scene = queue.front().scene;
            std::vector<Request> batch;
            uint64_t bytes = 0;
            for (auto it = queue.begin(); it != queue.end() && (int)batch.size() < cap;) {
                if (it->scene != scene) {
                    ++it;
                    continue;
                }
                uint64_t b = predict_bytes(*it);
                bool fits = inflight_bytes + bytes + b <= cfg.hbm_budget_bytes;
                if (!fits && !(batch.empty() && busy == 0)) break;   // alone on the GPU: always admitted
                bytes += b;
                auto q = queued_ticket_of_client.find(it->client);
                if (q != queued_ticket_of_client.end() && q->second == it->ticket) queued_ticket_of_client.erase(q);
                batch.push_back(*it);
                it = queue.erase(it);
            }
            if (batch.empty()) {
                // over budget: wait for a batch in flight to finish
                const uint64_t gen = batches_done;
                cv_work.wait(lk, [&] { return stop || batches_done != gen || busy == 0; });
                continue;
            }
            inflight_bytes += bytes;
            ++busy;
            const double admit = now_us();
            lk.unlock();

            const int V = (int)batch.size();
            std::vector<tigas_pose> poses(V);
            std::vector<tigas_intrinsics> intrs(V);
            std::vector<int> ws(V), hs(V);
            std::vector<uint8_t*> outs(V);
            for (int v = 0; v < V; ++v) {
                poses[v] = batch[v].pose;
                intrs[v] = batch[v].intr;
                ws[v] = batch[v].w;
                hs[v] = batch[v].h;
                outs[v] = batch[v].out;
            }
            // only the pair count is needed: no statistics, so the plain (uninstrumented) kernels run
            uint64_t n_pairs = 0;
            Status st = do_render(scene, V, poses.data(), intrs.data(), ws.data(), hs.data(), outs.data(), nullptr,
                                  nullptr, TIGAS_SORT_SLICED, nullptr, nullptr, &n_pairs);
            const double t_done = now_us();

            lk.lock();
            if (st.ok() && n_pairs > 0) {
                double px = 0;
                for (int v = 0; v < V; ++v) px += (double)ws[v] * hs[v] / (1920.0 * 1080.0);
                // P ~ n V (a f + 1)^2: update the 1080p estimate from this batch
                double per = (double)n_pairs / ((double)scene->view.n * V);
                double f = std::sqrt(px / V);
                double a = (std::sqrt(per) - 1.0) / std::max(f, 0.05);
                double est = (a + 1.0) * (a + 1.0);
                pairs_per_gaussian_1080 = 0.8 * pairs_per_gaussian_1080 + 0.2 * std::max(1.0, est);
            }
            for (auto& r : batch) complete(r, st.ok() ? TIGAS_OK : st.code, admit, t_done);
            inflight_bytes -= bytes;
            --busy;
            ++batches_done;
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }
};

}  // namespace tigas

using namespace tigas;

TIGAS_API tigas_status tigas_server_create(const tigas_server_config* cfg, tigas_server** out) {
    if (!out) return fail(TIGAS_ERR_INVALID, "null output");
    *out = nullptr;
    auto* s = new Server();
    if (cfg) s->cfg = *cfg;
    if (s->cfg.hbm_budget_bytes == 0) s->cfg.hbm_budget_bytes = 16ull << 30;
    if (s->cfg.max_batch == 0) s->cfg.max_batch = 16;
    if (s->cfg.max_inflight == 0) s->cfg.max_inflight = 2;
    if (s->cfg.max_batch < 1 || s->cfg.max_batch > kMaxViews || s->cfg.max_inflight < 1 || s->cfg.max_inflight > 8 ||
        s->cfg.batch_window_us < 0) {
        delete s;
        return fail(TIGAS_ERR_INVALID, "server config out of range");
    }
    for (int i = 0; i < s->cfg.max_inflight; ++i) s->workers.emplace_back([s] { s->worker(); });
    *out = reinterpret_cast<tigas_server*>(s);
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_server_destroy(tigas_server* server, int cancel) {
    if (!server) return fail(TIGAS_ERR_INVALID, "null server");
    auto* s = reinterpret_cast<Server*>(server);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        if (cancel) {
            const double t = now_us();
            for (auto& r : s->queue) s->complete(r, TIGAS_ERR_AGAIN, 0.0, t);
            s->queue.clear();
            s->queued_ticket_of_client.clear();
        }
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_server_submit(tigas_server* server, tigas_scene* scene, const tigas_pose* pose,
                                           const tigas_intrinsics* intr, int width, int height, uint8_t* out_rgba8,
                                           uint64_t client_id, uint64_t* out_ticket) {
    if (!server || !scene || !out_rgba8) return fail(TIGAS_ERR_INVALID, "null argument");
    Status v = validate_view(pose, intr, width, height);
    if (!v.ok()) return fail(v);
    auto* s = reinterpret_cast<Server*>(server);
    Request r{};
    r.client = client_id;
    r.scene = reinterpret_cast<Scene*>(scene);
    r.pose = *pose;
    r.intr = *intr;
    r.w = width;
    r.h = height;
    r.out = out_rgba8;
    r.submit_us = now_us();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return fail(TIGAS_ERR_INVALID, "server is stopping");
        if (s->queue.size() >= kQueueCap) return fail(TIGAS_ERR_AGAIN, "request queue full");
        r.ticket = s->next_ticket++;
        // latest pose wins: a queued request of this client is superseded
        auto it = s->queued_ticket_of_client.find(client_id);
        if (it != s->queued_ticket_of_client.end()) {
            for (auto q = s->queue.begin(); q != s->queue.end(); ++q) {
                if (q->ticket == it->second) {
                    s->complete(*q, TIGAS_ERR_AGAIN, 0.0, r.submit_us);
                    s->queue.erase(q);
                    break;
                }
            }
        }
        s->queued_ticket_of_client[client_id] = r.ticket;
        scene_acquire(r.scene);
        s->queue.push_back(r);
    }
    s->cv_work.notify_one();
    s->cv_done.notify_all();
    if (out_ticket) *out_ticket = r.ticket;
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_server_poll(tigas_server* server, tigas_completion* out, int max, int timeout_us,
                                         int* n_done) {
    if (!server || !n_done || (max > 0 && !out) || max < 0 || timeout_us < 0)
        return fail(TIGAS_ERR_INVALID, "bad poll arguments");
    auto* s = reinterpret_cast<Server*>(server);
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !s->done.empty(); });
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n_done = k;
    return TIGAS_OK;
}
