// Model registry (Sec. 4.1 "PLY Model and Primitives", Sec. 5.1 "Dynamic
// Multi-Model Runtime"): a directory of 3DGS models is scanned once for
// metadata (identifier, name, preview image, PLY header); a model's tensors are
// loaded into HBM on its first acquisition, shared by every client that
// acquires it, reference-counted while in use, and unloaded by an eviction pass
// once it has been idle for the inactivity timeout.  An optional resident-byte
// budget evicts idle models, least recently used first, before a load that
// would exceed it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <filesystem>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pipeline.cuh"

#define TIGAS_API extern "C" __attribute__((visibility("default")))

namespace fs = std::filesystem;

namespace tigas {

tigas_status fail(const Status& s);
tigas_status fail(tigas_status code, const std::string& msg);

struct ModelEntry {
    std::string id, name, ply, preview;
    uint64_t n = 0, file_bytes = 0;
    int sh_degree = 0;
    Scene* scene = nullptr;   // the registry's own reference while loaded
    bool loading = false;
    int users = 0;            // acquisitions not yet released
    uint64_t loads = 0;
    double last_use = 0.0;
};

struct Registry {
    std::string root;
    int storage = TIGAS_STORAGE_FP16;
    float bg[3] = {0, 0, 0};
    double idle_timeout = 60.0;
    uint64_t budget = 0;       // 0: unbounded
    std::mutex mu;
    std::condition_variable cv;            // load finished / evictor stop
    std::vector<std::unique_ptr<ModelEntry>> models;   // sorted by id
    std::unordered_map<Scene*, ModelEntry*> by_scene;
    double fake_now = -1.0;                // >= 0: test clock
    std::thread evictor;
    bool stop = false;
    uint64_t evictions = 0;

    double now() const {
        if (fake_now >= 0) return fake_now;
        using namespace std::chrono;
        return duration<double>(steady_clock::now().time_since_epoch()).count();
    }
    ModelEntry* find(const std::string& id) {
        for (auto& m : models)
            if (m->id == id) return m.get();
        return nullptr;
    }
    uint64_t resident() const {
        uint64_t b = 0;
        for (auto& m : models) {
            if (m->scene) b += m->scene->bytes;
            else if (m->loading) b += scene_bytes_for(m->n, storage);
        }
        return b;
    }
    void unload(ModelEntry* m) {   // caller holds mu; m->users == 0
        by_scene.erase(m->scene);
        scene_release(m->scene);
        m->scene = nullptr;
        ++evictions;
    }
    int evict_idle(double t) {
        int k = 0;
        for (auto& m : models)
            if (m->scene && m->users == 0 && t - m->last_use >= idle_timeout) {
                unload(m.get());
                ++k;
            }
        return k;
    }
    // Evict idle models, least recently used first, until need more bytes fit.
    bool make_room(uint64_t need) {
        if (budget == 0) return true;
        while (resident() + need > budget) {
            ModelEntry* lru = nullptr;
            for (auto& m : models)
                if (m->scene && m->users == 0 && (!lru || m->last_use < lru->last_use)) lru = m.get();
            if (!lru) return false;
            unload(lru);
        }
        return true;
    }
};

namespace {

const char* kPreviewNames[] = {"preview.png", "preview.jpg", "preview.jpeg"};

// The PLY of a model folder: the highest point_cloud/iteration_<k>/point_cloud.ply
// (the layout 3DGS training writes), else the first *.ply in the folder.
std::string model_ply(const fs::path& dir) {
    std::error_code ec;
    long best = -1;
    std::string best_path;
    fs::path pc = dir / "point_cloud";
    if (fs::is_directory(pc, ec)) {
        for (auto& it : fs::directory_iterator(pc, ec)) {
            std::string name = it.path().filename().string();
            if (name.compare(0, 10, "iteration_") != 0) continue;
            char* end = nullptr;
            long k = strtol(name.c_str() + 10, &end, 10);
            if (!end || *end || k < 0) continue;
            fs::path f = it.path() / "point_cloud.ply";
            if (k > best && fs::is_regular_file(f, ec)) {
                best = k;
                best_path = f.string();
            }
        }
    }
    if (!best_path.empty()) return best_path;
    std::vector<std::string> plys;
    for (auto& it : fs::directory_iterator(dir, ec))
        if (it.is_regular_file(ec) && it.path().extension() == ".ply") plys.push_back(it.path().string());
    std::sort(plys.begin(), plys.end());
    return plys.empty() ? std::string() : plys[0];
}

std::string find_preview(const fs::path& dir, const std::string& stem) {
    std::error_code ec;
    if (stem.empty()) {
        for (const char* p : kPreviewNames)
            if (fs::is_regular_file(dir / p, ec)) return (dir / p).string();
    } else {
        for (const char* ext : {".png", ".jpg", ".jpeg"})
            if (fs::is_regular_file(dir / (stem + ext), ec)) return (dir / (stem + ext)).string();
    }
    return {};
}

}  // namespace

// Rescan the root folder.  Models already known keep their state; models
// whose files disappeared are dropped unless loaded.
Status registry_scan(Registry* r, int* n_models, int* n_skipped) {
    std::error_code ec;
    fs::path root(r->root);
    if (!fs::is_directory(root, ec)) return {TIGAS_ERR_IO, "not a directory: " + r->root};
    struct Found { std::string id, ply, preview; };
    std::map<std::string, Found> found;
    std::vector<fs::directory_entry> entries;
    for (auto& it : fs::directory_iterator(root, ec)) entries.push_back(it);
    if (ec) return {TIGAS_ERR_IO, "cannot list " + r->root + ": " + ec.message()};
    std::sort(entries.begin(), entries.end(),
              [](const fs::directory_entry& a, const fs::directory_entry& b) { return a.path() < b.path(); });
    for (auto& it : entries) {   // folders first: a folder wins over a same-named top-level file
        if (!it.is_directory(ec)) continue;
        std::string ply = model_ply(it.path());
        if (ply.empty()) continue;
        std::string id = it.path().filename().string();
        found[id] = {id, ply, find_preview(it.path(), "")};
    }
    for (auto& it : entries) {
        if (!it.is_regular_file(ec) || it.path().extension() != ".ply") continue;
        std::string id = it.path().stem().string();
        if (found.count(id)) continue;
        found[id] = {id, it.path().string(), find_preview(root, id)};
    }
    int skipped = 0;
    std::vector<std::unique_ptr<ModelEntry>> next;
    std::lock_guard<std::mutex> lk(r->mu);
    for (auto& kv : found) {
        PlyLayout lay;
        if (!ply_probe(kv.second.ply.c_str(), &lay).ok()) {
            ++skipped;
            continue;
        }
        std::unique_ptr<ModelEntry> m;
        for (auto& old : r->models)
            if (old && old->id == kv.first) m = std::move(old);
        if (!m) {
            m.reset(new ModelEntry());
            m->id = kv.first;
            m->name = kv.first;
        }
        m->ply = kv.second.ply;   // a load in progress already holds its own copy
        m->preview = kv.second.preview;
        if (!m->scene && !m->loading) {
            m->n = lay.n;
            m->sh_degree = lay.sh_degree;
            m->file_bytes = lay.file_bytes;
        }
        next.push_back(std::move(m));
    }
    for (auto& old : r->models)   // vanished but still resident: keep until unloaded
        if (old && (old->scene || old->loading)) next.push_back(std::move(old));
    std::sort(next.begin(), next.end(), [](const std::unique_ptr<ModelEntry>& a, const std::unique_ptr<ModelEntry>& b) {
        return a->id < b->id;
    });
    r->models = std::move(next);
    if (n_models) *n_models = (int)r->models.size();
    if (n_skipped) *n_skipped = skipped;
    return {};
}

Status registry_acquire(Registry* r, const char* id, Scene** out) {
    *out = nullptr;
    std::unique_lock<std::mutex> lk(r->mu);
    ModelEntry* m = r->find(id);
    if (!m) return {TIGAS_ERR_NOT_FOUND, std::string("unknown model '") + id + "'"};
    r->cv.wait(lk, [&] { return !m->loading; });
    if (!m->scene) {
        if (!r->make_room(scene_bytes_for(m->n, r->storage)))
            return {TIGAS_ERR_OOM, std::string("registry budget cannot hold model '") + id + "'"};
        m->loading = true;
        const std::string ply = m->ply;
        lk.unlock();
        Scene* s = nullptr;
        Status st = scene_load_ply(ply.c_str(), r->storage, r->bg, &s);
        lk.lock();
        m->loading = false;
        r->cv.notify_all();
        if (!st.ok()) return st;
        m->scene = s;
        m->n = s->view.n;
        m->sh_degree = s->view.sh_degree;
        ++m->loads;
        r->by_scene[s] = m;
    }
    ++m->users;
    m->last_use = r->now();
    scene_acquire(m->scene);
    *out = m->scene;
    return {};
}

Status registry_release(Registry* r, Scene* s) {
    std::lock_guard<std::mutex> lk(r->mu);
    auto it = r->by_scene.find(s);
    if (it == r->by_scene.end() || it->second->users <= 0)
        return {TIGAS_ERR_INVALID, "scene was not acquired from this registry"};
    ModelEntry* m = it->second;
    --m->users;
    m->last_use = r->now();
    scene_release(s);   // the registry's own reference keeps the scene resident
    return {};
}

int registry_evict_idle(Registry* r) {
    std::lock_guard<std::mutex> lk(r->mu);
    return r->evict_idle(r->now());
}

void registry_start_evictor(Registry* r, double period_s) {
    std::lock_guard<std::mutex> lk(r->mu);
    if (r->evictor.joinable()) return;
    r->stop = false;
    r->evictor = std::thread([r, period_s] {
        std::unique_lock<std::mutex> lk(r->mu);
        while (!r->stop) {
            r->cv.wait_for(lk, std::chrono::duration<double>(period_s), [&] { return r->stop; });
            if (!r->stop) r->evict_idle(r->now());
        }
    });
}

void registry_close(Registry* r) {
    {
        std::lock_guard<std::mutex> lk(r->mu);
        r->stop = true;
    }
    r->cv.notify_all();
    if (r->evictor.joinable()) r->evictor.join();
    std::unique_lock<std::mutex> lk(r->mu);
    r->cv.wait(lk, [&] {
        for (auto& m : r->models)
            if (m->loading) return false;
        return true;
    });
    for (auto& m : r->models)
        if (m->scene) {
            r->by_scene.erase(m->scene);
            scene_release(m->scene);   // acquisitions still held keep their scene alive
            m->scene = nullptr;
        }
}

void registry_info(Registry* r, int index, tigas_model_info* out, Status* st) {
    std::lock_guard<std::mutex> lk(r->mu);
    if (index < 0 || index >= (int)r->models.size()) {
        *st = {TIGAS_ERR_INVALID, "model index out of range"};
        return;
    }
    const ModelEntry& m = *r->models[index];
    memset(out, 0, sizeof(*out));
    auto put = [](char* dst, size_t cap, const std::string& s) {
        size_t k = std::min(cap - 1, s.size());
        memcpy(dst, s.data(), k);
        dst[k] = 0;
    };
    put(out->id, sizeof(out->id), m.id);
    put(out->name, sizeof(out->name), m.name);
    put(out->ply_path, sizeof(out->ply_path), m.ply);
    put(out->preview_path, sizeof(out->preview_path), m.preview);
    out->n = m.n;
    out->sh_degree = m.sh_degree;
    out->loaded = m.scene != nullptr;
    out->users = m.users;
    out->file_bytes = m.file_bytes;
    out->resident_bytes = m.scene ? m.scene->bytes : 0;
    out->loads = m.loads;
    out->idle_seconds = m.scene && m.users == 0 ? r->now() - m.last_use : 0.0;
    *st = {};
}

}  // namespace tigas

// ------------------------------------------------------------------ C ABI

using namespace tigas;

TIGAS_API tigas_status tigas_ply_probe(const char* path, tigas_ply_info* out) {
    set_error("");
    if (!path || !out) return fail(TIGAS_ERR_INVALID, "null argument");
    PlyLayout lay;
    Status st = ply_probe(path, &lay);
    if (!st.ok()) return fail(st);
    out->n = lay.n;
    out->file_bytes = lay.file_bytes;
    out->body_offset = lay.body_offset;
    out->sh_degree = lay.sh_degree;
    out->format = lay.format;
    out->row_bytes = lay.row_bytes;
    out->n_properties = (uint32_t)lay.prop_type.size();
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_ply_decode(const char* path, float* means, float* log_scales, float* quats,
                                        float* opacity_logits, float* sh, int outputs_on_device) {
    set_error("");
    if (!path || !means || !log_scales || !quats || !opacity_logits || !sh)
        return fail(TIGAS_ERR_INVALID, "null argument");
    PlyLayout lay;
    Status st = ply_probe(path, &lay);
    if (!st.ok()) return fail(st);
    const uint64_t n = lay.n;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(TIGAS_ERR_CUDA, "stream creation failed");
    }
    if (outputs_on_device) {
        st = ply_decode(path, lay, means, log_scales, quats, opacity_logits, sh, s);
    } else {
        float* d = nullptr;
        if (device_alloc(&d, n * kPlyFields * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamDestroy(s);
            return fail(TIGAS_ERR_OOM, "decode staging allocation failed");
        }
        float* dst[5] = {d, d + 3 * n, d + 6 * n, d + 10 * n, d + 11 * n};
        float* host[5] = {means, log_scales, quats, opacity_logits, sh};
        const uint64_t len[5] = {3 * n, 3 * n, 4 * n, n, 48 * n};
        st = ply_decode(path, lay, dst[0], dst[1], dst[2], dst[3], dst[4], s);
        for (int k = 0; k < 5 && st.ok(); ++k) {
            cudaError_t e = cudaMemcpy(host[k], dst[k], len[k] * sizeof(float), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = {TIGAS_ERR_CUDA, cudaGetErrorString(e)};
        }
        cudaFree(d);
    }
    cudaStreamDestroy(s);
    return st.ok() ? TIGAS_OK : fail(st);
}

TIGAS_API tigas_status tigas_scene_load_ply(const char* path, int storage, const float background[3],
                                            tigas_scene** out) {
    set_error("");
    if (!path || !out) return fail(TIGAS_ERR_INVALID, "null argument");
    *out = nullptr;
    if (storage != TIGAS_STORAGE_FP32 && storage != TIGAS_STORAGE_FP16) return fail(TIGAS_ERR_INVALID, "unknown storage");
    float bg[3] = {0, 0, 0};
    if (background)
        for (int c = 0; c < 3; ++c) {
            if (!std::isfinite(background[c])) return fail(TIGAS_ERR_INVALID, "non-finite background");
            bg[c] = background[c];
        }
    Scene* s = nullptr;
    Status st = scene_load_ply(path, storage, bg, &s);
    if (!st.ok()) return fail(st);
    *out = reinterpret_cast<tigas_scene*>(s);
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_registry_open(const char* root_dir, int storage, double idle_timeout_s,
                                           uint64_t budget, const float background[3], tigas_registry** out) {
    set_error("");
    if (!root_dir || !out) return fail(TIGAS_ERR_INVALID, "null argument");
    *out = nullptr;
    if (storage != TIGAS_STORAGE_FP32 && storage != TIGAS_STORAGE_FP16) return fail(TIGAS_ERR_INVALID, "unknown storage");
    if (!(idle_timeout_s >= 0) || !std::isfinite(idle_timeout_s))
        return fail(TIGAS_ERR_INVALID, "idle_timeout_s must be finite and >= 0");
    auto* r = new Registry();
    r->root = root_dir;
    r->storage = storage;
    r->idle_timeout = idle_timeout_s;
    r->budget = budget;
    if (background)
        for (int c = 0; c < 3; ++c) {
            if (!std::isfinite(background[c])) {
                delete r;
                return fail(TIGAS_ERR_INVALID, "non-finite background");
            }
            r->bg[c] = background[c];
        }
    Status st = registry_scan(r, nullptr, nullptr);
    if (!st.ok()) {
        delete r;
        return fail(st);
    }
    *out = reinterpret_cast<tigas_registry*>(r);
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_registry_scan(tigas_registry* reg, int* n_models, int* n_skipped) {
    set_error("");
    if (!reg) return fail(TIGAS_ERR_INVALID, "null registry");
    Status st = registry_scan(reinterpret_cast<Registry*>(reg), n_models, n_skipped);
    return st.ok() ? TIGAS_OK : fail(st);
}

TIGAS_API tigas_status tigas_registry_count(tigas_registry* reg, int* n_models) {
    if (!reg || !n_models) return fail(TIGAS_ERR_INVALID, "null argument");
    auto* r = reinterpret_cast<Registry*>(reg);
    std::lock_guard<std::mutex> lk(r->mu);
    *n_models = (int)r->models.size();
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_registry_info(tigas_registry* reg, int index, tigas_model_info* out) {
    if (!reg || !out) return fail(TIGAS_ERR_INVALID, "null argument");
    Status st;
    registry_info(reinterpret_cast<Registry*>(reg), index, out, &st);
    return st.ok() ? TIGAS_OK : fail(st);
}

TIGAS_API tigas_status tigas_registry_acquire(tigas_registry* reg, const char* model_id, tigas_scene** out) {
    set_error("");
    if (!reg || !model_id || !out) return fail(TIGAS_ERR_INVALID, "null argument");
    Scene* s = nullptr;
    Status st = registry_acquire(reinterpret_cast<Registry*>(reg), model_id, &s);
    *out = reinterpret_cast<tigas_scene*>(s);
    return st.ok() ? TIGAS_OK : fail(st);
}

TIGAS_API tigas_status tigas_registry_release(tigas_registry* reg, tigas_scene* scene) {
    if (!reg || !scene) return fail(TIGAS_ERR_INVALID, "null argument");
    Status st = registry_release(reinterpret_cast<Registry*>(reg), reinterpret_cast<Scene*>(scene));
    return st.ok() ? TIGAS_OK : fail(st);
}

TIGAS_API tigas_status tigas_registry_evict_idle(tigas_registry* reg, int* n_evicted) {
    if (!reg) return fail(TIGAS_ERR_INVALID, "null registry");
    int k = registry_evict_idle(reinterpret_cast<Registry*>(reg));
    if (n_evicted) *n_evicted = k;
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_registry_start_eviction(tigas_registry* reg, double period_s) {
    if (!reg) return fail(TIGAS_ERR_INVALID, "null registry");
    if (!(period_s > 0) || !std::isfinite(period_s)) return fail(TIGAS_ERR_INVALID, "period_s must be finite and > 0");
    registry_start_evictor(reinterpret_cast<Registry*>(reg), period_s);
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_registry_set_clock(tigas_registry* reg, double now_s) {
    if (!reg) return fail(TIGAS_ERR_INVALID, "null registry");
    if (std::isnan(now_s) || std::isinf(now_s)) return fail(TIGAS_ERR_INVALID, "now_s must be finite");
    auto* r = reinterpret_cast<Registry*>(reg);
    std::lock_guard<std::mutex> lk(r->mu);
    r->fake_now = now_s >= 0 ? now_s : -1.0;
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_registry_close(tigas_registry* reg) {
    if (!reg) return fail(TIGAS_ERR_INVALID, "null registry");
    auto* r = reinterpret_cast<Registry*>(reg);
    registry_close(r);
    delete r;
    return TIGAS_OK;
}
