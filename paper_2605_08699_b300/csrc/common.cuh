// Shared definitions of the CUDA path: status plumbing, view parameters, the
// resident scene layout, and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/tigas.h"

namespace tigas {

constexpr int kTile = 16;              // 16x16 pixel tiles
// SMs of a B300 (two dies of 74).  Grid-size heuristics only: every kernel is
// correct for any grid it sizes from this.
constexpr int kSmCount = 148;
constexpr int kMaxViews = 64;          // views per fused launch set
constexpr int kMaxDim = 8192;          // largest width / height accepted
constexpr int kMaxDevices = 64;        // device ordinals with their own one-time set-up

// ---------------------------------------------------------------- errors

void set_error(const std::string& msg);
const char* last_error();
extern std::atomic<uint64_t> g_launches;

struct Status {
    tigas_status code = TIGAS_OK;
    std::string msg;
    bool ok() const { return code == TIGAS_OK; }
};

#define TIGAS_CUDA_TRY(expr)                                                            \
    do {                                                                                \
        cudaError_t e__ = (expr);                                                       \
        if (e__ != cudaSuccess) {                                                       \
            return ::tigas::Status{e__ == cudaErrorMemoryAllocation ? TIGAS_ERR_OOM     \
                                                                    : TIGAS_ERR_CUDA,   \
                                   std::string(#expr) + ": " + cudaGetErrorString(e__)}; \
        }                                                                               \
    } while (0)

#define TIGAS_TRY(expr)                     \
    do {                                    \
        ::tigas::Status s__ = (expr);       \
        if (!s__.ok()) return s__;          \
    } while (0)

// Every device and pinned-host allocation of the library goes through these,
// so that tests can make the nth one fail (tigas_debug_fail_alloc): the failure
// is injected on the host, as cudaErrorMemoryAllocation, and nothing is asked of
// the GPU.  kind 0: device memory, kind 1: pinned host memory.
cudaError_t device_alloc(void** p, size_t bytes);
cudaError_t pinned_alloc(void** p, size_t bytes);
template <typename T>
inline cudaError_t device_alloc(T** p, size_t bytes) {
    return device_alloc(reinterpret_cast<void**>(p), bytes);
}
template <typename T>
inline cudaError_t pinned_alloc(T** p, size_t bytes) {
    return pinned_alloc(reinterpret_cast<void**>(p), bytes);
}
// Arm (nth >= 1) or clear (nth = 0) the injection for one kind: allocations
// nth .. nth + count - 1 from now fail.
void inject_alloc_failures(int kind, int64_t nth, int64_t count);

// Check a launch and count it.
#define TIGAS_LAUNCHED()                                                        \
    do {                                                                        \
        ::tigas::g_launches.fetch_add(1, std::memory_order_relaxed);            \
        cudaError_t e__ = cudaGetLastError();                                   \
        if (e__ != cudaSuccess)                                                 \
            return ::tigas::Status{TIGAS_ERR_CUDA,                              \
                                   std::string("kernel launch: ") + cudaGetErrorString(e__)}; \
    } while (0)

// ------------------------------------------------------------- scene layout
//
// Resident scene: an array-of-structures-of-arrays with 32 Gaussians per
// block.  Each Gaussian is a fixed number of 16-byte chunks; chunk c of
// Gaussian i lives at chunk index ((i / 32) * C + c) * 32 + (i % 32), so a
// warp reading chunk c of 32 consecutive Gaussians touches 512 contiguous
// bytes.
//
//  FP32 storage, C = 15:
//    chunk 0: (x, y, z, opacity)            f32 x4
//    chunk 1: (qw, qx, qy, qz)  unit        f32 x4
//    chunk 2: (sx, sy, sz, 0)   exp(log s)  f32 x4
//    chunk 3..14: SH [16][3]                f32 x48
//  FP16 storage, C = 8:
//    chunk 0: (x, y, z) f32, (opacity, sx) f16x2
//    chunk 1: (sy, sz) f16x2, (qw, qx) f16x2, (qy, qz) f16x2, pad
//    chunk 2..7: SH [16][3]                 f16 x48
constexpr int kChunksF32 = 15;
constexpr int kChunksF16 = 8;

struct SceneView {
    const uint4* chunks = nullptr;   // AoSoA32 storage
    uint32_t n = 0;
    int sh_degree = 3;
    int storage = TIGAS_STORAGE_FP32;
    float bg[3] = {0.f, 0.f, 0.f};
};

__host__ __device__ inline size_t chunk_index(uint32_t i, int c, int C) {
    return ((size_t)(i >> 5) * C + c) * 32 + (i & 31);
}

// ----------------------------------------------------------------- views

// One view of a fused launch set.  Everything the kernels need per view.
struct ViewParams {
    float Rt[9];          // world->camera rotation R^T, row-major
    float campos[3];      // camera centre t
    float fx, fy, cx, cy;
    float limx, limy;     // 1.3 * W / (2 fx), 1.3 * H / (2 fy)
    int W, H, TX, TY;
    uint32_t tile_base;   // first global tile id of this view
    uint32_t sat_base;    // sliced schedule: offset of this view's running-tile table ((TY+1) x (TX+1))
    uint8_t* out_rgba8;   // device pointer or null
    float* out_rgba_f32;  // device pointer or null
};

// Per-view preprocess output, indexed by entry e = view * n + gaussian.
// The blend evaluates alpha = min(0.99, 2^(a' dx^2 + b' dx dy + c' dy^2 + log2 o))
// = min(0.99, o exp(power)).
struct SplatArrays {
    float4* geom;         // (u, v, a', b')   a' = -A/2 log2e, b' = -B log2e
    float4* appear;       // (c', log2(opacity), r, g)  c' = -C/2 log2e
    float* blue;          // b
    uint32_t* depth_key;  // float bits of view z, 0xFFFFFFFF when culled
    uint32_t* tiles;      // tiles touched (0 when culled)
    uint2* rect;          // wide: (x_lo | x_hi << 10 | view << 20, y_lo | y_hi << 10); (0, 0) when culled
                          // compact: (x_lo | x_hi << 7 | y_lo << 14 | y_hi << 21 | view << 28, entry)
    float* q_dbg;         // optional: 3 sqrt(lambda) per entry (parity diagnostics)
    uint32_t* key_range;  // optional: [min, max] of the kept depth keys of the launch set
    int tight_rect;       // 1: rect = the 3-sigma rectangle cut to the tiles the alpha >= 1/255 region
                          // can reach (result-invariant; the sliced schedule), 0: the 3-sigma rectangle
    int compact_rect;     // 1: compact rect carrying its entry id (every view has TX, TY <= kCompactTiles
                          // and there are at most 16 views), so that a depth sort moves no separate values
};

// Compact rectangle: 7 bits per tile bound, 4 bits of view.
constexpr int kCompactTiles = 127;
constexpr int kCompactViews = 16;
struct TileRect {
    uint32_t xlo, xhi, ylo, yhi, v;
};
__host__ __device__ inline uint32_t pack_rect_compact(uint32_t xlo, uint32_t xhi, uint32_t ylo, uint32_t yhi,
                                                      uint32_t v) {
    return xlo | (xhi << 7) | (ylo << 14) | (yhi << 21) | (v << 28);
}
template <bool COMPACT>
__host__ __device__ inline TileRect unpack_rect(uint2 r) {
    if (COMPACT)
        return {r.x & 0x7Fu, (r.x >> 7) & 0x7Fu, (r.x >> 14) & 0x7Fu, (r.x >> 21) & 0x7Fu, r.x >> 28};
    return {r.x & 0x3FFu, (r.x >> 10) & 0x3FFu, r.y & 0x3FFu, (r.y >> 10) & 0x3FFu, r.x >> 20};
}

__host__ __device__ inline uint32_t ceil_div_u32(uint32_t a, uint32_t b) { return (a + b - 1) / b; }

}  // namespace tigas
