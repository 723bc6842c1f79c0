// K6 per-tile blend: one CTA per 16x16 tile, one pixel per thread.  The
// tile's depth-ordered list is consumed in batches of 256 Gaussians that are
// gathered into shared memory with cp.async (double-buffered: batch b+1 is in
// flight while batch b is composited).  Each pixel composites front to back
// (the 3DGS rasterizer of Sec. 4.1): alpha = min(0.99, o exp(power)), entries
// with alpha < 1/255 are skipped, and the pixel stops before the entry that
// would bring T below 1e-4.  Warp votes make the skip and the stop uniform:
// a warp skips the blend step when no lane gains from an entry, and leaves the
// batch once every lane has stopped; the CTA leaves the list once all 256
// pixels have stopped.  Warps cover 8x4 pixel blocks so their lanes stop at
// similar depths.
#include "kernels.cuh"
#include "sliced.cuh"

namespace tigas {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 256;
constexpr uint32_t kFull = 0xFFFFFFFFu;

struct __align__(16) BlendSmem {
    float4 geom[2][kBatch];
    float4 appear[2][kBatch];
    float blue[2][kBatch];
};

__device__ inline void cp_async16(void* smem, const void* gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ inline void cp_async4(void* smem, const void* gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ inline float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ inline uint8_t to_u8(float x) {
    return (uint8_t)__float2uint_rd(fminf(fmaxf(x, 0.0f), 1.0f) * 255.0f + 0.5f);
}

// SLICED = false: one CTA per tile (blockIdx.x), whole list, fresh pixels.
// SLICED = true: persistent CTAs take tiles from the slice's active list,
// start from and store back each pixel's (C, T), and mark finished tiles.
template <bool SLICED>
__global__ void __launch_bounds__(kThreads)
k_blend(const uint2* __restrict__ ranges, const uint32_t* __restrict__ values, SplatArrays sp,
        const ViewParams* __restrict__ views_g, int V, uint32_t n_entries, float bg_r, float bg_g, float bg_b,
        unsigned long long* counters, SliceBlendArgs sl) {
    __shared__ BlendSmem sm;
    __shared__ uint32_t s_tb[kMaxViews];
    __shared__ uint32_t s_item;
    for (int k = threadIdx.x; k < V; k += kThreads) s_tb[k] = views_g[k].tile_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t n_eval = 0, n_fetched = 0;
    const uint32_t n_items = SLICED ? *sl.n_active : 1u;
    for (;;) {
        uint32_t g;
        if (SLICED) {
            __syncthreads();   // previous tile done with shared memory and s_item
            if (threadIdx.x == 0) s_item = atomicAdd(sl.work_counter, 1u);
            __syncthreads();
            if (s_item >= n_items) break;
            g = sl.active[s_item];
        } else {
            __syncthreads();
            g = blockIdx.x;
        }
        int v = 0;
        {
            int lo = 0, hi = V;   // last view with tile_base <= g
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_tb[mid] <= g) lo = mid; else hi = mid;
            }
            v = lo;
        }
        const ViewParams& vp = views_g[v];
        const int W = vp.W, H = vp.H, TX = vp.TX;
        const uint32_t local = g - s_tb[v];
        const int ty = (int)(local / TX), tx = (int)(local % TX);
        const int px = tx * kTile + (warp & 1) * 8 + (lane & 7);
        const int py = ty * kTile + (warp >> 1) * 4 + (lane >> 3);
        const bool inside = px < W && py < H;
        const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
        const size_t pix = (size_t)py * W + px;

        const uint2 rg = ranges[g];
        const uint32_t start = rg.x, end = rg.y > rg.x ? rg.y : rg.x;
        const int nb = (int)((end - start + kBatch - 1) / kBatch);

        float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
        bool done = !inside;
        if (SLICED && inside) {
            const float4 s0 = sl.state[sl.pix_base[v] + pix];
            cr = s0.x; cg = s0.y; cb = s0.z;
            T = fabsf(s0.w);
            done = s0.w < 0.0f;
        }

        auto stage = [&](int b, int buf) {
            const uint32_t idx = start + (uint32_t)b * kBatch + threadIdx.x;
            if (idx < end) {
                const uint32_t e = values[idx];
                if (e < n_entries) {
                    cp_async16(&sm.geom[buf][threadIdx.x], sp.geom + e);
                    cp_async16(&sm.appear[buf][threadIdx.x], sp.appear + e);
                    cp_async4(&sm.blue[buf][threadIdx.x], sp.blue + e);
                } else {
                    // out-of-range entry (cannot happen for a consistent frame): contributes nothing
                    sm.geom[buf][threadIdx.x] = make_float4(-1e30f, -1e30f, 0.f, 0.f);
                    sm.appear[buf][threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                    sm.blue[buf][threadIdx.x] = 0.f;
                }
            }
            cp_async_commit();
        };

        if (nb > 0) stage(0, 0);
        for (int b = 0; b < nb; ++b) {
            const int buf = b & 1;
            if (b + 1 < nb) {
                stage(b + 1, buf ^ 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            // all pixels of the tile stopped: leave the list
            if (__syncthreads_count(done) == kThreads) break;
            const uint32_t rem = end - start - (uint32_t)b * kBatch;
            const int cnt = rem < (uint32_t)kBatch ? (int)rem : kBatch;
            n_fetched += (uint32_t)cnt;
            for (int j = 0; j < cnt; ++j) {
                if (__all_sync(kFull, done)) break;
                const float4 gm = sm.geom[buf][j];
                const float4 ap = sm.appear[buf][j];
                const float dx = gm.x - pxf, dy = gm.y - pyf;
                // power * log2(e), with the conic pre-scaled by -log2(e)/2 (off-diagonal -log2(e))
                const float p = fmaf(gm.z * dx, dx, fmaf(ap.x * dy, dy, gm.w * dx * dy));
                const float alpha = fminf(0.99f, ap.y * ex2_approx(p));
                const bool contrib = !done && p <= 0.0f && alpha >= (1.0f / 255.0f);
                n_eval += done ? 0u : 1u;
                if (__any_sync(kFull, contrib)) {
                    if (contrib) {
                        const float test_T = T * (1.0f - alpha);
                        if (test_T < 1e-4f) {
                            done = true;
                        } else {
                            const float w = alpha * T;
                            cr = fmaf(ap.z, w, cr);
                            cg = fmaf(ap.w, w, cg);
                            cb = fmaf(sm.blue[buf][j], w, cb);
                            T = test_T;
                        }
                    }
                }
            }
            __syncthreads();   // buffer `buf` is refilled by the next iteration's stage
        }
        cp_async_wait<0>();

        if (inside) {
            if (SLICED) sl.state[sl.pix_base[v] + pix] = make_float4(cr, cg, cb, done ? -T : T);
            const float r = fmaf(T, bg_r, cr), gg = fmaf(T, bg_g, cg), bb = fmaf(T, bg_b, cb), a = 1.0f - T;
            if (vp.out_rgba8) {
                const uchar4 o = make_uchar4(to_u8(r), to_u8(gg), to_u8(bb), to_u8(a));
                reinterpret_cast<uchar4*>(vp.out_rgba8)[pix] = o;
            }
            if (vp.out_rgba_f32) reinterpret_cast<float4*>(vp.out_rgba_f32)[pix] = make_float4(r, gg, bb, a);
        }
        if (SLICED) {
            if (__syncthreads_count(done) == kThreads && threadIdx.x == 0) atomicOr(&sl.done[g >> 5], 1u << (g & 31));
        } else {
            break;
        }
    }
    if (counters) {
        uint32_t s = n_eval;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
        if (lane == 0 && s) atomicAdd(&counters[0], (unsigned long long)s);
        if (threadIdx.x == 0 && n_fetched) atomicAdd(&counters[1], (unsigned long long)n_fetched);
    }
}

}  // namespace

Status launch_blend(const uint2* ranges, const uint32_t* values, const SplatArrays& sp, const ViewParams* views,
                    int V, uint32_t total_tiles, uint32_t n_entries, const float* bg, unsigned long long* counters,
                    cudaStream_t st) {
    if (total_tiles == 0) return {};
    k_blend<false><<<total_tiles, kThreads, 0, st>>>(ranges, values, sp, views, V, n_entries, bg[0], bg[1], bg[2],
                                                     counters, SliceBlendArgs{});
    TIGAS_LAUNCHED();
    return {};
}

Status launch_blend_slice(const uint2* ranges, const uint32_t* values, const SplatArrays& sp,
                          const ViewParams* views, int V, uint32_t n_entries, const float* bg,
                          unsigned long long* counters, const SliceBlendArgs& sl, cudaStream_t st) {
    static int grid = 0;
    if (grid == 0) {
        int per_sm = 0;
        TIGAS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blend<true>, kThreads, 0));
        int dev = 0, sms = 0;
        TIGAS_CUDA_TRY(cudaGetDevice(&dev));
        TIGAS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        grid = (per_sm > 0 ? per_sm : 1) * sms;
    }
    TIGAS_CUDA_TRY(cudaMemsetAsync(sl.work_counter, 0, sizeof(uint32_t), st));
    k_blend<true><<<grid, kThreads, 0, st>>>(ranges, values, sp, views, V, n_entries, bg[0], bg[1], bg[2], counters,
                                             sl);
    TIGAS_LAUNCHED();
    return {};
}

}  // namespace tigas
