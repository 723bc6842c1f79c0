// K6 per-tile blend: one 16x16 tile per CTA of 128 threads, two pixels per
// thread (rows y and y + 4 of the thread's warp's 8x8 block).  The tile's
// depth-ordered list is consumed in batches of 256 Gaussians gathered into
// shared memory with cp.async, double-buffered (batch b+1 in flight while b is
// composited), so each staged entry's shared-memory loads serve two pixels.
// Each pixel composites front to back (the 3DGS rasterizer of Sec. 4.1):
// alpha = min(0.99, o exp(power)), computed as 2^(power log2 e + log2 o);
// entries with alpha < 1/255 are skipped before any exponential, and the
// pixel stops before the entry that would bring T below 1e-4.  Warp votes make
// the skip and the stop uniform: a warp skips the blend step when no lane
// gains from an entry and leaves the batch once all its pixels have stopped;
// the CTA leaves the list once all 256 pixels have stopped.
#include "kernels.cuh"
#include "sliced.cuh"

namespace tigas {

namespace {

constexpr int kThreads = 128;
constexpr int kBatch = 256;
// alpha >= 1/255  <=>  power log2 e + log2 o >= log2(1/255)
constexpr float kMinLog2Alpha = -7.99435343685885793f;
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
// COUNT: accumulate list entries evaluated per pixel and entries staged.
template <bool SLICED, bool COUNT>
__global__ void __launch_bounds__(kThreads)
k_blend(const uint2* __restrict__ ranges, const uint32_t* __restrict__ values, SplatArrays sp,
        const ViewParams* __restrict__ views_g, int V, uint32_t n_entries, float bg_r, float bg_g, float bg_b,
        unsigned long long* counters, SliceBlendArgs sl) {
    __shared__ BlendSmem sm;
    __shared__ uint32_t s_tb[kMaxViews];
    __shared__ uint32_t s_item;
    for (int k = threadIdx.x; k < V; k += kThreads) s_tb[k] = views_g[k].tile_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t n_eval = 0, n_fetched = 0, n_blend = 0;
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
        const int py0 = ty * kTile + (warp >> 1) * 8 + (lane >> 3);
        const int py1 = py0 + 4;
        const bool in0 = px < W && py0 < H, in1 = px < W && py1 < H;
        const float pxf = (float)px + 0.5f, py0f = (float)py0 + 0.5f;
        const size_t pix0 = (size_t)py0 * W + px, pix1 = (size_t)py1 * W + px;

        const uint2 rg = ranges[g];
        const uint32_t start = rg.x, end = rg.y > rg.x ? rg.y : rg.x;
        const int nb = (int)((end - start + kBatch - 1) / kBatch);

        float T0 = 1.0f, r0 = 0.0f, g0 = 0.0f, b0 = 0.0f;
        float T1 = 1.0f, r1 = 0.0f, g1 = 0.0f, b1 = 0.0f;
        bool d0 = !in0, d1 = !in1;
        if (SLICED) {
            if (in0) {
                const float4 s0 = sl.state[sl.pix_base[v] + pix0];
                r0 = s0.x; g0 = s0.y; b0 = s0.z; T0 = fabsf(s0.w); d0 = s0.w < 0.0f;
            }
            if (in1) {
                const float4 s1 = sl.state[sl.pix_base[v] + pix1];
                r1 = s1.x; g1 = s1.y; b1 = s1.z; T1 = fabsf(s1.w); d1 = s1.w < 0.0f;
            }
        }

        auto stage = [&](int b, int buf) {
#pragma unroll
            for (int h = 0; h < kBatch / kThreads; ++h) {
                const int slot = h * kThreads + threadIdx.x;
                const uint32_t idx = start + (uint32_t)b * kBatch + slot;
                if (idx < end) {
                    const uint32_t e = values[idx];
                    if (e < n_entries) {
                        cp_async16(&sm.geom[buf][slot], sp.geom + e);
                        cp_async16(&sm.appear[buf][slot], sp.appear + e);
                        cp_async4(&sm.blue[buf][slot], sp.blue + e);
                    } else {
                        // out-of-range entry (cannot happen for a consistent frame): contributes nothing
                        sm.geom[buf][slot] = make_float4(-1e30f, -1e30f, 0.f, 0.f);
                        sm.appear[buf][slot] = make_float4(0.f, -1e30f, 0.f, 0.f);
                        sm.blue[buf][slot] = 0.f;
                    }
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
            if (__syncthreads_count(d0 && d1) == kThreads) break;
            const uint32_t rem = end - start - (uint32_t)b * kBatch;
            const int cnt = rem < (uint32_t)kBatch ? (int)rem : kBatch;
            if (COUNT) n_fetched += (uint32_t)cnt;
#pragma unroll 4
            for (int j = 0; j < cnt; ++j) {
                if ((j & 3) == 0 && __all_sync(kFull, d0 && d1)) break;
                const float4 gm = sm.geom[buf][j];     // (u, v, a', b')
                const float4 ap = sm.appear[buf][j];   // (c', log2 o, r, g)
                const float dx = gm.x - pxf;
                const float dy0 = gm.y - py0f;
                const float dy1 = dy0 - 4.0f;
                const float adx = gm.z * dx, bdx = gm.w * dx;
                // power log2 e = a' dx^2 + dy (b' dx + c' dy)
                const float p0 = fmaf(adx, dx, dy0 * fmaf(ap.x, dy0, bdx));
                const float p1 = fmaf(adx, dx, dy1 * fmaf(ap.x, dy1, bdx));
                const float e0 = p0 + ap.y, e1 = p1 + ap.y;
                const bool c0 = !d0 && p0 <= 0.0f && e0 >= kMinLog2Alpha;
                const bool c1 = !d1 && p1 <= 0.0f && e1 >= kMinLog2Alpha;
                if (COUNT) n_eval += (d0 ? 0u : 1u) + (d1 ? 0u : 1u);
                if (__any_sync(kFull, c0 || c1)) {
                    const float cb = sm.blue[buf][j];
                    if (c0) {
                        const float alpha = fminf(0.99f, ex2_approx(e0));
                        const float tT = fmaf(-T0, alpha, T0);
                        if (tT < 1e-4f) {
                            d0 = true;
                        } else {
                            if (COUNT) ++n_blend;
                            const float w = alpha * T0;
                            r0 = fmaf(ap.z, w, r0);
                            g0 = fmaf(ap.w, w, g0);
                            b0 = fmaf(cb, w, b0);
                            T0 = tT;
                        }
                    }
                    if (c1) {
                        const float alpha = fminf(0.99f, ex2_approx(e1));
                        const float tT = fmaf(-T1, alpha, T1);
                        if (tT < 1e-4f) {
                            d1 = true;
                        } else {
                            if (COUNT) ++n_blend;
                            const float w = alpha * T1;
                            r1 = fmaf(ap.z, w, r1);
                            g1 = fmaf(ap.w, w, g1);
                            b1 = fmaf(cb, w, b1);
                            T1 = tT;
                        }
                    }
                }
            }
            __syncthreads();   // buffer `buf` is refilled by the next iteration's stage
        }
        cp_async_wait<0>();

        if (in0) {
            if (SLICED) sl.state[sl.pix_base[v] + pix0] = make_float4(r0, g0, b0, d0 ? -T0 : T0);
            const float r = fmaf(T0, bg_r, r0), gg = fmaf(T0, bg_g, g0), bb = fmaf(T0, bg_b, b0), a = 1.0f - T0;
            if (vp.out_rgba8)
                reinterpret_cast<uchar4*>(vp.out_rgba8)[pix0] = make_uchar4(to_u8(r), to_u8(gg), to_u8(bb), to_u8(a));
            if (vp.out_rgba_f32) reinterpret_cast<float4*>(vp.out_rgba_f32)[pix0] = make_float4(r, gg, bb, a);
        }
        if (in1) {
            if (SLICED) sl.state[sl.pix_base[v] + pix1] = make_float4(r1, g1, b1, d1 ? -T1 : T1);
            const float r = fmaf(T1, bg_r, r1), gg = fmaf(T1, bg_g, g1), bb = fmaf(T1, bg_b, b1), a = 1.0f - T1;
            if (vp.out_rgba8)
                reinterpret_cast<uchar4*>(vp.out_rgba8)[pix1] = make_uchar4(to_u8(r), to_u8(gg), to_u8(bb), to_u8(a));
            if (vp.out_rgba_f32) reinterpret_cast<float4*>(vp.out_rgba_f32)[pix1] = make_float4(r, gg, bb, a);
        }
        if (SLICED) {
            if (__syncthreads_count(d0 && d1) == kThreads && threadIdx.x == 0)
                atomicOr(&sl.done[g >> 5], 1u << (g & 31));
        } else {
            break;
        }
    }
    if (COUNT && counters) {
        uint32_t s = n_eval;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
        if (lane == 0 && s) atomicAdd(&counters[0], (unsigned long long)s);
        uint32_t c = n_blend;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
        if (lane == 0 && c) atomicAdd(&counters[2], (unsigned long long)c);
        if (threadIdx.x == 0 && n_fetched) atomicAdd(&counters[1], (unsigned long long)n_fetched);
    }
}

}  // namespace

Status launch_blend(const uint2* ranges, const uint32_t* values, const SplatArrays& sp, const ViewParams* views,
                    int V, uint32_t total_tiles, uint32_t n_entries, const float* bg, unsigned long long* counters,
                    cudaStream_t st) {
    if (total_tiles == 0) return {};
    if (counters)
        k_blend<false, true><<<total_tiles, kThreads, 0, st>>>(ranges, values, sp, views, V, n_entries, bg[0], bg[1],
                                                               bg[2], counters, SliceBlendArgs{});
    else
        k_blend<false, false><<<total_tiles, kThreads, 0, st>>>(ranges, values, sp, views, V, n_entries, bg[0], bg[1],
                                                                bg[2], nullptr, SliceBlendArgs{});
    TIGAS_LAUNCHED();
    return {};
}

Status launch_blend_slice(const uint2* ranges, const uint32_t* values, const SplatArrays& sp,
                          const ViewParams* views, int V, uint32_t n_entries, const float* bg,
                          unsigned long long* counters, const SliceBlendArgs& sl, cudaStream_t st) {
    static int grid = 0;
    if (grid == 0) {
        int per_sm = 0;
        TIGAS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blend<true, false>, kThreads, 0));
        int dev = 0, sms = 0;
        TIGAS_CUDA_TRY(cudaGetDevice(&dev));
        TIGAS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        grid = (per_sm > 0 ? per_sm : 1) * sms;
    }
    TIGAS_CUDA_TRY(cudaMemsetAsync(sl.work_counter, 0, sizeof(uint32_t), st));
    if (counters)
        k_blend<true, true><<<grid, kThreads, 0, st>>>(ranges, values, sp, views, V, n_entries, bg[0], bg[1], bg[2],
                                                       counters, sl);
    else
        k_blend<true, false><<<grid, kThreads, 0, st>>>(ranges, values, sp, views, V, n_entries, bg[0], bg[1], bg[2],
                                                        nullptr, sl);
    TIGAS_LAUNCHED();
    return {};
}

}  // namespace tigas
