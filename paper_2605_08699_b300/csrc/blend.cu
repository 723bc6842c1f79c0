// K6 per-tile blend, the 3DGS front-to-back compositing the backend relies
// on (Sec. 4.1): one warp per 16x16 tile, 8 pixels per thread (column
// lane % 16, rows lane / 16 + 2k), four independent warps per CTA and no
// CTA-wide barrier; a tile with a long list in a slice is split into strips
// of 8 rows (two 16x8 halves, 4 pixels per thread) or, for the longest lists
// of the slices whose tail they set, 4 rows (2 pixels per thread), that
// separate warps composite at once.  The tile's depth-ordered list is
// consumed in batches of 32 entries that the warp gathers into shared memory
// with cp.async, double-buffered (batch b+1 in flight while b is composited).
//
// For each staged entry the warp first tests the bounding box of its
// alpha >= 1/255 region against the bounding box of the tile's pixels that are
// still compositing; a ballot over the batch keeps only entries that can reach
// one of them (a result-invariant skip: a pixel the box excludes would skip
// the entry by the alpha test, a pixel that stopped ignores it).  For
// the kept entries each pixel computes alpha = min(0.99, o exp(power)) as
// 2^(power log2 e + log2 o) (two FMAs per pixel after the row-independent part),
// skips alpha < 1/255 before any exponential, and
// stops before the entry that would bring T below 1e-4.  The blend step takes
// a thread's pixel rows in pairs, one branch per pair that some pixel of the
// warp takes (a row that does not take the entry blends with alpha 0, which
// leaves it unchanged bit for bit), and the warp leaves the list once all its
// pixels have stopped.
#include "kernels.cuh"
#include "sliced.cuh"

namespace tigas {

namespace {

constexpr int kWarps = 4;                 // tiles per CTA
constexpr int kThreads = 32 * kWarps;
// Entries per warp batch (a schedule parameter): 32 (one per lane) or 16.
constexpr int kPix = 8;                   // pixels per thread
#ifndef TIGAS_BLEND_MIN_BLOCKS
#define TIGAS_BLEND_MIN_BLOCKS 8
#endif
constexpr int kMinBlocks = TIGAS_BLEND_MIN_BLOCKS;   // CTAs per SM the register budget targets
constexpr uint32_t kFull = 0xFFFFFFFFu;
// alpha >= 1/255  <=>  power log2 e + log2 o >= log2(1/255)
constexpr float kMinLog2Alpha = -7.99435343685885793f;

// Batches in flight per warp: the gathers of the next kStages - 1 batches are
// issued while one is composited, and each batch's list indices are loaded
// one batch before its gather (so a batch costs one memory round trip, not
// two, when compositing it is quick, as in the late slices' long lists).
// Measured on the 8-view 1080p launch set: 2 stages with the index prefetch
// 1.287 ms of blend, without it 1.319; 3 stages 1.307, 4 stages 1.421 (the
// larger shared-memory share leaves less L1).
#ifndef TIGAS_BLEND_STAGES
#define TIGAS_BLEND_STAGES 2
#endif
constexpr int kStages = TIGAS_BLEND_STAGES;
static_assert(kStages >= 2 && kStages <= 4, "two to four staging buffers");

template <int kWB>
struct __align__(16) WarpStage {
    static_assert(kWB >= 1 && kWB <= 32, "a batch holds one entry per lane at most");
    float4 geom[kStages][kWB];     // (u, v, a', b')
    float4 appear[kStages][kWB];   // (c', log2 o, r, g)
    float blue[kStages][kWB];
};

// 16-byte gathers bypass L1 (.cg; measured a little ahead of .ca: blend 1.109 -> 1.106 ms)
__device__ inline void cp_async16(void* smem, const void* gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ inline void cp_async4(void* smem, const void* gmem) {
    uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

#ifndef TIGAS_BLEND_F32X2
#define TIGAS_BLEND_F32X2 1
#endif
// Packed two-lane FP32 arithmetic (each lane rounds as the scalar instruction).
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ inline float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// floor(clamp(x, 0, 1) 255 + 0.5) with one rounding of the fused x 255 + 0.5
__device__ inline uint8_t to_u8(float x) {
    return (uint8_t)__float2uint_rd(__fmaf_rn(fminf(fmaxf(x, 0.0f), 1.0f), 255.0f, 0.5f));
}

#ifndef TIGAS_BOX_APPROX
#define TIGAS_BOX_APPROX 1
#endif

// Does the alpha >= 1/255 region of the entry meet the pixel-centre rectangle
// [x0, x1] x [y0, y1]?  With q(d) = -(a' dx^2 + b' dx dy + c' dy^2) (positive
// definite) the region is q(d) <= tau = log2 o - log2(1/255), an ellipse with
// half-extents sqrt(tau (M^-1)_xx), sqrt(tau (M^-1)_yy), M = [[-a', -b'/2],
// [-b'/2, -c']]; inflated by 1% + 0.05 px so FP32 rounding of the per-pixel
// test can never put a contributing pixel outside it.
__device__ inline bool alpha_box_meets(const float4& gm, const float4& ap, float x0, float x1, float y0, float y1) {
    const float tau = ap.y - kMinLog2Alpha;
    const float m00 = -gm.z, m11 = -ap.x, m01 = -0.5f * gm.w;
    const float det = fmaf(m00, m11, -m01 * m01);
    if (!(tau >= 0.0f) || !(det > 0.0f)) return false;
#if TIGAS_BOX_APPROX
    // hardware division and square roots: the 1 % + 0.05 px inflation covers their error
    const float inv = __fdividef(tau, det);
    float hx, hy;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(hx) : "f"(m11 * inv));
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(hy) : "f"(m00 * inv));
    hx = fmaf(hx, 1.01f, 0.05f);
    hy = fmaf(hy, 1.01f, 0.05f);
#else
    const float inv = tau / det;
    const float hx = fmaf(sqrtf(m11 * inv), 1.01f, 0.05f);
    const float hy = fmaf(sqrtf(m00 * inv), 1.01f, 0.05f);
#endif
    return gm.x - hx <= x1 && gm.x + hx >= x0 && gm.y - hy <= y1 && gm.y + hy >= y0;
}

#ifndef TIGAS_BLEND_EXACT_CULL
#define TIGAS_BLEND_EXACT_CULL 1
#endif
// The same question answered exactly for the ellipse (the bounding box above
// keeps entries whose ellipse misses the rectangle but whose box does not):
// is the minimum of q(mu - p) over p in [x0, x1] x [y0, y1] at most tau?  q is
// convex, so the minimum is 0 when mu lies in the rectangle, else it lies on a
// side that faces mu (at most two): on the side x = xe the best dy is
// -m01 dx / m11 clamped to the side, on y = ye the best dx is -m01 dy / m00.
// The answer is widened (tau 1.02 + 0.02, and any point of a side counts) so
// that FP32 rounding here or in the per-pixel test can never drop an entry a
// pixel takes: a pixel centre inside the rectangle with
// q(mu - p) <= tau has min <= q(mu - p) <= tau.
__device__ inline bool alpha_ellipse_meets(const float4& gm, const float4& ap, float x0, float x1, float y0,
                                           float y1) {
    const float tau = ap.y - kMinLog2Alpha;
    const float m00 = -gm.z, m11 = -ap.x, m01 = -0.5f * gm.w;
    const float det = fmaf(m00, m11, -m01 * m01);
    if (!(tau >= 0.0f) || !(det > 0.0f)) return false;
    const float u = gm.x, v = gm.y;
    const float xe = fminf(fmaxf(u, x0), x1), ye = fminf(fmaxf(v, y0), y1);
    if (xe == u && ye == v) return true;   // the centre lies in the rectangle
    const float lim = fmaf(tau, 1.02f, 0.02f);
    float best = __int_as_float(0x7f800000);
    if (xe != u) {   // the side x = xe
        const float dx = u - xe;
        const float dy = fminf(fmaxf(__fdividef(-m01 * dx, m11), v - y1), v - y0);
        best = fminf(best, fmaf(m00 * dx, dx, dy * fmaf(2.0f * m01, dx, m11 * dy)));
    }
    if (ye != v) {   // the side y = ye
        const float dy = v - ye;
        const float dx = fminf(fmaxf(__fdividef(-m01 * dy, m00), u - x1), u - x0);
        best = fminf(best, fmaf(m11 * dy, dy, dx * fmaf(2.0f * m01, dy, m00 * dx)));
    }
    return best <= lim;
}

struct BlendCounts {
    unsigned long long eval = 0, fetched = 0, blend = 0;
};

// One warp composites tile g's list onto 2 NP pixel rows of the tile, starting
// at row0: thread lane takes column lane % 16 and rows row0 + lane / 16 + 2k,
// k < NP.  SLICED: start from and store back each pixel's carried (C, T).
// Returns (warp-uniform) whether every pixel of these rows has stopped.
template <bool SLICED, bool COUNT, int NP, int kWB>
__device__ __forceinline__ bool blend_rows(WarpStage<kWB>& sm, int lane, const uint2* __restrict__ ranges,
                                           const uint32_t* __restrict__ values, const SplatArrays& sp,
                                           const ViewParams& vp, uint32_t g, uint32_t local, int row0,
                                           uint64_t sbase, uint32_t n_entries, float bg_r, float bg_g, float bg_b,
                                           const SliceBlendArgs& sl, BlendCounts& cnt) {
    static_assert(NP % 2 == 0, "the blend step takes pixel rows in pairs");
    const int W = vp.W, H = vp.H, TX = vp.TX;
    const int ty = (int)(local / TX), tx = (int)(local % TX);
    const uint32_t col = lane & 15, row = (uint32_t)row0 + (lane >> 4);   // rows row + 2k of the tile
    const int px = tx * kTile + (int)col;
    const int py0 = ty * kTile + (int)row;
    const float pxf = (float)px + 0.5f, py0f = (float)py0 + 0.5f;
    const float tx0 = (float)(tx * kTile) + 0.5f, ty0 = (float)(ty * kTile) + 0.5f;   // first pixel centre

    float T[NP], cr[NP], cg[NP], cb[NP];
    uint32_t live = 0;   // bit k: pixel k still compositing
    // the tile's pixels carry (C, T) from an earlier slice (kStripSeen: set only
    // between slices, so the strips of a long tile, which run in the same slice,
    // all see the same value); otherwise they start from (0, 1).  The state is
    // read together with the strip word rather than after it (one dependent
    // load less per visit; on a first visit the words read are in bounds and
    // unused)
    const uint32_t sw = SLICED ? sl.strips[g] : 0u;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        T[k] = 1.0f; cr[k] = 0.0f; cg[k] = 0.0f; cb[k] = 0.0f;
        const int py = py0 + 2 * k;
        if (px < W && py < H) {
            if (SLICED) {
                const float4 s0 = sl.state[sbase + (size_t)py * W + px];
                if (sw & kStripSeen) {
                    cr[k] = s0.x; cg[k] = s0.y; cb[k] = s0.z; T[k] = fabsf(s0.w);
                    if (!(s0.w < 0.0f)) live |= 1u << k;
                } else {
                    live |= 1u << k;
                }
            } else {
                live |= 1u << k;
            }
        }
    }

    float thr[NP];   // per pixel: log2 of the smallest alpha that counts, or +inf (not compositing)
#pragma unroll
    for (int k = 0; k < NP; ++k) thr[k] = ((live >> k) & 1u) ? kMinLog2Alpha : __int_as_float(0x7f800000);

    const uint2 rg = ranges[g];
    const uint32_t start = rg.x, end = rg.y > rg.x ? rg.y : rg.x;
    const int nb = (int)((end - start + kWB - 1) / kWB);
    // the lane's entry of batch b, or ~0u past the list (loaded a batch ahead of its gather)
    auto index_of = [&](int b) -> uint32_t {
        const uint32_t idx = start + (uint32_t)b * kWB + lane;
        return lane < kWB && idx < end ? values[idx] : ~0u;
    };
    auto stage = [&](uint32_t e, int buf) {   // one staged entry per lane of the batch
        if (e < n_entries) {
            cp_async16(&sm.geom[buf][lane], sp.geom + e);
            cp_async16(&sm.appear[buf][lane], sp.appear + e);
            cp_async4(&sm.blue[buf][lane], sp.blue + e);
        } else if (e != ~0u) {
            // out-of-range entry (cannot happen for a consistent frame): contributes nothing
            sm.geom[buf][lane] = make_float4(-1e30f, -1e30f, 0.f, 0.f);
            sm.appear[buf][lane] = make_float4(0.f, -1e30f, 0.f, 0.f);
            sm.blue[buf][lane] = 0.f;
        }
    };

    // prologue: gathers of batches 0 .. kStages - 2 in flight, the indices of the next one loaded
#pragma unroll
    for (int q = 0; q < kStages - 1; ++q) {
        if (q < nb) stage(index_of(q), q);
        cp_async_commit();   // one group per batch slot, empty past the list (uniform group counts)
    }
    uint32_t e_next = kStages - 1 < nb ? index_of(kStages - 1) : ~0u;
    for (int b = 0; b < nb; ++b) {
        const int buf = b % kStages;
        {
            // the gather of batch b + kStages - 1 into the buffer batch b - 1 used, then the
            // indices of the batch after it
            const int bn = b + kStages - 1;
            if (bn < nb) stage(e_next, bn % kStages);
            cp_async_commit();
            e_next = bn + 1 < nb ? index_of(bn + 1) : ~0u;
        }
        cp_async_wait<kStages - 1>();   // batch b's group has landed
        const uint32_t rem = end - start - (uint32_t)b * kWB;
        const int n_b = rem < (uint32_t)kWB ? (int)rem : kWB;
        if (__all_sync(kFull, live == 0)) break;
        // bounding box of the pixels still compositing (at least one is)
        const uint32_t c_lo = __reduce_min_sync(kFull, live ? col : 16u);
        const uint32_t c_hi = __reduce_max_sync(kFull, live ? col : 0u);
        const uint32_t r_lo = __reduce_min_sync(kFull, live ? row + 2u * (uint32_t)(__ffs(live) - 1) : 16u);
        const uint32_t r_hi = __reduce_max_sync(kFull, live ? row + 2u * (uint32_t)(31 - __clz(live)) : 0u);
        // the lane's own staged entry: can it reach one of those pixels?
        bool meets = lane < n_b && alpha_box_meets(sm.geom[buf][lane], sm.appear[buf][lane], tx0 + (float)c_lo,
                                                   tx0 + (float)c_hi, ty0 + (float)r_lo, ty0 + (float)r_hi);
        if (TIGAS_BLEND_EXACT_CULL && meets)
            meets = alpha_ellipse_meets(sm.geom[buf][lane], sm.appear[buf][lane], tx0 + (float)c_lo,
                                        tx0 + (float)c_hi, ty0 + (float)r_lo, ty0 + (float)r_hi);
        uint32_t kept = __ballot_sync(kFull, meets);
        __syncwarp();   // every lane's copies visible to the warp
        if (COUNT) cnt.fetched += (uint64_t)n_b;
        int counted = 0;   // entries of this batch already counted as evaluated
        bool stopped = false;
        while (kept) {
            const int j = __ffs(kept) - 1;
            kept &= kept - 1;
            if (COUNT) {
                // entries up to and including j meet the pixels still running before j
                cnt.eval += (uint64_t)(j + 1 - counted) * (uint64_t)__popc(live);
                counted = j + 1;
            }
            const float4 gm = sm.geom[buf][j];
            const float4 ap = sm.appear[buf][j];
            const float dx = gm.x - pxf;
            const float bdx = gm.w * dx;
            // log2(o exp(power)) = (a' dx^2 + log2 o) + dy (b' dx + c' dy); the
            // quadratic form is negative definite, so power <= 0 needs no test
            const float p0 = fmaf(gm.z * dx, dx, ap.y);
            const float dyb = gm.y - py0f;
            float e[NP];
            bool con[NP];
            if constexpr (TIGAS_BLEND_F32X2 != 0 && NP % 2 == 0) {
                // rows k = 2j, 2j + 1 in one packed lane pair: dy = dyb - 2k, e = dy (c' dy + b' dx) + p0
                const unsigned long long dyb2 = f2_pack(dyb, dyb), ax2 = f2_pack(ap.x, ap.x);
                const unsigned long long bdx2 = f2_pack(bdx, bdx), p02 = f2_pack(p0, p0);
#pragma unroll
                for (int j = 0; j < NP / 2; ++j) {
                    const unsigned long long dy2 = f2_add(dyb2, f2_pack(-4.0f * (float)j, -4.0f * (float)j - 2.0f));
                    const unsigned long long e2 = f2_fma(dy2, f2_fma(ax2, dy2, bdx2), p02);
                    f2_unpack(e2, e[2 * j], e[2 * j + 1]);
                }
#pragma unroll
                for (int k = 0; k < NP; ++k)
                    con[k] = e[k] >= thr[k];   // thr: the alpha cut-off, +inf once the pixel stopped
            } else {
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const float dy = dyb - 2.0f * (float)k;
                    e[k] = fmaf(dy, fmaf(ap.x, dy, bdx), p0);
                    con[k] = e[k] >= thr[k];   // thr: the alpha cut-off, +inf once the pixel stopped
                }
            }
            {
                // The blend step, two pixel rows per branch.  A row that does not take
                // the entry gets alpha = 0, and the step leaves it unchanged bit for bit:
                // T - T 0 = T (one fused rounding) and C + c (0 T) = C.  Only a pair in
                // which some pixel stops takes the per-pixel path.  (Fewer, less
                // divergent branches than one per row, and no warp vote before them.)
                const float cbl = sm.blue[buf][j];
#pragma unroll
                for (int q = 0; q < NP / 2; ++q) {
                    const int k0 = 2 * q, k1 = 2 * q + 1;
                    if (con[k0] || con[k1]) {
                        const float a0 = con[k0] ? fminf(0.99f, ex2_approx(e[k0])) : 0.0f;
                        const float a1 = con[k1] ? fminf(0.99f, ex2_approx(e[k1])) : 0.0f;
                        const float t0 = fmaf(-T[k0], a0, T[k0]);
                        const float t1 = fmaf(-T[k1], a1, T[k1]);
                        if (t0 < 1e-4f || t1 < 1e-4f) {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int k = k0 + h;
                                const float a = h ? a1 : a0, tT = h ? t1 : t0;
                                if (!con[k]) continue;
                                if (tT < 1e-4f) {   // stops before this entry
                                    live &= ~(1u << k);
                                    thr[k] = __int_as_float(0x7f800000);
                                } else {
                                    if (COUNT) ++cnt.blend;
                                    const float w = a * T[k];
                                    cr[k] = fmaf(ap.z, w, cr[k]);
                                    cg[k] = fmaf(ap.w, w, cg[k]);
                                    cb[k] = fmaf(cbl, w, cb[k]);
                                    T[k] = tT;
                                }
                            }
                        } else {
                            if (COUNT) cnt.blend += (uint64_t)con[k0] + (uint64_t)con[k1];
                            const float w0 = a0 * T[k0], w1 = a1 * T[k1];
                            cr[k0] = fmaf(ap.z, w0, cr[k0]);
                            cg[k0] = fmaf(ap.w, w0, cg[k0]);
                            cb[k0] = fmaf(cbl, w0, cb[k0]);
                            cr[k1] = fmaf(ap.z, w1, cr[k1]);
                            cg[k1] = fmaf(ap.w, w1, cg[k1]);
                            cb[k1] = fmaf(cbl, w1, cb[k1]);
                            T[k0] = t0;
                            T[k1] = t1;
                        }
                    }
                }
                if (__all_sync(kFull, live == 0)) {
                    stopped = true;
                    break;
                }
            }
        }
        if (COUNT && !stopped) cnt.eval += (uint64_t)(n_b - counted) * (uint64_t)__popc(live);
        __syncwarp();   // buffer `buf` is refilled by the next iteration's stage
    }
    cp_async_wait<0>();
    __syncwarp();

    const bool all = __all_sync(kFull, live == 0);
    // a whole tile whose pixels all stopped is done and never visited again: no state
    const bool keep = !(NP == kPix && all);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int py = py0 + 2 * k;
        if (px < W && py < H) {
            const size_t pix = (size_t)py * W + px;
            if (SLICED && keep)
                sl.state[sbase + pix] = make_float4(cr[k], cg[k], cb[k], ((live >> k) & 1u) ? T[k] : -T[k]);
            const float r = fmaf(T[k], bg_r, cr[k]), gg = fmaf(T[k], bg_g, cg[k]);
            const float bb = fmaf(T[k], bg_b, cb[k]), a = 1.0f - T[k];
            if (vp.out_rgba8)
                reinterpret_cast<uchar4*>(vp.out_rgba8)[pix] = make_uchar4(to_u8(r), to_u8(gg), to_u8(bb), to_u8(a));
            if (vp.out_rgba_f32) reinterpret_cast<float4*>(vp.out_rgba_f32)[pix] = make_float4(r, gg, bb, a);
        }
    }
    // the tile's pixels now carry state (and have their outputs written)
    if (SLICED && !(sw & kStripSeen) && lane == 0) atomicOr(&sl.strips[g], kStripSeenNow);
    return all;
}

// SLICED = false: warp w of CTA b blends tile 4b + w over its whole list from
// fresh pixels.  SLICED = true: persistent warps take items from the slice's
// active list (a whole tile, or one 4-row strip of a long tile), carry each
// pixel's (C, T) across slices, and mark tiles whose pixels all stopped.
// COUNT: accumulate list entries evaluated per pixel (up to its stop), entries
// staged, and entries blended.
template <bool SLICED, bool COUNT, int kWB>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
k_blend(const uint2* __restrict__ ranges, const uint32_t* __restrict__ values, SplatArrays sp,
        const ViewParams* __restrict__ views_g, int V, uint32_t total_tiles, uint32_t n_entries, float bg_r,
        float bg_g, float bg_b, unsigned long long* counters, SliceBlendArgs sl) {
    __shared__ WarpStage<kWB> stage_sm[kWarps];
    __shared__ uint32_t s_tb[kMaxViews];
    for (int k = threadIdx.x; k < V; k += kThreads) s_tb[k] = views_g[k].tile_base;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpStage<kWB>& sm = stage_sm[warp];
    BlendCounts cnt;
    // the strips of the longest lists (from the front), of the other long lists (from the
    // middle down), then whole tiles (from the back)
    const uint32_t n_first = SLICED ? sl.n_active[0] : 0u;
    const uint32_t n_long = SLICED ? n_first + sl.n_active[3] : 0u;
    const uint32_t n_items = SLICED ? n_long + sl.n_active[1] : total_tiles;
    uint32_t item = SLICED ? 0u : blockIdx.x * kWarps + warp;
    for (;;) {
        if (SLICED) {
            uint32_t it = 0;
            if (lane == 0) it = atomicAdd(sl.work_counter, 1u);
            item = __shfl_sync(kFull, it, 0);
        }
        if (item >= n_items) break;
        // regions: [0, 4n) up, [4n, 6n) down from 6n - 1, [6n, 7n) down from 7n - 1
        const uint32_t n7 = sl.active_cap / kActivePerTile;
        const uint32_t raw = !SLICED ? item
                             : sl.active[item < n_first  ? item
                                         : item < n_long ? 6u * n7 - 1u - (item - n_first)
                                                         : 7u * n7 - 1u - (item - n_long)];
        const uint32_t g = raw & kTileMask;
        const uint32_t code = raw >> kStripShift;   // 0: whole tile, else a strip (kCode8 + s, kCode4 + s)
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
        const uint32_t local = g - s_tb[v];
        const uint64_t sbase = SLICED ? sl.pix_base[v] : 0;
        if (!SLICED || code == 0) {
            const bool all = blend_rows<SLICED, COUNT, kPix, kWB>(sm, lane, ranges, values, sp, vp, g, local, 0, sbase,
                                                             n_entries, bg_r, bg_g, bg_b, sl, cnt);
            if (!SLICED) break;
            if (all && lane == 0) atomicOr(&sl.done[g >> 5], 1u << (g & 31));
        } else {
            const bool eight = code < kCode4;
            const uint32_t s = code - (eight ? kCode8 : kCode4);
            const bool all =
                eight ? blend_rows<SLICED, COUNT, 4, kWB>(sm, lane, ranges, values, sp, vp, g, local, 8 * (int)s,
                                                         sbase, n_entries, bg_r, bg_g, bg_b, sl, cnt)
                      : blend_rows<SLICED, COUNT, 2, kWB>(sm, lane, ranges, values, sp, vp, g, local, 4 * (int)s,
                                                         sbase, n_entries, bg_r, bg_g, bg_b, sl, cnt);
            if (all && lane == 0) {
                // the strip's rows have stopped; the tile is done once all 16 rows have
                const uint32_t rows = (eight ? 0xFFu << (8 * s) : 0xFu << (4 * s)) << kRowShift;
                const uint32_t old = atomicOr(&sl.strips[g], rows);
                if (((old | rows) & kRowsAll) == kRowsAll) atomicOr(&sl.done[g >> 5], 1u << (g & 31));
            }
        }
    }
    if (COUNT && counters) {
        unsigned long long n_eval = cnt.eval, n_blend = cnt.blend;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            n_eval += __shfl_xor_sync(kFull, n_eval, d);
            n_blend += __shfl_xor_sync(kFull, n_blend, d);
        }
        if (lane == 0) {
            if (n_eval) atomicAdd(&counters[0], n_eval);
            if (cnt.fetched) atomicAdd(&counters[1], cnt.fetched);
            if (n_blend) atomicAdd(&counters[2], n_blend);
        }
    }
}

}  // namespace

Status launch_blend(const uint2* ranges, const uint32_t* values, const SplatArrays& sp, const ViewParams* views,
                    int V, uint32_t total_tiles, uint32_t n_entries, const float* bg, unsigned long long* counters,
                    cudaStream_t st) {
    if (total_tiles == 0) return {};
    const unsigned grid = (total_tiles + kWarps - 1) / kWarps;
    if (counters)
        k_blend<false, true, 32><<<grid, kThreads, 0, st>>>(ranges, values, sp, views, V, total_tiles, n_entries, bg[0],
                                                        bg[1], bg[2], counters, SliceBlendArgs{});
    else
        k_blend<false, false, 32><<<grid, kThreads, 0, st>>>(ranges, values, sp, views, V, total_tiles, n_entries, bg[0],
                                                         bg[1], bg[2], nullptr, SliceBlendArgs{});
    TIGAS_LAUNCHED();
    return {};
}

Status launch_blend_slice(const uint2* ranges, const uint32_t* values, const SplatArrays& sp,
                          const ViewParams* views, int V, uint32_t n_entries, const float* bg,
                          unsigned long long* counters, const SliceBlendArgs& sl, int ctas_per_sm, int batch,
                          cudaStream_t st) {
    if (batch != 16 && batch != 32) return {TIGAS_ERR_INVALID, "blend batch must be 16 or 32"};
    struct Fit {
        int per_sm = 1, sms = 0;   // CTAs per SM that fit, SM count
        cudaError_t err = cudaSuccess;
    };
    // thread-safe one-time queries, per batch size (the kernels' resources differ)
    auto fit = [](auto kernel) {
        Fit r;
        int per_sm = 0, dev = 0;
        r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
        if (r.err == cudaSuccess) r.err = cudaGetDevice(&dev);
        if (r.err == cudaSuccess) r.err = cudaDeviceGetAttribute(&r.sms, cudaDevAttrMultiProcessorCount, dev);
        r.per_sm = per_sm > 0 ? per_sm : 1;
        return r;
    };
    static const Fit f32 = fit(k_blend<true, false, 32>);
    static const Fit f16 = fit(k_blend<true, false, 16>);
    const Fit& f = batch == 16 ? f16 : f32;
    TIGAS_CUDA_TRY(f.err);
    const int grid = (ctas_per_sm > 0 && ctas_per_sm < f.per_sm ? ctas_per_sm : f.per_sm) * f.sms;
#define TIGAS_BLEND_SLICE(WB)                                                                                        \
    do {                                                                                                             \
        if (counters)                                                                                                \
            k_blend<true, true, WB><<<grid, kThreads, 0, st>>>(ranges, values, sp, views, V, 0, n_entries, bg[0],    \
                                                               bg[1], bg[2], counters, sl);                          \
        else                                                                                                         \
            k_blend<true, false, WB><<<grid, kThreads, 0, st>>>(ranges, values, sp, views, V, 0, n_entries, bg[0],   \
                                                                bg[1], bg[2], nullptr, sl);                          \
    } while (0)
    if (batch == 16)
        TIGAS_BLEND_SLICE(16);
    else
        TIGAS_BLEND_SLICE(32);
#undef TIGAS_BLEND_SLICE
    TIGAS_LAUNCHED();
    return {};
}

}  // namespace tigas
