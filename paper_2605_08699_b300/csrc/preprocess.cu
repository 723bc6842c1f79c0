// K1 preprocess: per Gaussian and view, camera transform and pinhole
// projection (Sec. 5.1, T_{w->c} and lambda [u v 1]^T = K p_c), culling, EWA
// projection of the 3D covariance to a 2D conic with low-pass dilation,
// 3-sigma radius, 16x16 tile rectangle, and SH colour (the 3DGS rasterizer
// the backend relies on, Sec. 4.1 "Rendering Engine", Kerbl et al. 2023).
//
// One thread per Gaussian loops over all views of the launch set, so a batch
// of V views reads the scene once instead of V times.  Compiled without
// fast-math: the integer decisions (near cull, opacity cull, ceil of the
// radius, rect floors) use IEEE FP32 arithmetic, except where a hardware
// approximation's error lies far inside the guard bands around those
// decisions (the radius's square roots, x / z as x times 1 / z); the values
// no decision depends on (the conic, the colour's view direction, the
// alpha-cut rectangle, which is widened) take hardware approximations.
#include "kernels.cuh"

namespace tigas {

namespace {

#ifndef TIGAS_CONIC_APPROX
#define TIGAS_CONIC_APPROX 1
#endif
#ifndef TIGAS_RADIUS_APPROX
#define TIGAS_RADIUS_APPROX 1
#endif
#ifndef TIGAS_PROJ_RCP
#define TIGAS_PROJ_RCP 1
#endif
#ifndef TIGAS_TIGHT_APPROX
#define TIGAS_TIGHT_APPROX 1
#endif
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

#ifndef TIGAS_SH_RSQRT
#define TIGAS_SH_RSQRT 1
#endif

constexpr float kNear = 0.2f;
constexpr float kMinOpacity = 1.0f / 255.0f;
constexpr float kDilation = 0.3f;
constexpr float kLog2e = 1.4426950408889634f;

// Real SH basis constants (Condon-Shortley phase), from the closed forms:
constexpr float kY00 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;    // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;    // sqrt(15/pi)/2
constexpr float kY2b = 0.31539156525252005f;   // sqrt(5/pi)/4
constexpr float kY2c = 0.54627421529603959f;   // sqrt(15/pi)/4
constexpr float kY3a = 0.59004358992664352f;   // sqrt(35/(2 pi))/4
constexpr float kY3b = 2.8906114426405538f;    // sqrt(105/pi)/2
constexpr float kY3c = 0.45704579946446572f;   // sqrt(21/(2 pi))/4
constexpr float kY3d = 0.3731763325901154f;    // sqrt(7/pi)/4
constexpr float kY3e = 1.4453057213202769f;    // sqrt(105/pi)/4

struct Attr {
    float x, y, z, o;
    float qw, qx, qy, qz;
    float s0, s1, s2;
};

__device__ inline float2 unpack_half2(uint32_t u) {
    __half2 h = *reinterpret_cast<__half2*>(&u);
    return __half22float2(h);
}

template <int STORAGE>
__device__ inline void load_geom(const uint4* __restrict__ ch, uint32_t i, Attr& a) {
    if (STORAGE == TIGAS_STORAGE_FP32) {
        uint4 c0 = __ldg(ch + chunk_index(i, 0, kChunksF32));
        a.x = __uint_as_float(c0.x); a.y = __uint_as_float(c0.y); a.z = __uint_as_float(c0.z);
        a.o = __uint_as_float(c0.w);
    } else {
        uint4 c0 = __ldg(ch + chunk_index(i, 0, kChunksF16));
        a.x = __uint_as_float(c0.x); a.y = __uint_as_float(c0.y); a.z = __uint_as_float(c0.z);
        float2 os = unpack_half2(c0.w);
        a.o = os.x; a.s0 = os.y;
    }
}

template <int STORAGE>
__device__ inline void load_shape(const uint4* __restrict__ ch, uint32_t i, Attr& a) {
    if (STORAGE == TIGAS_STORAGE_FP32) {
        uint4 c1 = __ldg(ch + chunk_index(i, 1, kChunksF32));
        uint4 c2 = __ldg(ch + chunk_index(i, 2, kChunksF32));
        a.qw = __uint_as_float(c1.x); a.qx = __uint_as_float(c1.y);
        a.qy = __uint_as_float(c1.z); a.qz = __uint_as_float(c1.w);
        a.s0 = __uint_as_float(c2.x); a.s1 = __uint_as_float(c2.y); a.s2 = __uint_as_float(c2.z);
    } else {
        uint4 c1 = __ldg(ch + chunk_index(i, 1, kChunksF16));
        float2 s12 = unpack_half2(c1.x), qwx = unpack_half2(c1.y), qyz = unpack_half2(c1.z);
        a.s1 = s12.x; a.s2 = s12.y;
        a.qw = qwx.x; a.qx = qwx.y; a.qy = qyz.x; a.qz = qyz.y;
    }
}

// SH coefficients of one Gaussian, [16][3] order.  FP32 storage keeps floats;
// FP16 storage keeps the packed half pairs (24 registers instead of 48) and
// converts each coefficient where it is used.
template <int STORAGE>
struct ShCoefs;
template <>
struct ShCoefs<TIGAS_STORAGE_FP32> {
    float c[48];
    __device__ inline float get(int i) const { return c[i]; }
};
template <>
struct ShCoefs<TIGAS_STORAGE_FP16> {
    uint32_t w[24];
    __device__ inline float get(int i) const {
        const float2 h = unpack_half2(w[i >> 1]);
        return (i & 1) ? h.y : h.x;
    }
};

template <int STORAGE>
__device__ inline void load_sh(const uint4* __restrict__ ch, uint32_t i, int degree, ShCoefs<STORAGE>& sc) {
    const int n_float = 3 * (degree + 1) * (degree + 1);
    if constexpr (STORAGE == TIGAS_STORAGE_FP32) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            if (4 * k < n_float) {
                uint4 v = __ldg(ch + chunk_index(i, 3 + k, kChunksF32));
                sc.c[4 * k] = __uint_as_float(v.x); sc.c[4 * k + 1] = __uint_as_float(v.y);
                sc.c[4 * k + 2] = __uint_as_float(v.z); sc.c[4 * k + 3] = __uint_as_float(v.w);
            } else {
                sc.c[4 * k] = sc.c[4 * k + 1] = sc.c[4 * k + 2] = sc.c[4 * k + 3] = 0.0f;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (8 * k < n_float) {
                uint4 v = __ldg(ch + chunk_index(i, 2 + k, kChunksF16));
                sc.w[4 * k] = v.x; sc.w[4 * k + 1] = v.y; sc.w[4 * k + 2] = v.z; sc.w[4 * k + 3] = v.w;
            } else {
                sc.w[4 * k] = sc.w[4 * k + 1] = sc.w[4 * k + 2] = sc.w[4 * k + 3] = 0u;
            }
        }
    }
}

// Sigma = M M^T with M = R(q) diag(s); upper triangle (xx, xy, xz, yy, yz, zz).
__device__ inline void covariance3d(const Attr& a, float* S) {
    float w = a.qw, x = a.qx, y = a.qy, z = a.qz;
    float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                  2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                  2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        M[3 * r] = R[3 * r] * a.s0;
        M[3 * r + 1] = R[3 * r + 1] * a.s1;
        M[3 * r + 2] = R[3 * r + 2] * a.s2;
    }
    S[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    S[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    S[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    S[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    S[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    S[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
}

// RGB from SH coefficients at unit direction (x, y, z).
template <typename Coefs>
__device__ inline void sh_to_rgb(int degree, const Coefs& c, float x, float y, float z, float* rgb) {
    float b[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) b[k] = 0.0f;
    b[0] = kY00;
    if (degree >= 1) {
        b[1] = -kY1 * y; b[2] = kY1 * z; b[3] = -kY1 * x;
    }
    if (degree >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        b[4] = kY2a * x * y;
        b[5] = -kY2a * y * z;
        b[6] = kY2b * (2.f * zz - xx - yy);
        b[7] = -kY2a * x * z;
        b[8] = kY2c * (xx - yy);
        if (degree >= 3) {
            b[9] = -kY3a * y * (3.f * xx - yy);
            b[10] = kY3b * x * y * z;
            b[11] = -kY3c * y * (4.f * zz - xx - yy);
            b[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            b[13] = -kY3c * x * (4.f * zz - xx - yy);
            b[14] = kY3e * z * (xx - yy);
            b[15] = -kY3a * x * (xx - 3.f * yy);
        }
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fmaf(b[k], c.get(3 * k + ch), acc);
        rgb[ch] = fmaxf(acc + 0.5f, 0.0f);
    }
}

// floor(x / 16) clamped to [-1, hi] (exact: division by a power of two)
__device__ inline int floor_div16_clamped(float x, int hi) {
    float f = floorf(x * (1.0f / kTile));
    f = fminf(fmaxf(f, -1.0f), (float)hi);
    return (int)f;
}

template <int STORAGE>
#ifndef TIGAS_PRE_MIN_BLOCKS
#define TIGAS_PRE_MIN_BLOCKS 3
#endif
__global__ void __launch_bounds__(256, TIGAS_PRE_MIN_BLOCKS)
k_preprocess(SceneView scene, const ViewParams* __restrict__ views_g, int V, SplatArrays out,
             uint32_t* __restrict__ n_visible) {
    __shared__ ViewParams views[kMaxViews];
    __shared__ uint32_t vis_count[kMaxViews];
    for (int k = threadIdx.x; k < V; k += blockDim.x) {
        views[k] = views_g[k];
        vis_count[k] = 0;
    }
    __syncthreads();
    const uint32_t n = scene.n;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t vis_mask = 0;
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;   // depth keys this thread kept
    Attr a;
    if (i < n) {
        float S[6];
        load_geom<STORAGE>(scene.chunks, i, a);
        bool have_shape = false;
        for (int v = 0; v < V; ++v) {
            const ViewParams& vp = views[v];
            const size_t e = (size_t)v * n + i;
            // camera transform p_c = R^T (mu - t)
            float dx = a.x - vp.campos[0], dy = a.y - vp.campos[1], dz = a.z - vp.campos[2];
            float px = fmaf(vp.Rt[0], dx, fmaf(vp.Rt[1], dy, vp.Rt[2] * dz));
            float py = fmaf(vp.Rt[3], dx, fmaf(vp.Rt[4], dy, vp.Rt[5] * dz));
            float pz = fmaf(vp.Rt[6], dx, fmaf(vp.Rt[7], dy, vp.Rt[8] * dz));
            uint32_t tiles = 0;
            if (pz > kNear && a.o >= kMinOpacity) {
                if (!have_shape) {
                    load_shape<STORAGE>(scene.chunks, i, a);
                    covariance3d(a, S);
                    have_shape = true;
                }
                // projection
#if TIGAS_PROJ_RCP
                // x / z and y / z as products with 1 / z: within an ulp of the quotients,
                // far inside the oracle's 2^-18 guard band on the pixel decisions
                const float iz0 = 1.0f / pz;
                float xz = px * iz0, yz = py * iz0;
#else
                float xz = px / pz, yz = py / pz;
#endif
                float u = fmaf(vp.fx, xz, vp.cx);
                float vv = fmaf(vp.fy, yz, vp.cy);
                // EWA Jacobian at the guard-band-clamped point
                float tx = fminf(vp.limx, fmaxf(-vp.limx, xz)) * pz;
                float ty = fminf(vp.limy, fmaxf(-vp.limy, yz)) * pz;
#if TIGAS_PROJ_RCP
                const float iz = iz0;
#else
                float iz = 1.0f / pz;
#endif
                float j00 = vp.fx * iz, j02 = -vp.fx * tx * iz * iz;
                float j11 = vp.fy * iz, j12 = -vp.fy * ty * iz * iz;
                // T = J W, W = R^T (rows Rt[0..2], Rt[3..5], Rt[6..8])
                float t0x = fmaf(j00, vp.Rt[0], j02 * vp.Rt[6]);
                float t0y = fmaf(j00, vp.Rt[1], j02 * vp.Rt[7]);
                float t0z = fmaf(j00, vp.Rt[2], j02 * vp.Rt[8]);
                float t1x = fmaf(j11, vp.Rt[3], j12 * vp.Rt[6]);
                float t1y = fmaf(j11, vp.Rt[4], j12 * vp.Rt[7]);
                float t1z = fmaf(j11, vp.Rt[5], j12 * vp.Rt[8]);
                // Sigma T0, Sigma T1
                float s0x = fmaf(S[0], t0x, fmaf(S[1], t0y, S[2] * t0z));
                float s0y = fmaf(S[1], t0x, fmaf(S[3], t0y, S[4] * t0z));
                float s0z = fmaf(S[2], t0x, fmaf(S[4], t0y, S[5] * t0z));
                float s1x = fmaf(S[0], t1x, fmaf(S[1], t1y, S[2] * t1z));
                float s1y = fmaf(S[1], t1x, fmaf(S[3], t1y, S[4] * t1z));
                float s1z = fmaf(S[2], t1x, fmaf(S[4], t1y, S[5] * t1z));
                float ca = fmaf(t0x, s0x, fmaf(t0y, s0y, t0z * s0z)) + kDilation;
                float cb = fmaf(t0x, s1x, fmaf(t0y, s1y, t0z * s1z));
                float cc = fmaf(t1x, s1x, fmaf(t1y, s1y, t1z * s1z)) + kDilation;
                float det = fmaf(ca, cc, -cb * cb);
                if (det > 0.0f) {
#if TIGAS_CONIC_APPROX
                    // the conic feeds only the blend's exponent (no integer decision here):
                    // the hardware reciprocal, within an ulp or two of 1 / det
                    float idet;
                    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(idet) : "f"(det));
#else
                    float idet = 1.0f / det;
#endif
                    float conA = cc * idet, conB = -cb * idet, conC = ca * idet;
                    float mid = 0.5f * (ca + cc);
                    float hd = 0.5f * (ca - cc);
                    float disc = fmaf(hd, hd, cb * cb);          // mid^2 - det, cancellation-free
#if TIGAS_RADIUS_APPROX
                    // hardware square roots: their error (about 2^-22 relative) lies far
                    // inside the oracle's 2^-16 guard band on the radius decision
                    float lam = mid + sqrt_approx(fmaxf(0.1f, disc));
                    float q = 3.0f * sqrt_approx(lam);
#else
                    float lam = mid + sqrtf(fmaxf(0.1f, disc));
                    float q = 3.0f * sqrtf(lam);
#endif
                    float r = ceilf(q);
                    // tiles overlapped by [u - r, u + r] x [v - r, v + r]
                    int xlo = max(0, floor_div16_clamped(u - r, vp.TX));
                    int xhi = min(vp.TX, floor_div16_clamped(u + r, vp.TX) + 1);
                    int ylo = max(0, floor_div16_clamped(vv - r, vp.TY));
                    int yhi = min(vp.TY, floor_div16_clamped(vv + r, vp.TY) + 1);
                    if (xhi > xlo && yhi > ylo) tiles = (uint32_t)((xhi - xlo) * (yhi - ylo));
                    if (out.q_dbg) out.q_dbg[e] = q;
                    if (tiles > 0 && out.tight_rect) {
                        // only the tiles the alpha >= 1/255 ellipse d^T S^-1 d <= 2 ln(255 o) can
                        // reach: its box has half-extents sqrt(tau S_xx), sqrt(tau S_yy), taken
                        // 2 % + 1 px wider so that FP32 rounding in the blend cannot fall outside
#if TIGAS_TIGHT_APPROX
                        // the widening (2 % + 1 px) covers the hardware logarithm's and square
                        // root's error many times over, so approximate ones keep the cut exact
                        const float tau = 2.0f * __logf(255.0f * a.o);
                        const float hx = fmaf(sqrt_approx(fmaxf(tau, 0.0f) * ca), 1.02f, 1.0f);
                        const float hy = fmaf(sqrt_approx(fmaxf(tau, 0.0f) * cc), 1.02f, 1.0f);
#else
                        const float tau = 2.0f * logf(255.0f * a.o);
                        const float hx = fmaf(sqrtf(fmaxf(tau, 0.0f) * ca), 1.02f, 1.0f);
                        const float hy = fmaf(sqrtf(fmaxf(tau, 0.0f) * cc), 1.02f, 1.0f);
#endif
                        xlo = max(xlo, floor_div16_clamped(u - hx, vp.TX));
                        xhi = min(xhi, floor_div16_clamped(u + hx, vp.TX) + 1);
                        ylo = max(ylo, floor_div16_clamped(vv - hy, vp.TY));
                        yhi = min(yhi, floor_div16_clamped(vv + hy, vp.TY) + 1);
                        if (xhi <= xlo || yhi <= ylo) xlo = xhi = ylo = yhi = 0;   // reaches no pixel
                    }
                    if (tiles > 0) {
                        out.geom[e] = make_float4(u, vv, -0.5f * kLog2e * conA, -kLog2e * conB);
                        reinterpret_cast<float2*>(out.appear)[2 * e] =
                            make_float2(-0.5f * kLog2e * conC, log2f(a.o));
                        out.rect[e] = out.compact_rect
                                          ? make_uint2(pack_rect_compact((uint32_t)xlo, (uint32_t)xhi, (uint32_t)ylo,
                                                                         (uint32_t)yhi, (uint32_t)v),
                                                       (uint32_t)e)
                                          : make_uint2((uint32_t)xlo | ((uint32_t)xhi << 10) | ((uint32_t)v << 20),
                                                       (uint32_t)ylo | ((uint32_t)yhi << 10));
                        const uint32_t key = __float_as_uint(pz);
                        out.depth_key[e] = key;
                        kmin = min(kmin, key);
                        kmax = max(kmax, key);
                        vis_mask |= 1ull << v;
                    }
                }
            }
            if (!out.tight_rect) out.tiles[e] = tiles;   // the sliced render path reads rectangles only
            if (tiles == 0) {
                out.depth_key[e] = 0xFFFFFFFFu;
                out.rect[e] = make_uint2(0u, out.compact_rect ? (uint32_t)e : 0u);   // empty rectangle
            }
        }
    }
    // colour for the views that kept this Gaussian
    if (vis_mask) {
        ShCoefs<STORAGE> c;
        load_sh<STORAGE>(scene.chunks, i, scene.sh_degree, c);
        uint64_t m = vis_mask;
        while (m) {
            int v = __ffsll((long long)m) - 1;
            m &= m - 1;
            const ViewParams& vp = views[v];
            const size_t e = (size_t)v * n + i;
            float dx = a.x - vp.campos[0], dy = a.y - vp.campos[1], dz = a.z - vp.campos[2];
#if TIGAS_SH_RSQRT
            // the direction feeds the colour only (no integer decision): the hardware
            // reciprocal square root instead of an IEEE square root and division
            float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
#else
            float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
#endif
            float rgb[3];
            sh_to_rgb(scene.sh_degree, c, dx * inv, dy * inv, dz * inv, rgb);
            reinterpret_cast<float2*>(out.appear)[2 * e + 1] = make_float2(rgb[0], rgb[1]);
            out.blue[e] = rgb[2];
            atomicAdd(&vis_count[v], 1u);
        }
    }
    if (out.key_range) {
        kmin = __reduce_min_sync(0xFFFFFFFFu, kmin);
        kmax = __reduce_max_sync(0xFFFFFFFFu, kmax);
        if ((threadIdx.x & 31) == 0 && kmin <= kmax) {
            atomicMin(&out.key_range[0], kmin);
            atomicMax(&out.key_range[1], kmax);
        }
    }
    __syncthreads();
    if (n_visible)
        for (int k = threadIdx.x; k < V; k += blockDim.x)
            if (vis_count[k]) atomicAdd(&n_visible[k], vis_count[k]);
}

}  // namespace

Status launch_preprocess(const SceneView& scene, const ViewParams* views, int V, const SplatArrays& out,
                         uint32_t* n_visible, cudaStream_t st, bool counters_set) {
    if (V < 1 || V > kMaxViews) return {TIGAS_ERR_INVALID, "view count out of range"};
    if (n_visible && !counters_set) TIGAS_CUDA_TRY(cudaMemsetAsync(n_visible, 0, sizeof(uint32_t) * V, st));
    if (out.key_range && !counters_set) {   // [min, max] of the kept depth keys: start from [0xFFFFFFFF, 0]
        TIGAS_CUDA_TRY(cudaMemsetAsync(out.key_range, 0xFF, sizeof(uint32_t), st));
        TIGAS_CUDA_TRY(cudaMemsetAsync(out.key_range + 1, 0, sizeof(uint32_t), st));
    }
    if (scene.n == 0) return {};
    dim3 grid(ceil_div_u32(scene.n, 256));
    if (scene.storage == TIGAS_STORAGE_FP32)
        k_preprocess<TIGAS_STORAGE_FP32><<<grid, 256, 0, st>>>(scene, views, V, out, n_visible);
    else
        k_preprocess<TIGAS_STORAGE_FP16><<<grid, 256, 0, st>>>(scene, views, V, out, n_visible);
    TIGAS_LAUNCHED();
    return {};
}

}  // namespace tigas
