// Post-session quality evaluation (Sec. 5.3 "Sampled OPFS Capture and
// Post-Session Materialization", Sec. 6 quality metrics): a resampler that
// brings a transmitted frame to the ground truth's resolution, and one pass
// computing SSIM and the squared error for PSNR between two RGBA8 frames.
//
// SSIM follows Wang et al. (IEEE TIP 2004): per colour channel, an 11 x 11
// Gaussian window (sigma 1.5, normalised), K1 = 0.01, K2 = 0.03, L = 255,
// evaluated at every window position inside the image; the result is the
// mean over positions and the three channels.  Alpha is ignored.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "pipeline.cuh"

namespace tigas {

namespace {

constexpr int kWin = 11;
constexpr int kHalf = 5;
constexpr int kTx = 32;              // output tile width (threads per row)
constexpr int kTy = 8;               // output tile height
constexpr int kInW = kTx + kWin - 1; // 42
constexpr int kInH = kTy + kWin - 1; // 18
constexpr float kC1 = (0.01f * 255.0f) * (0.01f * 255.0f);
constexpr float kC2 = (0.03f * 255.0f) * (0.03f * 255.0f);

__constant__ float c_gauss[kWin];

// Bilinear resample with 16.16 fixed-point source coordinates (pixel centres
// aligned: src = (dst + 0.5) * w / W - 0.5, clamped to the edge) and 8-bit
// weights; integer arithmetic throughout, so the result is exact.
__global__ void __launch_bounds__(256)
k_resample(const uchar4* __restrict__ src, int w, int h, uchar4* __restrict__ dst, int W, int H) {
    const int dx = blockIdx.x * blockDim.x + threadIdx.x;
    const int dy = blockIdx.y;
    if (dx >= W || dy >= H) return;
    auto coord = [](int d, int s, int D, int* i0, int* i1, int* f) {
        long long num = (long long)(2 * d + 1) * s * 65536;
        long long c = num / (2LL * D) - 32768;
        if (c < 0) c = 0;
        int i = (int)(c >> 16);
        int fr = (int)((c >> 8) & 255);
        if (i >= s - 1) {
            i = s - 1;
            fr = 0;
        }
        *i0 = i;
        *i1 = min(i + 1, s - 1);
        *f = fr;
    };
    int x0, x1, fx, y0, y1, fy;
    coord(dx, w, W, &x0, &x1, &fx);
    coord(dy, h, H, &y0, &y1, &fy);
    const uchar4 p00 = src[(size_t)y0 * w + x0], p01 = src[(size_t)y0 * w + x1];
    const uchar4 p10 = src[(size_t)y1 * w + x0], p11 = src[(size_t)y1 * w + x1];
    auto mix = [&](int a, int b, int c, int d) {
        int top = a * (256 - fx) + b * fx;
        int bot = c * (256 - fx) + d * fx;
        return (unsigned char)((top * (256 - fy) + bot * fy + 32768) >> 16);
    };
    dst[(size_t)dy * W + dx] = make_uchar4(mix(p00.x, p01.x, p10.x, p11.x), mix(p00.y, p01.y, p10.y, p11.y),
                                           mix(p00.z, p01.z, p10.z, p11.z), mix(p00.w, p01.w, p10.w, p11.w));
}

// One CTA per 32 x 8 tile of the image.  It computes the SSIM of the window
// positions whose top-left corner lies in the tile (and inside the valid
// region), and the squared error of the tile's own pixels.  Samples are
// centred (x - 128) before the moments are taken, which keeps E[x^2] - mu^2
// within 2^14 in FP32.
__global__ void __launch_bounds__(256)
k_ssim(const uchar4* __restrict__ a, const uchar4* __restrict__ b, int W, int H, double* __restrict__ partial,
       unsigned long long* __restrict__ sse, float* __restrict__ map) {
    __shared__ uint8_t s_in[2][3][kInH][kInW];       // samples of both frames
    __shared__ float s_h[5][3][kInH][kTx];           // horizontal Gaussian sums
    __shared__ double s_red[8];
    __shared__ unsigned long long s_sse[8];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kTx, y0 = blockIdx.y * kTy;
    const int OW = W - (kWin - 1), OH = H - (kWin - 1);

    for (int k = tid; k < kInH * kInW; k += 256) {
        const int r = k / kInW, c = k - r * kInW;
        const int x = x0 + c, y = y0 + r;
        uchar4 pa = make_uchar4(128, 128, 128, 0), pb = pa;   // outside: feeds no valid window
        if (x < W && y < H) {
            pa = a[(size_t)y * W + x];
            pb = b[(size_t)y * W + x];
        }
        s_in[0][0][r][c] = pa.x;
        s_in[0][1][r][c] = pa.y;
        s_in[0][2][r][c] = pa.z;
        s_in[1][0][r][c] = pb.x;
        s_in[1][1][r][c] = pb.y;
        s_in[1][2][r][c] = pb.z;
    }
    __syncthreads();
    for (int k = tid; k < kInH * kTx * 3; k += 256) {
        const int ch = k / (kInH * kTx);
        const int rem = k - ch * (kInH * kTx);
        const int r = rem / kTx, c = rem - r * kTx;
        float mx = 0, my = 0, xx = 0, yy = 0, xy = 0;
#pragma unroll
        for (int t = 0; t < kWin; ++t) {
            const float g = c_gauss[t];
            const float u = (float)s_in[0][ch][r][c + t] - 128.0f, v = (float)s_in[1][ch][r][c + t] - 128.0f;
            mx = fmaf(g, u, mx);
            my = fmaf(g, v, my);
            xx = fmaf(g * u, u, xx);
            yy = fmaf(g * v, v, yy);
            xy = fmaf(g * u, v, xy);
        }
        s_h[0][ch][r][c] = mx;
        s_h[1][ch][r][c] = my;
        s_h[2][ch][r][c] = xx;
        s_h[3][ch][r][c] = yy;
        s_h[4][ch][r][c] = xy;
    }
    __syncthreads();

    const int tx = tid & (kTx - 1), ty = tid >> 5;
    const int ox = x0 + tx, oy = y0 + ty;
    double local = 0.0;
    if (ox < OW && oy < OH) {
        float acc = 0.0f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float mx = 0, my = 0, xx = 0, yy = 0, xy = 0;
#pragma unroll
            for (int t = 0; t < kWin; ++t) {
                const float g = c_gauss[t];
                mx = fmaf(g, s_h[0][ch][ty + t][tx], mx);
                my = fmaf(g, s_h[1][ch][ty + t][tx], my);
                xx = fmaf(g, s_h[2][ch][ty + t][tx], xx);
                yy = fmaf(g, s_h[3][ch][ty + t][tx], yy);
                xy = fmaf(g, s_h[4][ch][ty + t][tx], xy);
            }
            const float vx = xx - mx * mx, vy = yy - my * my, cxy = xy - mx * my;
            // means of the uncentred samples: mu + 128
            const float ux = mx + 128.0f, uy = my + 128.0f;
            const float num = (2.0f * ux * uy + kC1) * (2.0f * cxy + kC2);
            const float den = (ux * ux + uy * uy + kC1) * (vx + vy + kC2);
            acc += num / den;
        }
        if (map) map[(size_t)oy * OW + ox] = acc * (1.0f / 3.0f);
        local = (double)acc;
    }
    unsigned long long e2 = 0;
    if (x0 + tx < W && y0 + ty < H) {
        const int r = ty, c = tx;
        for (int ch = 0; ch < 3; ++ch) {
            const int d = (int)s_in[0][ch][r][c] - (int)s_in[1][ch][r][c];
            e2 += (unsigned long long)(d * d);
        }
    }
    // fixed-order block reduction (deterministic)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        local += __shfl_down_sync(0xffffffffu, local, o);
        e2 += __shfl_down_sync(0xffffffffu, e2, o);
    }
    if ((tid & 31) == 0) {
        s_red[tid >> 5] = local;
        s_sse[tid >> 5] = e2;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        unsigned long long u = 0;
        for (int k = 0; k < 8; ++k) {
            t += s_red[k];
            u += s_sse[k];
        }
        partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
        atomicAdd(sse, u);
    }
}

// Sum of the per-tile partials in a fixed order: out[0] = sum.
__global__ void __launch_bounds__(256) k_sum_partials(const double* __restrict__ partial, int n,
                                                      double* __restrict__ out) {
    __shared__ double s[256];
    double t = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) t += partial[k];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0];
}

std::once_flag g_gauss_once;
cudaError_t g_gauss_err = cudaSuccess;

}  // namespace

Status launch_resample(const uint8_t* src, int w, int h, uint8_t* dst, int W, int H, cudaStream_t st) {
    dim3 grid((W + 255) / 256, H);
    k_resample<<<grid, 256, 0, st>>>((const uchar4*)src, w, h, (uchar4*)dst, W, H);
    TIGAS_LAUNCHED();
    TIGAS_CUDA_TRY(cudaGetLastError());
    return {};
}

size_t quality_tmp_bytes(int W, int H) {
    const size_t tiles = (size_t)((W + kTx - 1) / kTx) * ((H + kTy - 1) / kTy);
    return tiles * sizeof(double) + 2 * sizeof(double);
}

Status launch_quality(const uint8_t* a, const uint8_t* b, int W, int H, void* tmp, float* map, cudaStream_t st) {
    std::call_once(g_gauss_once, [] {
        double g[kWin], s = 0.0;
        for (int t = 0; t < kWin; ++t) {
            const double d = t - kHalf;
            g[t] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
            s += g[t];
        }
        float gf[kWin];
        for (int t = 0; t < kWin; ++t) gf[t] = (float)(g[t] / s);
        g_gauss_err = cudaMemcpyToSymbol(c_gauss, gf, sizeof(gf));
    });
    TIGAS_CUDA_TRY(g_gauss_err);
    dim3 grid((W + kTx - 1) / kTx, (H + kTy - 1) / kTy);
    double* out = (double*)tmp;                    // [0] SSIM sum, [1] squared error (u64)
    double* partial = out + 2;
    TIGAS_CUDA_TRY(cudaMemsetAsync(out, 0, 2 * sizeof(double), st));
    k_ssim<<<grid, 256, 0, st>>>((const uchar4*)a, (const uchar4*)b, W, H, partial,
                                 reinterpret_cast<unsigned long long*>(out + 1), map);
    TIGAS_LAUNCHED();
    k_sum_partials<<<1, 256, 0, st>>>(partial, (int)(grid.x * grid.y), out);
    TIGAS_LAUNCHED();
    TIGAS_CUDA_TRY(cudaGetLastError());
    return {};
}

// Host wrappers: host or device frames, scratch from the context's encoder arena.
Status resample_rgba8(RenderContext& ctx, const uint8_t* src, int w, int h, uint8_t* dst, int W, int H,
                      cudaStream_t st) {
    if (!src || !dst) return {TIGAS_ERR_INVALID, "resample: null argument"};
    if (w < 1 || h < 1 || W < 1 || H < 1 || w > kMaxDim || h > kMaxDim || W > kMaxDim || H > kMaxDim)
        return {TIGAS_ERR_INVALID, "resample: sizes out of 1..8192"};
    const bool dev_in = is_device_pointer(src), dev_out = is_device_pointer(dst);
    const size_t in_bytes = (size_t)w * h * 4, out_bytes = (size_t)W * H * 4;
    TIGAS_TRY(ctx.jpeg.reserve((dev_in ? 0 : in_bytes) + (dev_out ? 0 : out_bytes) + 1024));
    ctx.jpeg.reset();
    const uint8_t* d_src = src;
    uint8_t* d_dst = dst;
    if (!dev_in) {
        uint8_t* t = ctx.jpeg.take<uint8_t>(in_bytes);
        TIGAS_CUDA_TRY(cudaMemcpyAsync(t, src, in_bytes, cudaMemcpyHostToDevice, st));
        d_src = t;
    }
    if (!dev_out) d_dst = ctx.jpeg.take<uint8_t>(out_bytes);
    TIGAS_TRY(launch_resample(d_src, w, h, d_dst, W, H, st));
    if (!dev_out) TIGAS_CUDA_TRY(cudaMemcpyAsync(dst, d_dst, out_bytes, cudaMemcpyDeviceToHost, st));
    TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
    return {};
}

Status image_quality(RenderContext& ctx, const uint8_t* a, const uint8_t* b, int W, int H, float* map,
                     double* ssim, double* psnr, cudaStream_t st) {
    if (!a || !b) return {TIGAS_ERR_INVALID, "quality: null frame"};
    if (W < kWin || H < kWin || W > kMaxDim || H > kMaxDim)
        return {TIGAS_ERR_INVALID, "quality: width/height out of 11..8192"};
    const bool dev_a = is_device_pointer(a), dev_b = is_device_pointer(b), dev_map = map && is_device_pointer(map);
    const size_t px = (size_t)W * H * 4;
    const size_t map_bytes = (size_t)(W - kWin + 1) * (H - kWin + 1) * sizeof(float);
    TIGAS_TRY(ctx.jpeg.reserve(quality_tmp_bytes(W, H) + (dev_a ? 0 : px) + (dev_b ? 0 : px) +
                               (map && !dev_map ? map_bytes : 0) + 4096));
    ctx.jpeg.reset();
    void* tmp = ctx.jpeg.take<double>(quality_tmp_bytes(W, H) / sizeof(double));
    const uint8_t* da = a;
    const uint8_t* db = b;
    if (!dev_a) {
        uint8_t* t = ctx.jpeg.take<uint8_t>(px);
        TIGAS_CUDA_TRY(cudaMemcpyAsync(t, a, px, cudaMemcpyHostToDevice, st));
        da = t;
    }
    if (!dev_b) {
        uint8_t* t = ctx.jpeg.take<uint8_t>(px);
        TIGAS_CUDA_TRY(cudaMemcpyAsync(t, b, px, cudaMemcpyHostToDevice, st));
        db = t;
    }
    float* dmap = map && !dev_map ? ctx.jpeg.take<float>(map_bytes / sizeof(float)) : map;
    TIGAS_TRY(launch_quality(da, db, W, H, tmp, dmap, st));
    double h_out[2];
    TIGAS_CUDA_TRY(cudaMemcpyAsync(h_out, tmp, sizeof(h_out), cudaMemcpyDeviceToHost, st));
    if (map && !dev_map) TIGAS_CUDA_TRY(cudaMemcpyAsync(map, dmap, map_bytes, cudaMemcpyDeviceToHost, st));
    TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
    uint64_t sse;
    memcpy(&sse, &h_out[1], sizeof(sse));
    const double windows = 3.0 * (W - kWin + 1) * (double)(H - kWin + 1);
    if (ssim) *ssim = h_out[0] / windows;
    if (psnr) {
        const double mse = (double)sse / (3.0 * W * (double)H);
        *psnr = sse == 0 ? INFINITY : 10.0 * std::log10(255.0 * 255.0 / mse);
    }
    return {};
}

}  // namespace tigas
