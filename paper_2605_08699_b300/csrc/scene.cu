// a0 / K7: scene residency.  Raw PLY-style attributes are activated once at
// load (Sec. 5.1, "PLY Model and Primitives": scale = exp(s), opacity =
// sigmoid(logit), unit quaternion) and packed into the resident AoSoA32
// layout, in FP32 or in FP16 (positions stay FP32).
#include "pipeline.cuh"

namespace tigas {

namespace {

__device__ inline uint32_t pack_half2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

template <int STORAGE>
__global__ void __launch_bounds__(256)
k_scene_pack(const float* __restrict__ means, const float* __restrict__ log_scales,
             const float* __restrict__ quats, const float* __restrict__ logits,
             const float* __restrict__ sh, uint32_t n, int sh_degree, uint4* __restrict__ chunks) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    constexpr int C = STORAGE == TIGAS_STORAGE_FP32 ? kChunksF32 : kChunksF16;
    float x = means[3 * i], y = means[3 * i + 1], z = means[3 * i + 2];
    float o = 1.0f / (1.0f + expf(-logits[i]));
    float s0 = expf(log_scales[3 * i]), s1 = expf(log_scales[3 * i + 1]), s2 = expf(log_scales[3 * i + 2]);
    float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
    float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw /= qn; qx /= qn; qy /= qn; qz /= qn;
    const int n_coef = (sh_degree + 1) * (sh_degree + 1);
    float c[48];
#pragma unroll
    for (int k = 0; k < 48; ++k) c[k] = (k / 3) < n_coef ? sh[48 * (size_t)i + k] : 0.0f;

    if (STORAGE == TIGAS_STORAGE_FP32) {
        chunks[chunk_index(i, 0, C)] = make_uint4(__float_as_uint(x), __float_as_uint(y), __float_as_uint(z),
                                                  __float_as_uint(o));
        chunks[chunk_index(i, 1, C)] = make_uint4(__float_as_uint(qw), __float_as_uint(qx), __float_as_uint(qy),
                                                  __float_as_uint(qz));
        chunks[chunk_index(i, 2, C)] = make_uint4(__float_as_uint(s0), __float_as_uint(s1), __float_as_uint(s2), 0u);
#pragma unroll
        for (int k = 0; k < 12; ++k)
            chunks[chunk_index(i, 3 + k, C)] =
                make_uint4(__float_as_uint(c[4 * k]), __float_as_uint(c[4 * k + 1]), __float_as_uint(c[4 * k + 2]),
                           __float_as_uint(c[4 * k + 3]));
    } else {
        chunks[chunk_index(i, 0, C)] = make_uint4(__float_as_uint(x), __float_as_uint(y), __float_as_uint(z),
                                                  pack_half2(o, s0));
        chunks[chunk_index(i, 1, C)] = make_uint4(pack_half2(s1, s2), pack_half2(qw, qx), pack_half2(qy, qz), 0u);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            chunks[chunk_index(i, 2 + k, C)] =
                make_uint4(pack_half2(c[8 * k], c[8 * k + 1]), pack_half2(c[8 * k + 2], c[8 * k + 3]),
                           pack_half2(c[8 * k + 4], c[8 * k + 5]), pack_half2(c[8 * k + 6], c[8 * k + 7]));
    }
}

}  // namespace

Status launch_scene_pack(const float* means, const float* log_scales, const float* quats,
                         const float* opacity_logits, const float* sh, uint32_t n, int sh_degree,
                         int storage, uint4* chunks, cudaStream_t st) {
    if (n == 0) return {};
    dim3 grid(ceil_div_u32(n, 256));
    if (storage == TIGAS_STORAGE_FP32)
        k_scene_pack<TIGAS_STORAGE_FP32><<<grid, 256, 0, st>>>(means, log_scales, quats, opacity_logits, sh, n,
                                                               sh_degree, chunks);
    else
        k_scene_pack<TIGAS_STORAGE_FP16><<<grid, 256, 0, st>>>(means, log_scales, quats, opacity_logits, sh, n,
                                                               sh_degree, chunks);
    TIGAS_LAUNCHED();
    return {};
}

size_t scene_bytes_for(uint64_t n, int storage) {
    const int C = storage == TIGAS_STORAGE_FP32 ? kChunksF32 : kChunksF16;
    return (size_t)((n + 31) / 32) * 32 * C * 16;
}

Status scene_create(const float* means, const float* log_scales, const float* quats, const float* logits,
                    const float* sh, uint32_t n, int sh_degree, int storage, const float bg[3], cudaStream_t st,
                    Scene** out) {
    *out = nullptr;
    static std::atomic<uint64_t> next_id{1};
    auto* s = new Scene();
    s->id = next_id.fetch_add(1, std::memory_order_relaxed);
    s->view.n = n;
    s->view.sh_degree = sh_degree;
    s->view.storage = storage;
    for (int c = 0; c < 3; ++c) s->view.bg[c] = bg[c];
    s->bytes = scene_bytes_for(n, storage);
    cudaError_t e = device_alloc(&s->chunks, s->bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return {TIGAS_ERR_OOM, "scene allocation failed"};
    }
    s->view.chunks = s->chunks;
    Status r = launch_scene_pack(means, log_scales, quats, logits, sh, n, sh_degree, storage, s->chunks, st);
    if (r.ok()) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = {TIGAS_ERR_CUDA, cudaGetErrorString(e)};
    }
    if (!r.ok()) {
        cudaFree(s->chunks);
        delete s;
        return r;
    }
    *out = s;
    return {};
}

}  // namespace tigas
