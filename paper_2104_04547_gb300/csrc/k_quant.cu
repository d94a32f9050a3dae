// Per-pose FP8 (E4M3) quantization of NDHWC bf16 activations for the FP8
// convolution path.  Each pose gets its own scale s = max|x| / 448 (the
// largest finite E4M3 value), so a pose's result does not depend on the other
// poses of its batch.  amax_per_pose_kernel reduces max|x| per pose;
// quantize_per_pose_kernel writes code = E4M3(x / s) (round to nearest even,
// saturating) and the scale s used later to dequantize (x ~ code * s).
#include "fusion_internal.cuh"

#include <cuda_fp8.h>

namespace fusion {

namespace {

constexpr float kE4M3Max = 448.f;

__global__ void amax_per_pose_kernel(const __nv_bfloat16 *x, size_t per_pose, float *amax) {
    const int b = blockIdx.y;
    const uint4 *src = reinterpret_cast<const uint4 *>(x + (size_t)b * per_pose);
    const size_t n8 = per_pose / 8;
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 t = src[i];
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&t);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(h[e]);
            m = fmaxf(m, fmaxf(fabsf(f.x), fabsf(f.y)));
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(reinterpret_cast<unsigned *>(amax + b), __float_as_uint(m));
}

__global__ void quantize_per_pose_kernel(const __nv_bfloat16 *x, uint8_t *q, size_t per_pose, const float *amax,
                                         float *scale) {
    const int b = blockIdx.y;
    const float am = amax[b];
    const float s = am > 0.f ? am / kE4M3Max : 1.f;
    const float inv = 1.f / s;
    if (blockIdx.x == 0 && threadIdx.x == 0) scale[b] = s;
    const uint4 *src = reinterpret_cast<const uint4 *>(x + (size_t)b * per_pose);
    uint2 *dst = reinterpret_cast<uint2 *>(q + (size_t)b * per_pose);
    const size_t n8 = per_pose / 8;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 t = src[i];
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&t);
        uint2 out;
        uint16_t *o16 = reinterpret_cast<uint16_t *>(&out);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(h[e]);
            o16[e] = __nv_cvt_float2_to_fp8x2(make_float2(f.x * inv, f.y * inv), __NV_SATFINITE, __NV_E4M3);
        }
        dst[i] = out;
    }
}

}  // namespace

void launch_amax_per_pose(const void *x_bf16, int B, size_t per_pose, float *amax, cudaStream_t s) {
    const unsigned gx = (unsigned)((per_pose / 8 + 255) / 256 < 64 ? (per_pose / 8 + 255) / 256 : 64);
    amax_per_pose_kernel<<<dim3(gx > 0 ? gx : 1, B), 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(x_bf16), per_pose,
                                                                  amax);
}

void launch_quantize_per_pose(const void *x_bf16, void *q_fp8, int B, size_t per_pose, const float *amax, float *scale,
                              cudaStream_t s) {
    const unsigned gx = (unsigned)((per_pose / 8 + 255) / 256 < 128 ? (per_pose / 8 + 255) / 256 : 128);
    quantize_per_pose_kernel<<<dim3(gx > 0 ? gx : 1, B), 256, 0, s>>>(
        static_cast<const __nv_bfloat16 *>(x_bf16), static_cast<uint8_t *>(q_fp8), per_pose, amax, scale);
}

}  // namespace fusion
