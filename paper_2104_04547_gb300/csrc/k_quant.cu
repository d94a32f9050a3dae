// Per-pose FP8 (E4M3) quantization of NDHWC bf16 activations for the FP8
// convolution path (stored NDHWC, or channel-blocked for the stride-1 layers,
// whose halos are then loaded in rows of hw x 16 contiguous bytes).  Each pose gets its own scale s = max|x| / 448 (the
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

// The quantizers take the poses last to first: the producer wrote them first to last, so the last ones are
// still in L2, and the quantized first poses, which the next convolution reads first, stay there for it.
__global__ void quantize_per_pose_kernel(const __nv_bfloat16 *x, uint8_t *q, size_t per_pose, const float *amax,
                                         float *scale) {
    const int b = gridDim.y - 1 - blockIdx.y;
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

// Channel-blocked output: item (voxel v, 16-channel block cb) reads 16 bf16 (32 bytes) and writes 16 codes
// to [b][z][y][cb][x][16]; cb varies fastest across threads, so the reads are contiguous and each
// block's writes form runs of consecutive x.  split != 0 (n even, h = n / 2): the same blocks of each of the
// 8 parity sub-grids, [b][(z&1) 4 + (y&1) 2 + (x&1)][z/2][y/2][cb][x/2][16], read by a stride-2 layer.
__global__ void quantize_blocked_kernel(const __nv_bfloat16 *x, uint8_t *q, int n, int C, const float *amax,
                                        float *scale, int split) {
    const int b = gridDim.y - 1 - blockIdx.y;       // last pose first, as in quantize_per_pose_kernel
    const float am = amax[b];
    const float s = am > 0.f ? am / kE4M3Max : 1.f;
    const float inv = 1.f / s;
    if (blockIdx.x == 0 && threadIdx.x == 0) scale[b] = s;
    const int ncb = C / 16;
    const size_t nv = (size_t)n * n * n;
    const size_t items = nv * ncb;
    const __nv_bfloat16 *xb = x + (size_t)b * nv * C;
    uint8_t *qb = q + (size_t)b * nv * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < items; i += (size_t)gridDim.x * blockDim.x) {
        const size_t v = i / ncb;
        const int cb = (int)(i - v * ncb);
        const size_t row = v / n;                 // (z, y)
        const int xx = (int)(v - row * n);
        const uint4 *src = reinterpret_cast<const uint4 *>(xb + v * C + cb * 16);
        uint4 out;
        uint16_t *o16 = reinterpret_cast<uint16_t *>(&out);
#pragma unroll
        for (int hlf = 0; hlf < 2; ++hlf) {
            const uint4 t = src[hlf];
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&t);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(h[e]);
                o16[hlf * 4 + e] = __nv_cvt_float2_to_fp8x2(make_float2(f.x * inv, f.y * inv), __NV_SATFINITE, __NV_E4M3);
            }
        }
        size_t dst;
        if (split) {
            const size_t h = (size_t)(n >> 1);
            const int yy = (int)(row % n), zz = (int)(row / n);
            const size_t p = (size_t)(zz & 1) * 4 + (yy & 1) * 2 + (xx & 1);
            dst = ((((p * h + (zz >> 1)) * h + (yy >> 1)) * ncb + cb) * h + (xx >> 1)) * 16;
        } else {
            dst = ((row * ncb + cb) * n + xx) * 16;
        }
        *reinterpret_cast<uint4 *>(qb + dst) = out;
    }
}

// One CTA per 4 grid rows (b, z, y): the rows' channels 0..18 are loaded with 16-byte reads and
// quantized into shared memory (codes are the same E4M3(x / s) as quantize_per_pose_kernel gives),
// then each stored voxel j = 0 .. n of a row is assembled from them, as described at
// launch_quantize_fold_fp8, and written with 16-byte stores.
constexpr int kFoldRows = 4;

__global__ void __launch_bounds__(256) quantize_fold_fp8_kernel(const __nv_bfloat16 *g, uint8_t *q, int B, int n,
                                                                 int p, const float *amax, float *scale, int blocked) {
    extern __shared__ __align__(16) uint8_t s_code[];     // [kFoldRows][n][20] (19 channels + pad)
    const int rows = B * n * n;
    const int r0 = (gridDim.x - 1 - blockIdx.x) * kFoldRows;   // last rows first, as in quantize_per_pose_kernel
    const int nr = min(kFoldRows, rows - r0);
    const int nn = n * n;
    for (int e = threadIdx.x; e < nr * n * 3; e += blockDim.x) {
        // 8 channels (one 16-byte load) of voxel v of row r; chunks 0, 1 = channels 0..15, 2 = 16..23
        const int r = e / (n * 3), rem = e - r * n * 3, v = rem / 3, part = rem - v * 3;
        const int row = r0 + r, b = row / nn;
        const float am = amax[b];
        const float inv = 1.f / (am > 0.f ? am / kE4M3Max : 1.f);
        const uint4 t = reinterpret_cast<const uint4 *>(g + ((size_t)row * n + v) * 32)[part];
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&t);
        uint8_t *dst = s_code + ((size_t)r * n + v) * 20 + part * 8;
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            const float2 f = __bfloat1622float2(h[k2]);
            const uint16_t c2 = __nv_cvt_float2_to_fp8x2(make_float2(f.x * inv, f.y * inv), __NV_SATFINITE, __NV_E4M3);
            if (part < 2 || 2 * k2 < 3) dst[2 * k2] = (uint8_t)(c2 & 0xFF);
            if (part < 2 || 2 * k2 + 1 < 3) dst[2 * k2 + 1] = (uint8_t)(c2 >> 8);
        }
    }
    if (threadIdx.x < nr && (r0 + threadIdx.x) % nn == 0) {
        const int b = (r0 + threadIdx.x) / nn;
        scale[b] = amax[b] > 0.f ? amax[b] / kE4M3Max : 1.f;
    }
    __syncthreads();
    const int nx = n + 1;
    for (int e = threadIdx.x; e < nr * nx; e += blockDim.x) {
        const int r = e / nx, j = e - r * nx;
        const uint8_t *cr = s_code + (size_t)r * n * 20;
        __align__(16) uint8_t out[64];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int x = j - 1 + h;
            const bool in = x >= 0 && x < n;
#pragma unroll
            for (int c = 0; c < 16; ++c) out[16 * h + c] = in ? cr[x * 20 + c] : 0;
        }
#pragma unroll
        for (int qq = 32; qq < 64; ++qq) out[qq] = 0;
#pragma unroll
        for (int sl = 0; sl < 7; ++sl) {              // 2p + 1 <= 7 positions (k <= 7); constant slot indices
            const int x = j - 1 - p + sl;
            if (sl > 2 * p || x < 0 || x >= n) continue;
#pragma unroll
            for (int f = 0; f < 3; ++f) out[32 + 3 * sl + f] = cr[x * 20 + 16 + f];
        }
        if (blocked) {
            // [row][16-byte block u][x = j][16]
#pragma unroll
            for (int u = 0; u < 4; ++u)
                *reinterpret_cast<uint4 *>(q + (((size_t)(r0 + r) * 4 + u) * nx + j) * 16) = reinterpret_cast<const uint4 *>(out)[u];
        } else {
            uint4 *dst = reinterpret_cast<uint4 *>(q + ((size_t)(r0 + r) * nx + j) * 64);
#pragma unroll
            for (int u = 0; u < 4; ++u) dst[u] = reinterpret_cast<const uint4 *>(out)[u];
        }
    }
}

}  // namespace

void launch_quantize_fold_fp8(const void *grid_bf16, void *q_fp8, int B, int n, int p, const float *amax,
                              float *scale, int blocked, cudaStream_t s) {
    const int rows = B * n * n;
    const size_t sm = (size_t)kFoldRows * n * 20;
    quantize_fold_fp8_kernel<<<(unsigned)((rows + kFoldRows - 1) / kFoldRows), 256, sm, s>>>(
        static_cast<const __nv_bfloat16 *>(grid_bf16), static_cast<uint8_t *>(q_fp8), B, n, p, amax, scale, blocked);
}

void launch_quantize_blocked(const void *x_bf16, void *q_fp8, int B, int n, int C, const float *amax, float *scale,
                             int split, cudaStream_t s) {
    const size_t items = (size_t)n * n * n * (C / 16);
    const unsigned gx = (unsigned)((items + 255) / 256 < 128 ? (items + 255) / 256 : 128);
    quantize_blocked_kernel<<<dim3(gx > 0 ? gx : 1, B), 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(x_bf16),
                                                                    static_cast<uint8_t *>(q_fp8), n, C, amax, scale,
                                                                    split && n % 2 == 0 ? 1 : 0);
}

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
