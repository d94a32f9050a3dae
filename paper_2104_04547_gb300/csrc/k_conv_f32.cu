// FP32 3D convolution as an implicit GEMM on the CUDA cores (Section 3.3.1,
// Table III: convolutions with bias and ReLU, residual blocks), plus the 2^3
// max-pool of Fig. 1.
//
// GEMM view: M = output voxels of the batch, N = output channels, K = k^3
// kernel offsets x input channels.  A CTA owns a 128-voxel x BN-channel tile;
// each K step stages 8 input channels of one kernel offset for the 128 voxels
// (gathered from NDHWC with zero fill outside the grid) and the matching 8 x BN
// weights in shared memory, double-buffered through registers.  Each thread
// accumulates a TM x 8 block in registers.  The epilogue adds the bias, applies
// ReLU, adds the residual input when the layer is a residual block, and
// stores with 16-byte vector stores.  Every output is a fixed-order sum, so the
// result of a pose does not depend on the batch it is in.
#include "fusion_internal.cuh"

namespace fusion {

namespace {

constexpr int BM = 128;
constexpr int BK = 8;
constexpr int NT = 128;

template <int BN>
__global__ void __launch_bounds__(NT) conv3d_f32_kernel(ConvArgs a) {
    constexpr int TN = 8;
    constexpr int NTN = BN / TN;        // thread columns
    constexpr int NTM = NT / NTN;       // thread rows
    constexpr int TM = BM / NTM;        // rows per thread (8 for BN=64, 4 for BN=32)
    constexpr int BQ = BN / 4;          // float4 per weight row
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];

    const int tid = threadIdx.x;
    const int n_out = a.n_out, n_in = a.n_in, cx = a.cx_in, co = a.c_out, k = a.k;
    const long long vout = (long long)n_out * n_out * n_out;
    const long long M = (long long)a.B * vout;
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;

    // A-load role: row m0 + tid
    const long long mrow = m0 + tid;
    const bool mvalid = mrow < M;
    int zi0 = 0, yi0 = 0, xi0 = 0;
    const float *xb = a.x;
    if (mvalid) {
        const long long b = mrow / vout;
        const long long r = mrow - b * vout;
        const int zo = (int)(r / (n_out * n_out));
        const int yo = (int)((r / n_out) % n_out);
        const int xo = (int)(r % n_out);
        zi0 = zo * a.stride - a.pad;
        yi0 = yo * a.stride - a.pad;
        xi0 = xo * a.stride - a.pad;
        xb = a.x + (size_t)b * n_in * n_in * n_in * cx;
    }
    // B-load role: weight row kk = tid / BQ, column quad (tid % BQ)
    const int bkk = tid / BQ, bq = tid % BQ;
    const bool bload = tid < BK * BQ;

    const int csteps = cx / BK;
    const int S = k * k * k * csteps;

    const int tn = tid % NTN, tm = tid / NTN;
    float acc[TM][8];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float4 ra0, ra1, rb;
    int kd = 0, kh = 0, kw = 0, c0 = 0, off = 0;

    auto load = [&](int kd_, int kh_, int kw_, int c0_, int off_) {
        const int iz = zi0 + kd_, iy = yi0 + kh_, ix = xi0 + kw_;
        if (mvalid && (unsigned)iz < (unsigned)n_in && (unsigned)iy < (unsigned)n_in && (unsigned)ix < (unsigned)n_in) {
            const float *src = xb + (((size_t)iz * n_in + iy) * n_in + ix) * cx + c0_;
            ra0 = *reinterpret_cast<const float4 *>(src);
            ra1 = *reinterpret_cast<const float4 *>(src + 4);
        } else {
            ra0 = make_float4(0.f, 0.f, 0.f, 0.f);
            ra1 = ra0;
        }
        if (bload) {
            rb = *reinterpret_cast<const float4 *>(a.w + ((size_t)off_ * cx + c0_ + bkk) * co + n0 + bq * 4);
        }
    };
    auto store = [&](int buf) {
        As[buf][0][tid] = ra0.x; As[buf][1][tid] = ra0.y; As[buf][2][tid] = ra0.z; As[buf][3][tid] = ra0.w;
        As[buf][4][tid] = ra1.x; As[buf][5][tid] = ra1.y; As[buf][6][tid] = ra1.z; As[buf][7][tid] = ra1.w;
        if (bload) *reinterpret_cast<float4 *>(&Bs[buf][bkk][bq * 4]) = rb;
    };
    auto advance = [&]() {
        c0 += BK;
        if (c0 == cx) {
            c0 = 0;
            ++off;
            if (++kw == k) {
                kw = 0;
                if (++kh == k) { kh = 0; ++kd; }
            }
        }
    };

    load(kd, kh, kw, c0, off);
    store(0);
    __syncthreads();
    for (int s = 0; s < S; ++s) {
        const int buf = s & 1;
        if (s + 1 < S) {
            advance();
            load(kd, kh, kw, c0, off);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float av[TM], bv[8];
#pragma unroll
            for (int i = 0; i < TM; i += 4) {
                const float4 t4 = *reinterpret_cast<const float4 *>(&As[buf][kk][tm * TM + i]);
                av[i] = t4.x; av[i + 1] = t4.y; av[i + 2] = t4.z; av[i + 3] = t4.w;
            }
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tn * 8]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tn * 8 + 4]);
            bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
            bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (s + 1 < S) store(buf ^ 1);
        __syncthreads();
    }

    // epilogue: bias, ReLU, residual, store
    float bias[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) bias[j] = a.bias[n0 + tn * 8 + j];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const long long m = m0 + tm * TM + i;
        if (m >= M) continue;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = fmaxf(acc[i][j] + bias[j], 0.f);
        if (a.residual) {
            const float *rx = a.x + (size_t)m * cx + n0 + tn * 8;
            const float4 r0 = *reinterpret_cast<const float4 *>(rx);
            const float4 r1 = *reinterpret_cast<const float4 *>(rx + 4);
            v[0] += r0.x; v[1] += r0.y; v[2] += r0.z; v[3] += r0.w;
            v[4] += r1.x; v[5] += r1.y; v[6] += r1.z; v[7] += r1.w;
        }
        float *dst = a.y + (size_t)m * co + n0 + tn * 8;
        *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
}

template <bool BF16>
__global__ void maxpool2_kernel(PoolArgs a) {
    // one thread per (pose, z, y, x, channel group) of the output: 8 bf16 channels (one 16-byte load per
    // source voxel) or 4 float channels
    constexpr int CG = BF16 ? 8 : 4;
    const int cq = a.c / CG;
    const long long total = (long long)a.B * a.n_out * a.n_out * a.n_out * cq;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e % cq);
        long long r = e / cq;
        const int x = (int)(r % a.n_out); r /= a.n_out;
        const int y = (int)(r % a.n_out); r /= a.n_out;
        const int z = (int)(r % a.n_out);
        const long long b = r / a.n_out;
        float m[CG];
#pragma unroll
        for (int j = 0; j < CG; ++j) m[j] = -INFINITY;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const size_t src = ((((size_t)b * a.n_in + 2 * z + dz) * a.n_in + 2 * y + dy) * a.n_in + 2 * x + dx) * a.c + q * CG;
                    if constexpr (BF16) {
                        const uint4 u = *reinterpret_cast<const uint4 *>(reinterpret_cast<const __nv_bfloat16 *>(a.x) + src);
                        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float2 f = __bfloat1622float2(h[j]);
                            m[2 * j] = fmaxf(m[2 * j], f.x);
                            m[2 * j + 1] = fmaxf(m[2 * j + 1], f.y);
                        }
                    } else {
                        const float4 v = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(a.x) + src);
                        m[0] = fmaxf(m[0], v.x); m[1] = fmaxf(m[1], v.y); m[2] = fmaxf(m[2], v.z); m[3] = fmaxf(m[3], v.w);
                    }
                }
        const size_t dst = e * CG;
        if constexpr (BF16) {
            uint4 u;
            __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
            for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(m[2 * j], m[2 * j + 1]);   // exact: maxima of bf16 values
            *reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(a.y) + dst) = u;
        } else {
            *reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.y) + dst) = make_float4(m[0], m[1], m[2], m[3]);
        }
    }
}

}  // namespace

void launch_conv3d_f32(const ConvArgs &a, cudaStream_t s) {
    const long long M = (long long)a.B * a.n_out * a.n_out * a.n_out;
    const unsigned gx = (unsigned)((M + BM - 1) / BM);
    if (a.c_out % 64 == 0) {
        conv3d_f32_kernel<64><<<dim3(gx, a.c_out / 64), NT, 0, s>>>(a);
    } else {
        conv3d_f32_kernel<32><<<dim3(gx, a.c_out / 32), NT, 0, s>>>(a);
    }
}

void launch_maxpool(const PoolArgs &a, cudaStream_t s) {
    const long long total = (long long)a.B * a.n_out * a.n_out * a.n_out * (a.c / (a.bf16 ? 8 : 4));
    long long nb = (total + 255) / 256;
    if (nb > 152LL * 16) nb = 152LL * 16;
    const int blocks = (int)(nb < 1 ? 1 : nb);
    if (a.bf16) maxpool2_kernel<true><<<blocks, 256, 0, s>>>(a);
    else maxpool2_kernel<false><<<blocks, 256, 0, s>>>(a);
}

}  // namespace fusion
