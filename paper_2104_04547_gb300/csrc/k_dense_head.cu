// CNN dense layer and fusion head.
//
// CNN dense (Section 3.3.1: flatten -> dense + ReLU): y[b][n] = ReLU(bias[n] +
// sum_k x[b][k] W[n][k]) with K = pooled voxels x channels (221,184 for the
// full-size model).  At small batch the weight stream dominates, so it is a
// split-K product: CTA (n-tile, split s, b-tile) multiplies a 64 x 64 tile over
// the K slice of split s from shared-memory tiles, and a second kernel adds the
// split partials in a fixed order (split count depends on K only, so a pose's
// result does not depend on its batch) and applies bias and ReLU.  The weight
// rows were permuted at model creation so that the flatten of the NDHWC pooled
// map is a plain row read.
//
// Fusion head (Section 3.3.3, Table V: fusion dense layers with SELU): one CTA
// per pose runs Linear -> SELU -> ... -> Linear on [cnn latent, sg latent].
#include "fusion_internal.cuh"

namespace fusion {

namespace {

constexpr int DT = 64;     // tile edge (poses and outputs)
constexpr int DBK = 32;    // K chunk

template <bool BF16>
__device__ __forceinline__ void load8(const void *base, size_t idx, bool ok, float *out) {
    if (!ok) {
#pragma unroll
        for (int j = 0; j < 8; ++j) out[j] = 0.f;
        return;
    }
    if constexpr (BF16) {
        const uint4 u = *reinterpret_cast<const uint4 *>(reinterpret_cast<const __nv_bfloat16 *>(base) + idx);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 f = __bfloat1622float2(h[j]);
            out[2 * j] = f.x;
            out[2 * j + 1] = f.y;
        }
    } else {
        const float *p = reinterpret_cast<const float *>(base) + idx;
        const float4 a = *reinterpret_cast<const float4 *>(p);
        const float4 b = *reinterpret_cast<const float4 *>(p + 4);
        out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
        out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
    }
}

template <bool BF16>
__global__ void __launch_bounds__(256) dense_splitk_kernel(DenseArgs a) {
    __shared__ __align__(16) float xs[DBK][DT + 4];
    __shared__ __align__(16) float ws[DBK][DT + 4];
    const int tid = threadIdx.x;
    const int n0 = blockIdx.x * DT;
    const int split = blockIdx.y;
    const int b0 = blockIdx.z * DT;
    const int kper = ((a.K + a.splits - 1) / a.splits + DBK - 1) / DBK * DBK;
    const int kbeg = split * kper;
    const int kend = min(a.K, kbeg + kper);

    // load role: row r = tid / 4 (0..63), k offset (tid % 4) * 8
    const int lr = tid >> 2, lk = (tid & 3) * 8;
    const int tr = tid / 16, tc = tid % 16;    // compute role: rows tr*4.., cols tc*4..
    float acc[4][4] = {};
    for (int kc = kbeg; kc < kend; kc += DBK) {
        float xv[8], wv[8];
        const int kk = kc + lk;
        const bool kin = kk < kend;      // K is a multiple of 8, so a chunk of 8 is all in or all out
        load8<BF16>(a.x, (size_t)(b0 + lr) * a.K + kk, kin && (b0 + lr) < a.B, xv);
        load8<BF16>(a.w, (size_t)(n0 + lr) * a.K + kk, kin && (n0 + lr) < a.N, wv);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            xs[lk + j][lr] = xv[j];
            ws[lk + j][lr] = wv[j];
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < DBK; ++q) {
            const float4 x4 = *reinterpret_cast<const float4 *>(&xs[q][tr * 4]);
            const float4 w4 = *reinterpret_cast<const float4 *>(&ws[q][tc * 4]);
            const float xr[4] = {x4.x, x4.y, x4.z, x4.w};
            const float wr[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xr[i], wr[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int b = b0 + tr * 4 + i;
        if (b >= a.B) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tc * 4 + j;
            if (n < a.N) a.part[((size_t)split * a.B + b) * a.N + n] = acc[i][j];
        }
    }
}

// Sum of the split partials in split order (fixed, so the result does not depend on the batch),
// plus bias and activation.  The partials are loaded 8 at a time ahead of the in-order additions so
// that a thread keeps several loads in flight instead of waiting on each one.
__global__ void dense_reduce_kernel(DenseArgs a) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.B * a.N) return;
    const int n = e % a.N;
    const size_t stride = (size_t)a.B * a.N;
    const float *p = a.part + e;
    float s = 0.f;
    int q = 0;
    for (; q + 8 <= a.splits; q += 8) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __ldg(p + (size_t)(q + j) * stride);
#pragma unroll
        for (int j = 0; j < 8; ++j) s += v[j];
    }
    for (; q < a.splits; ++q) s += __ldg(p + (size_t)q * stride);
    s += a.bias[n];
    a.y[e] = a.relu ? fmaxf(s, 0.f) : s;
}

__device__ __forceinline__ float selu(float x) {
    const float alpha = 1.6732632423543772848f, scale = 1.0507009873554804934f;
    return x > 0.f ? scale * x : scale * alpha * expm1f(x);
}

constexpr int kHeadThreads = 512;

// One dense layer of the head for one pose, all threads of the CTA: out[o] = act(b[o] + sum_k in[k] W[o][k])
// (weights stored transposed, [in][out]); act 0 = none, 1 = ReLU, 2 = SELU; `res` adds in[o] after the
// activation.  `in` and `out` are distinct shared-memory buffers.  A narrow layer splits its inputs into ks
// contiguous ranges (ks = 2, 4 or 8, as many as the CTA's threads allow), summed by different threads and
// added in range order after the bias, so its chains of dependent multiply-adds (and weight loads) are ks
// times shorter; the order depends only on the layer's shape.
__device__ void head_layer(const float *in, int fin, float *out, int fout, const float *wt, const float *bias,
                           int act, bool res) {
    __shared__ float part[kHeadThreads];
    int ks = 1;
    while (ks < 8 && fout * ks * 2 <= (int)blockDim.x) ks *= 2;
    if (ks == 1) {
        for (int o = threadIdx.x; o < fout; o += blockDim.x) {
            float s = bias[o];
            for (int k = 0; k < fin; ++k) s = fmaf(wt[(size_t)k * fout + o], in[k], s);
            if (act == 1) s = fmaxf(s, 0.f);
            else if (act == 2) s = selu(s);
            out[o] = res ? in[o] + s : s;
        }
        __syncthreads();
        return;
    }
    const int chunk = (fin + ks - 1) / ks;
    if ((int)threadIdx.x < fout * ks) {
        const int o = threadIdx.x % fout, q = threadIdx.x / fout;
        const int k1 = min(fin, (q + 1) * chunk);
        float s = 0.f;
        for (int k = q * chunk; k < k1; ++k) s = fmaf(wt[(size_t)k * fout + o], in[k], s);
        part[q * fout + o] = s;
    }
    __syncthreads();
    if ((int)threadIdx.x < fout) {
        const int o = threadIdx.x;
        float s = bias[o];
        for (int q = 0; q < ks; ++q) s += part[q * fout + o];
        if (act == 1) s = fmaxf(s, 0.f);
        else if (act == 2) s = selu(s);
        out[o] = res ? in[o] + s : s;
    }
    __syncthreads();
}

// Ask L2 for the CTA's share of a weight matrix's 128-byte lines (the head's weights, used by every CTA, are
// usually out of L2 after the convolutions' streams; each CTA otherwise walks them from DRAM in dependent rounds).
__device__ __forceinline__ void prefetch_share(const float *w, size_t n) {
    if (!w) return;
    const size_t lines = (n * 4 + 127) / 128;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < lines; q += (size_t)gridDim.x * blockDim.x)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(w) + q * 128));
}

// Coherent Fusion: fusion layers on [cnn, sg].  Mid-level: each latent through its branch layers (SELU
// after each), the two results appended after the latents, then the fusion layers.  Late: each latent
// through its own affinity stack (ReLU between, last linear), the mean of the two.
__global__ void __launch_bounds__(kHeadThreads) head_kernel(HeadArgs a) {
    __shared__ float v[3][kHeadMaxWidth];
    const int p = blockIdx.x;
    const int fin0 = a.Dc + a.G;
    {
        int fin = fin0;
        for (int br = 0; br < 2; ++br) {
            int bin = br == 0 ? a.Dc : a.G;
            for (int l = 0; l < a.n_branch[br]; ++l) {
                prefetch_share(a.bwt[br][l], (size_t)bin * a.bwidth[br][l]);
                bin = a.bwidth[br][l];
            }
            if (a.mode == FUSION_MID) fin += bin;
        }
        for (int l = 0; l < a.n_layers; ++l) {
            prefetch_share(a.wt[l], (size_t)fin * a.width[l]);
            fin = a.width[l];
        }
    }
    for (int i = threadIdx.x; i < fin0; i += blockDim.x)
        v[0][i] = i < a.Dc ? a.cnn[(size_t)p * a.Dc + i] : a.sg[(size_t)p * a.G + (i - a.Dc)];
    __syncthreads();
    if (a.mode == FUSION_LATE) {
        float aff[2];
        for (int br = 0; br < 2; ++br) {
            const float *in = v[0] + (br == 0 ? 0 : a.Dc);
            int fin = br == 0 ? a.Dc : a.G, cur = 1;
            for (int l = 0; l < a.n_branch[br]; ++l) {
                const bool last = l + 1 == a.n_branch[br];
                head_layer(in, fin, v[cur], a.bwidth[br][l], a.bwt[br][l], a.bb[br][l], last ? 0 : 1, false);
                in = v[cur];
                cur = cur == 1 ? 2 : 1;
                fin = a.bwidth[br][l];
            }
            aff[br] = in[0];
            __syncthreads();
        }
        if (threadIdx.x == 0) a.out[p] = 0.5f * (aff[0] + aff[1]);
        return;
    }
    int fin = fin0;
    if (a.mode == FUSION_MID) {
        for (int br = 0; br < 2; ++br) {
            const float *in = v[0] + (br == 0 ? 0 : a.Dc);
            int bin = br == 0 ? a.Dc : a.G, cur = 1;
            for (int l = 0; l < a.n_branch[br]; ++l) {
                head_layer(in, bin, v[cur], a.bwidth[br][l], a.bwt[br][l], a.bb[br][l], 2, false);
                in = v[cur];
                cur = cur == 1 ? 2 : 1;
                bin = a.bwidth[br][l];
            }
            for (int i = threadIdx.x; i < bin; i += blockDim.x) v[0][fin + i] = in[i];
            __syncthreads();
            fin += bin;
        }
    }
    int cur = 0;
    for (int l = 0; l < a.n_layers; ++l) {
        const int fout = a.width[l];
        const bool last = l + 1 == a.n_layers;
        const int nxt = cur == 0 ? 1 : 0;
        head_layer(v[cur], fin, v[nxt], fout, a.wt[l], a.b[l], last ? 0 : 2, !last && a.residual && fin == fout);
        cur = nxt;
        fin = fout;
    }
    if (threadIdx.x == 0) a.out[p] = v[cur][0];
}

}  // namespace

int dense_splits(int K) {
    int s = K / 2048;
    if (s < 1) s = 1;
    if (s > 128) s = 128;
    return s;
}

void launch_dense(const DenseArgs &a, cudaStream_t s) {
    dim3 grid((a.N + DT - 1) / DT, a.splits, (a.B + DT - 1) / DT);
    if (a.bf16) dense_splitk_kernel<true><<<grid, 256, 0, s>>>(a);
    else dense_splitk_kernel<false><<<grid, 256, 0, s>>>(a);
    launch_dense_reduce(a, s);
}

void launch_dense_reduce(const DenseArgs &a, cudaStream_t s) {
    const int tot = a.B * a.N;
    dense_reduce_kernel<<<(tot + 127) / 128, 128, 0, s>>>(a);
}

void launch_head(const HeadArgs &a, cudaStream_t s) {
    head_kernel<<<a.B, kHeadThreads, 0, s>>>(a);
}

}  // namespace fusion
