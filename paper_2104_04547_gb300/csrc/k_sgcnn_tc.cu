// The contractions of Section 3.3.1's gated graph convolution (PotentialNet's gated graph sequence steps,
// Table II) on the tcgen05 tensor cores, for the tensor-core models (BF16 / FP8): sg_gru_tc_kernel does a
// step's GRU update and the next step's edge transforms, sg_stage_tc_kernel a stage's input (the gate between
// stages) and its first transforms.
//
// Per step the message m_i (the segment sum of the neighbours' transforms, summed by sg_message_kernel in
// the SIMT path's order) and the node state h_i enter
//   [r | z] = m W_ih[r, z]^T + h W_hh[r, z]^T,   n_i = m W_ih[n]^T,   n_h = h W_hh[n]^T
//   r = sigmoid([r] + b_ir + b_hr), z = sigmoid([z] + b_iz + b_hz), n = tanh(n_i + b_in + r (n_h + b_hn))
//   h' = (1 - z) n + z h,           T_e = h' W_e^T + b_e  (the next step's neighbour transforms)
// These are dense [nodes x H] by [H x 3H] contractions, so a CTA takes 128 consecutive nodes (MMA M = 128)
// and runs them on the tensor cores with FP32 accumulators in tensor memory.  For FP32-class accuracy
// each operand x is split into two BF16 parts, x_hi = bf16(x) and x_lo = bf16(x - x_hi), and a product is
// the three MMAs x_lo y_hi + x_hi y_lo + x_hi y_hi (the dropped x_lo y_lo and the split's remainders are
// at most about 3 * 2^-16 of |x y|, a few 1e-6 of a dot product's sum of |terms|): the GRU runs on the
// tensor cores at close to FP32 accuracy, where plain BF16 graph arithmetic moved the affinity by 0.07.
//
// Layout: the weights are packed once per stage on the host as BF16 hi / lo parts, K-major
// ([k / 8][row][8], the no-swizzle core-matrix layout) and bulk-copied into shared memory once per
// persistent CTA.  The node tile's m and h arrive by coalesced loads (8 rows x 64 bytes per warp access),
// are split and stored in the same layout; h is also kept in FP32 for the z h term.  Tensor-memory columns:
// [r | z] 0 .. 2H, n_i 2H .. 3H, n_h 3H .. 4H; the transforms reuse columns 0 .. 2H after the GRU epilogue
// has read them.  Sixteen warps: warps w, w + 4, w + 8 and w + 12 read lane quarter w % 4 (node rows) and
// take a quarter of the output columns each.  Thread 0 issues the MMAs.  Every wait is bounded
// (FUSION_ERR_TIMEOUT).
#include "fusion_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

#include <cstring>
#include <vector>

namespace fusion {

namespace {

constexpr int kTileM = 128;
constexpr int kThreads = 512;
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s

// 32 lanes x 16 columns of 32-bit from tensor memory (this warp's lane quarter).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Shared-memory plan for width H (bytes).
template <int H>
struct Plan {
    static constexpr uint32_t kIH = 3 * H * H * 2;          // one BF16 part of W_ih or W_hh, [H/8][3H][8]
    static constexpr uint32_t kE = H * H * 2;               // one BF16 part of W_e, [H/8][H][8]
    static constexpr uint32_t kW = 4 * kIH + 4 * kE;        // the stage's weight image
    static constexpr uint32_t kA = kTileM * H * 2;          // one BF16 part of a node tile, [H/8][128][8]
    static constexpr uint32_t kHold = kTileM * H * 4;       // h in FP32, [128][H], float4 slots XOR-swizzled
    static constexpr uint32_t kBias = 6 * H * 4;            // b_ir+b_hr, b_iz+b_hz, b_in, b_hn, b_e0, b_e1
    static constexpr uint32_t oMhi = kW, oMlo = oMhi + kA, oHhi = oMlo + kA, oHlo = oHhi + kA;
    static constexpr uint32_t oHold = oHlo + kA;
    static constexpr uint32_t oBias = oHold + kHold;
    static constexpr uint32_t oBar = oBias + kBias;         // w_bar, mma_bar, tmem slot
    static constexpr uint32_t kSmem = oBar + 32;
    static constexpr uint32_t kTmemCols = 4 * H;            // 256 or 128: a power of two >= 32
    static constexpr int kCols = H / 4;                     // output columns per thread (four warps per quarter)
};

// Float4 slot of (row r, float4 column f4) in the FP32 h tile: rows are H floats, slots XOR-swizzled by r % 8,
// so both the loaders' 8-row x 4-slot writes and the epilogue's 32-row reads of one slot spread over all banks.
template <int H>
__device__ __forceinline__ int hold_slot(int r, int f4) { return r * (H / 4) + (f4 ^ (r & 7)); }

// x -> (bf16(x), bf16(x - bf16(x))) for four consecutive K values, as two 8-byte halves of core-matrix rows.
__device__ __forceinline__ void split4(const float4 &x, uint2 &hi, uint2 &lo) {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(x.x, x.y), h23 = __floats2bfloat162_rn(x.z, x.w);
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(x.x - f01.x, x.y - f01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(x.z - f23.x, x.w - f23.y);
    hi.x = *reinterpret_cast<const uint32_t *>(&h01);
    hi.y = *reinterpret_cast<const uint32_t *>(&h23);
    lo.x = *reinterpret_cast<const uint32_t *>(&l01);
    lo.y = *reinterpret_cast<const uint32_t *>(&l23);
}

// sigmoid and tanh from the exponential: 1 / (1 + e^-x) and 1 - 2 / (1 + e^2x) (both saturate correctly
// when the exponential overflows to infinity).
__device__ __forceinline__ float sigm_fast(float x) { return __fdividef(1.f, 1.f + __expf(-x)); }
__device__ __forceinline__ float tanh_fast(float x) { return 1.f - __fdividef(2.f, 1.f + __expf(2.f * x)); }

// 32 lanes x C columns (C = 8 or 16) of 32-bit from tensor memory (this warp's lane quarter).
template <int C>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[C]) {
    if constexpr (C == 16) {
        tmem_ld16(taddr, r);
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(taddr));
    }
}

// D (tensor memory, 128 x N) (+)= A B^T over K = H as three BF16 MMAs per K step (lo hi, hi lo, hi hi).
// A: a node tile part pair in shared memory; B: rows of a weight part pair, `brows` rows per k-slice.
template <int H>
__device__ __forceinline__ void product1(uint32_t d, uint32_t a, uint32_t b, int brows, uint32_t idesc,
                                         bool accumulate) {
    const uint64_t ad = tc::desc_kmajor(a, kTileM * 16, 128);
    const uint64_t bd = tc::desc_kmajor(b, (uint32_t)brows * 16, 128);
#pragma unroll
    for (int k = 0; k < H / 16; ++k)
        tc::mma_bf16(d, ad + (uint64_t)(k * 2 * kTileM), bd + (uint64_t)(k * 2 * brows), idesc,
                     (accumulate || k > 0) ? 1u : 0u);
}

template <int H>
__device__ __forceinline__ void product3(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                         int brows, uint32_t idesc, bool accumulate) {
    product1<H>(d, a_lo, b_hi, brows, idesc, accumulate);
    product1<H>(d, a_hi, b_lo, brows, idesc, true);
    product1<H>(d, a_hi, b_hi, brows, idesc, true);
}

template <int H>
__global__ void __launch_bounds__(kThreads, 1) sg_gru_tc_kernel(SgGruTcArgs a) {
    using P = Plan<H>;
    constexpr int C = P::kCols;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *w_bar = reinterpret_cast<uint64_t *>(smem + P::oBar);
    uint64_t *mma_bar = w_bar + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_bar + 1);
    float4 *hold = reinterpret_cast<float4 *>(smem + P::oHold);
    float *sb = reinterpret_cast<float *>(smem + P::oBias);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int A = a.A_dev ? *a.A_dev : a.A;
    if (A > a.A) A = a.A;
    const int n_tiles = (A + kTileM - 1) / kTileM;
    const bool any_T = a.T_out[0] || a.T_out[1];
    const uint64_t deadline = tc::globaltimer() + kWaitNs;

    if (tid == 0) {
        tc::mbar_init(w_bar, 1);
        tc::mbar_init(mma_bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, P::kTmemCols);
    for (int o = tid; o < H; o += kThreads) {
        sb[o] = a.bih[o] + a.bhh[o];
        sb[H + o] = a.bih[H + o] + a.bhh[H + o];
        sb[2 * H + o] = a.bih[2 * H + o];
        sb[3 * H + o] = a.bhh[2 * H + o];
        sb[4 * H + o] = a.T_out[0] ? a.be[0][o] : 0.f;
        sb[5 * H + o] = a.T_out[1] ? a.be[1][o] : 0.f;
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = *tmem_slot;

    // the stage's weights: W_ih and W_hh always, W_e where the next step's transforms are wanted
    bool w_issued = false, w_ready = false;
    if (tid == 0 && (int)blockIdx.x < n_tiles && !a.stall) {
        const unsigned char *g = reinterpret_cast<const unsigned char *>(a.w);
        uint32_t bytes = 4 * P::kIH;
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (a.T_out[e]) bytes += 2 * P::kE;
        tc::mbar_expect_tx(w_bar, bytes);
        tc::bulk_load(smem, g, 4 * P::kIH, w_bar);
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (a.T_out[e]) {
                const uint32_t o = 4 * P::kIH + e * 2 * P::kE;
                tc::bulk_load(smem + o, g + o, 2 * P::kE, w_bar);
            }
        w_issued = true;
    }

    const uint32_t s0 = tc::smem_u32(smem);
    const uint32_t sMhi = s0 + P::oMhi, sMlo = s0 + P::oMlo, sHhi = s0 + P::oHhi, sHlo = s0 + P::oHlo;
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;                  // this thread's node row in the tile
    const int o0 = (warp >> 2) * C;                       // its output columns o0 .. o0 + C
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    uint32_t phase = 0;
    bool pending = false;                                 // a commit not yet seen complete
    bool ok = true;

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int i0 = tile * kTileM;
        // ---- m and h of the tile -> BF16 hi / lo parts (and h in FP32); rows past A read as zero ----
        {
            constexpr int F4 = H / 4;                     // float4 per row
            constexpr int CG = F4 / 4;                    // 4-float4 column groups per row
#pragma unroll
            for (int idx = tid; idx < kTileM * F4; idx += kThreads) {
                const int g = idx >> 5, l = idx & 31;
                const int r = (g / CG) * 8 + (l >> 2);
                const int f4 = (g % CG) * 4 + (l & 3);
                const int gi = i0 + r;
                float4 xm = make_float4(0.f, 0.f, 0.f, 0.f), xh = xm;
                if (gi < A) {
                    xm = __ldg(reinterpret_cast<const float4 *>(a.m + (size_t)gi * H) + f4);
                    xh = __ldg(reinterpret_cast<const float4 *>(a.h_in + (size_t)gi * H) + f4);
                }
                const uint32_t o = (uint32_t)(((f4 >> 1) * kTileM + r) * 16 + (f4 & 1) * 8);
                uint2 hi, lo;
                split4(xm, hi, lo);
                *reinterpret_cast<uint2 *>(smem + P::oMhi + o) = hi;
                *reinterpret_cast<uint2 *>(smem + P::oMlo + o) = lo;
                split4(xh, hi, lo);
                *reinterpret_cast<uint2 *>(smem + P::oHhi + o) = hi;
                *reinterpret_cast<uint2 *>(smem + P::oHlo + o) = lo;
                hold[hold_slot<H>(r, f4)] = xh;
            }
        }
        tc::fence_proxy_async();
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();

        // ---- GRU products ----
        bool issued = true;
        if (tid == 0) {
            if (!w_ready) {
                w_ready = tc::mbar_wait(w_bar, 0, deadline, a.err, FUSION_ERR_TIMEOUT);
                issued = w_ready;
            }
            if (issued) {
                tc::tc_fence_after();
                const uint32_t ih_hi = s0, ih_lo = s0 + P::kIH, hh_hi = s0 + 2 * P::kIH, hh_lo = s0 + 3 * P::kIH;
                constexpr uint32_t I2 = tc::idesc_bf16(kTileM, 2 * H), I1 = tc::idesc_bf16(kTileM, H);
                constexpr uint32_t nrow = 2 * H * 16;     // byte offset of the n-gate rows
                product3<H>(tbase, sMhi, sMlo, ih_hi, ih_lo, 3 * H, I2, false);
                product3<H>(tbase, sHhi, sHlo, hh_hi, hh_lo, 3 * H, I2, true);
                product3<H>(tbase + 2 * H, sMhi, sMlo, ih_hi + nrow, ih_lo + nrow, 3 * H, I1, false);
                product3<H>(tbase + 3 * H, sHhi, sHlo, hh_hi + nrow, hh_lo + nrow, 3 * H, I1, false);
                tc::mma_commit(mma_bar);
                pending = true;
            }
        }
        if (!__syncthreads_and(issued)) { ok = false; break; }
        if (!__syncthreads_and(tc::mbar_wait(mma_bar, phase, deadline, a.err, FUSION_ERR_TIMEOUT))) {
            ok = false;
            break;
        }
        phase ^= 1;
        pending = false;
        tc::tc_fence_after();

        // ---- GRU epilogue: h' to global, and its BF16 parts over the tile's m ----
        const int gi = i0 + row;
        const bool valid = gi < A;
        {
            uint32_t vr[C], vz[C], vn[C], vh[C];
            tmem_ld_cols<C>(tbase + lane_addr + o0, vr);
            tmem_ld_cols<C>(tbase + lane_addr + H + o0, vz);
            tmem_ld_cols<C>(tbase + lane_addr + 2 * H + o0, vn);
            tmem_ld_cols<C>(tbase + lane_addr + 3 * H + o0, vh);
            tc::tmem_ld_wait();
            float hn[C];
#pragma unroll
            for (int q4 = 0; q4 < C / 4; ++q4) {
                const float4 ho = hold[hold_slot<H>(row, o0 / 4 + q4)];
                const float hv[4] = {ho.x, ho.y, ho.z, ho.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = 4 * q4 + u, o = o0 + q;
                    const float r = sigm_fast(__uint_as_float(vr[q]) + sb[o]);
                    const float z = sigm_fast(__uint_as_float(vz[q]) + sb[H + o]);
                    const float n = tanh_fast(__uint_as_float(vn[q]) + sb[2 * H + o] +
                                              r * (__uint_as_float(vh[q]) + sb[3 * H + o]));
                    hn[q] = (1.f - z) * n + z * hv[u];
                }
            }
            if (valid) {
                float4 *dst = reinterpret_cast<float4 *>(a.h_out + (size_t)gi * H + o0);
#pragma unroll
                for (int q = 0; q < C / 4; ++q) dst[q] = make_float4(hn[4 * q], hn[4 * q + 1], hn[4 * q + 2], hn[4 * q + 3]);
            }
#pragma unroll
            for (int s = 0; s < C / 8; ++s) {
                uint2 h0, l0, h1, l1;
                split4(make_float4(hn[8 * s], hn[8 * s + 1], hn[8 * s + 2], hn[8 * s + 3]), h0, l0);
                split4(make_float4(hn[8 * s + 4], hn[8 * s + 5], hn[8 * s + 6], hn[8 * s + 7]), h1, l1);
                const uint32_t o = (uint32_t)((((o0 >> 3) + s) * kTileM + row) * 16);
                *reinterpret_cast<uint4 *>(smem + P::oMhi + o) = make_uint4(h0.x, h0.y, h1.x, h1.y);
                *reinterpret_cast<uint4 *>(smem + P::oMlo + o) = make_uint4(l0.x, l0.y, l1.x, l1.y);
            }
        }

        if (any_T) {
            tc::fence_proxy_async();
            tc::tc_fence_before();
            __syncthreads();
            tc::tc_fence_after();
            // ---- next step's transforms T_e = h' W_e^T + b_e (columns e H .. (e + 1) H) ----
            if (tid == 0) {
                constexpr uint32_t I1 = tc::idesc_bf16(kTileM, H);
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    if (a.T_out[e]) {
                        const uint32_t we = s0 + 4 * P::kIH + e * 2 * P::kE;
                        product3<H>(tbase + e * H, sMhi, sMlo, we, we + P::kE, H, I1, false);
                    }
                tc::mma_commit(mma_bar);
                pending = true;
            }
            if (!__syncthreads_and(tc::mbar_wait(mma_bar, phase, deadline, a.err, FUSION_ERR_TIMEOUT))) {
                ok = false;
                break;
            }
            phase ^= 1;
            pending = false;
            tc::tc_fence_after();
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (!a.T_out[e]) continue;
                uint32_t v[C];
                tmem_ld_cols<C>(tbase + lane_addr + e * H + o0, v);
                tc::tmem_ld_wait();
                if (valid) {
                    const float *be = sb + (4 + e) * H + o0;
                    float4 *dst = reinterpret_cast<float4 *>(a.T_out[e] + (size_t)gi * H + o0);
#pragma unroll
                    for (int q = 0; q < C / 4; ++q)
                        dst[q] = make_float4(__uint_as_float(v[4 * q]) + be[4 * q], __uint_as_float(v[4 * q + 1]) + be[4 * q + 1],
                                             __uint_as_float(v[4 * q + 2]) + be[4 * q + 2],
                                             __uint_as_float(v[4 * q + 3]) + be[4 * q + 3]);
                }
            }
        }
        // the next tile overwrites the operand tiles and the accumulators
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
    }

    if (!ok) atomicOr(a.err, FUSION_ERR_TIMEOUT);
    // no copy or MMA of this CTA may still be writing when it frees tensor memory and exits
    if (tid == 0) {
        const uint64_t dl = tc::globaltimer() + 100000000ull;
        if (w_issued && !w_ready && !tc::mbar_wait(w_bar, 0, dl)) atomicOr(a.err, FUSION_ERR_TIMEOUT);
        if (pending && !tc::mbar_wait(mma_bar, phase, dl)) atomicOr(a.err, FUSION_ERR_TIMEOUT);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tbase, P::kTmemCols);
}

// ---- stage start: the stage input x and its first transforms ----
//
// x = sigmoid(W_i [h, h0] + b_i) * (W_j h + b_j) with the gate between stages, else x = h0 (the first stage:
// atom features zero-padded to H) or x = h (no gate); then T_e = W_e x + b_e for the stage's edge types.
// Tensor-memory columns: W_i [h, h0] at 0 .. H and W_j h at H .. 2H ([W_i,h ; W_j] is one N = 2H product of
// h, W_i,h0 h0 accumulates onto the first half); the transforms reuse 0 .. 2H.
template <int H>
struct StagePlan {
    static constexpr uint32_t kGa = 2 * H * H * 2;          // one BF16 part of [W_i,h ; W_j], [H/8][2H][8]
    static constexpr uint32_t kGb = H * H * 2;              // one BF16 part of W_i,h0, [H/8][H][8]
    static constexpr uint32_t kE = H * H * 2;               // one BF16 part of W_e
    static constexpr uint32_t oGb = 2 * kGa, oE = oGb + 2 * kGb, kW = oE + 4 * kE;
    static constexpr uint32_t kA = kTileM * H * 2;
    static constexpr uint32_t oXhi = kW, oXlo = oXhi + kA, oYhi = oXlo + kA, oYlo = oYhi + kA;
    static constexpr uint32_t oBias = oYlo + kA;            // b_i, b_j, b_e0, b_e1
    static constexpr uint32_t oBar = oBias + 4 * H * 4;
    static constexpr uint32_t kSmem = oBar + 32;
    static constexpr uint32_t kTmemCols = 2 * H;            // 128 or 64
    static constexpr int kCols = H / 4;
};

template <int H>
__global__ void __launch_bounds__(kThreads, 1) sg_stage_tc_kernel(SgStageTcArgs a) {
    using P = StagePlan<H>;
    constexpr int C = P::kCols;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *w_bar = reinterpret_cast<uint64_t *>(smem + P::oBar);
    uint64_t *mma_bar = w_bar + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_bar + 1);
    float *sb = reinterpret_cast<float *>(smem + P::oBias);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int A = a.A_dev ? *a.A_dev : a.A;
    if (A > a.A) A = a.A;
    const int n_tiles = (A + kTileM - 1) / kTileM;
    const bool gate = a.wg != nullptr && a.h_in != nullptr;
    const bool any_T = a.T_out[0] || a.T_out[1];
    const uint64_t deadline = tc::globaltimer() + kWaitNs;

    if (tid == 0) {
        tc::mbar_init(w_bar, 1);
        tc::mbar_init(mma_bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, P::kTmemCols);
    for (int o = tid; o < H; o += kThreads) {
        sb[o] = gate ? a.gbi[o] : 0.f;
        sb[H + o] = gate ? a.gbj[o] : 0.f;
        sb[2 * H + o] = a.T_out[0] ? a.be[0][o] : 0.f;
        sb[3 * H + o] = a.T_out[1] ? a.be[1][o] : 0.f;
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = *tmem_slot;

    bool w_issued = false, w_ready = false;
    if (tid == 0 && (int)blockIdx.x < n_tiles && (gate || any_T) && !a.stall) {
        uint32_t bytes = gate ? 2 * P::kGa + 2 * P::kGb : 0;
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (a.T_out[e]) bytes += 2 * P::kE;
        tc::mbar_expect_tx(w_bar, bytes);
        if (gate) tc::bulk_load(smem, a.wg, 2 * P::kGa + 2 * P::kGb, w_bar);
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (a.T_out[e])
                tc::bulk_load(smem + P::oE + e * 2 * P::kE, reinterpret_cast<const unsigned char *>(a.we) + e * 2 * P::kE,
                              2 * P::kE, w_bar);
        w_issued = true;
    }

    const uint32_t s0 = tc::smem_u32(smem);
    const uint32_t sXhi = s0 + P::oXhi, sXlo = s0 + P::oXlo, sYhi = s0 + P::oYhi, sYlo = s0 + P::oYlo;
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int o0 = (warp >> 2) * C;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    uint32_t phase = 0;
    bool pending = false, ok = true;

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int i0 = tile * kTileM;
        // ---- operands: gate: X = h, Y = h0; otherwise X = x (= h0 or h), also written out here ----
        {
            constexpr int F4 = H / 4, CG = F4 / 4;
#pragma unroll
            for (int idx = tid; idx < kTileM * F4; idx += kThreads) {
                const int g = idx >> 5, l = idx & 31;
                const int r = (g / CG) * 8 + (l >> 2);
                const int f4 = (g % CG) * 4 + (l & 3);
                const int gi = i0 + r;
                float4 h0 = make_float4(0.f, 0.f, 0.f, 0.f), h = h0;
                if (gi < A) {
                    float f[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int o = 4 * f4 + u;
                        f[u] = o < kFeat ? __ldg(a.feat + (size_t)gi * kFeat + o) : 0.f;
                    }
                    h0 = make_float4(f[0], f[1], f[2], f[3]);
                    if (a.h_in) h = __ldg(reinterpret_cast<const float4 *>(a.h_in + (size_t)gi * H) + f4);
                }
                const float4 x = gate ? h : (a.h_in ? h : h0);
                const uint32_t o = (uint32_t)(((f4 >> 1) * kTileM + r) * 16 + (f4 & 1) * 8);
                uint2 hi, lo;
                split4(x, hi, lo);
                *reinterpret_cast<uint2 *>(smem + P::oXhi + o) = hi;
                *reinterpret_cast<uint2 *>(smem + P::oXlo + o) = lo;
                if (gate) {
                    split4(h0, hi, lo);
                    *reinterpret_cast<uint2 *>(smem + P::oYhi + o) = hi;
                    *reinterpret_cast<uint2 *>(smem + P::oYlo + o) = lo;
                } else if (gi < A) {
                    reinterpret_cast<float4 *>(a.x_out + (size_t)gi * H)[f4] = x;
                }
            }
        }
        tc::fence_proxy_async();
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();

        const int gi = i0 + row;
        const bool valid = gi < A;
        if (gate) {
            bool issued = true;
            if (tid == 0) {
                if (!w_ready) {
                    w_ready = tc::mbar_wait(w_bar, 0, deadline, a.err, FUSION_ERR_TIMEOUT);
                    issued = w_ready;
                }
                if (issued) {
                    tc::tc_fence_after();
                    constexpr uint32_t I2 = tc::idesc_bf16(kTileM, 2 * H), I1 = tc::idesc_bf16(kTileM, H);
                    product3<H>(tbase, sXhi, sXlo, s0, s0 + P::kGa, 2 * H, I2, false);
                    product3<H>(tbase, sYhi, sYlo, s0 + P::oGb, s0 + P::oGb + P::kGb, H, I1, true);
                    tc::mma_commit(mma_bar);
                    pending = true;
                }
            }
            if (!__syncthreads_and(issued)) { ok = false; break; }
            if (!__syncthreads_and(tc::mbar_wait(mma_bar, phase, deadline, a.err, FUSION_ERR_TIMEOUT))) {
                ok = false;
                break;
            }
            phase ^= 1;
            pending = false;
            tc::tc_fence_after();
            // ---- x = sigmoid(gi + b_i) * (gj + b_j): to global and as the transforms' operand ----
            uint32_t vi[C], vj[C];
            tmem_ld_cols<C>(tbase + lane_addr + o0, vi);
            tmem_ld_cols<C>(tbase + lane_addr + H + o0, vj);
            tc::tmem_ld_wait();
            float x[C];
#pragma unroll
            for (int q = 0; q < C; ++q)
                x[q] = sigm_fast(__uint_as_float(vi[q]) + sb[o0 + q]) * (__uint_as_float(vj[q]) + sb[H + o0 + q]);
            if (valid) {
                float4 *dst = reinterpret_cast<float4 *>(a.x_out + (size_t)gi * H + o0);
#pragma unroll
                for (int q = 0; q < C / 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
            }
#pragma unroll
            for (int s = 0; s < C / 8; ++s) {
                uint2 h0, l0, h1, l1;
                split4(make_float4(x[8 * s], x[8 * s + 1], x[8 * s + 2], x[8 * s + 3]), h0, l0);
                split4(make_float4(x[8 * s + 4], x[8 * s + 5], x[8 * s + 6], x[8 * s + 7]), h1, l1);
                const uint32_t o = (uint32_t)((((o0 >> 3) + s) * kTileM + row) * 16);
                *reinterpret_cast<uint4 *>(smem + P::oXhi + o) = make_uint4(h0.x, h0.y, h1.x, h1.y);
                *reinterpret_cast<uint4 *>(smem + P::oXlo + o) = make_uint4(l0.x, l0.y, l1.x, l1.y);
            }
            tc::fence_proxy_async();
            tc::tc_fence_before();
            __syncthreads();
            tc::tc_fence_after();
        }

        if (any_T) {
            // ---- T_e = x W_e^T + b_e (columns e H .. (e + 1) H) ----
            bool issued = true;
            if (tid == 0) {
                if (!w_ready) {
                    w_ready = tc::mbar_wait(w_bar, 0, deadline, a.err, FUSION_ERR_TIMEOUT);
                    issued = w_ready;
                }
                if (issued) {
                    tc::tc_fence_after();
                    constexpr uint32_t I1 = tc::idesc_bf16(kTileM, H);
#pragma unroll
                    for (int e = 0; e < 2; ++e)
                        if (a.T_out[e]) {
                            const uint32_t we = s0 + P::oE + e * 2 * P::kE;
                            product3<H>(tbase + e * H, sXhi, sXlo, we, we + P::kE, H, I1, false);
                        }
                    tc::mma_commit(mma_bar);
                    pending = true;
                }
            }
            if (!__syncthreads_and(issued)) { ok = false; break; }
            if (!__syncthreads_and(tc::mbar_wait(mma_bar, phase, deadline, a.err, FUSION_ERR_TIMEOUT))) {
                ok = false;
                break;
            }
            phase ^= 1;
            pending = false;
            tc::tc_fence_after();
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (!a.T_out[e]) continue;
                uint32_t v[C];
                tmem_ld_cols<C>(tbase + lane_addr + e * H + o0, v);
                tc::tmem_ld_wait();
                if (valid) {
                    const float *be = sb + (2 + e) * H + o0;
                    float4 *dst = reinterpret_cast<float4 *>(a.T_out[e] + (size_t)gi * H + o0);
#pragma unroll
                    for (int q = 0; q < C / 4; ++q)
                        dst[q] = make_float4(__uint_as_float(v[4 * q]) + be[4 * q], __uint_as_float(v[4 * q + 1]) + be[4 * q + 1],
                                             __uint_as_float(v[4 * q + 2]) + be[4 * q + 2],
                                             __uint_as_float(v[4 * q + 3]) + be[4 * q + 3]);
                }
            }
        }
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
    }

    if (!ok) atomicOr(a.err, FUSION_ERR_TIMEOUT);
    if (tid == 0) {
        const uint64_t dl = tc::globaltimer() + 100000000ull;
        if (w_issued && !w_ready && !tc::mbar_wait(w_bar, 0, dl)) atomicOr(a.err, FUSION_ERR_TIMEOUT);
        if (pending && !tc::mbar_wait(mma_bar, phase, dl)) atomicOr(a.err, FUSION_ERR_TIMEOUT);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tbase, P::kTmemCols);
}

uint16_t host_bf16(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float host_f32(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// [rows][H] row-major -> hi part at dst, lo part at dst + rows * H, each [H / 8][rows][8].
void pack_parts(const float *w, int rows, int H, uint16_t *dst) {
    uint16_t *lo = dst + (size_t)rows * H;
    for (int r = 0; r < rows; ++r)
        for (int k = 0; k < H; ++k) {
            const float x = w[(size_t)r * H + k];
            const uint16_t h = host_bf16(x);
            const size_t o = ((size_t)(k / 8) * rows + r) * 8 + k % 8;
            dst[o] = h;
            lo[o] = host_bf16(x - host_f32(h));
        }
}

}  // namespace

size_t sg_gru_tc_image_elems(int H) { return (size_t)16 * H * H; }

size_t sg_stage_tc_image_elems(int H) { return (size_t)6 * H * H; }

void sg_stage_tc_pack(const float *wi, const float *wj, int H, uint16_t *img) {
    // [W_i,h ; W_j] ([2H][H]: W_i's columns of h, then W_j), then W_i,h0 ([H][H]: W_i's columns of h0)
    std::vector<float> ga((size_t)2 * H * H), gb((size_t)H * H);
    for (int r = 0; r < H; ++r)
        for (int k = 0; k < H; ++k) {
            ga[(size_t)r * H + k] = wi[(size_t)r * 2 * H + k];
            ga[(size_t)(H + r) * H + k] = wj[(size_t)r * H + k];
            gb[(size_t)r * H + k] = wi[(size_t)r * 2 * H + H + k];
        }
    pack_parts(ga.data(), 2 * H, H, img);
    pack_parts(gb.data(), H, H, img + (size_t)4 * H * H);
}

void sg_gru_tc_pack(const float *wih, const float *whh, const float *we0, const float *we1, int H, uint16_t *img) {
    const size_t nIH = (size_t)3 * H * H, nE = (size_t)H * H;
    pack_parts(wih, 3 * H, H, img);
    pack_parts(whh, 3 * H, H, img + 2 * nIH);
    uint16_t *e = img + 4 * nIH;
    for (int s = 0; s < 2; ++s) {
        const float *w = s == 0 ? we0 : we1;
        if (w) pack_parts(w, H, H, e + s * 2 * nE);
        else std::memset(e + s * 2 * nE, 0, 2 * nE * sizeof(uint16_t));
    }
}

// Persistent grid: the SMs times the CTAs of the kernel that fit one SM.
template <class K>
static int grid_cap(K kernel, uint32_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
    return (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
}

template <int H>
static int gru_cap() {
    static int cap = grid_cap(sg_gru_tc_kernel<H>, Plan<H>::kSmem);
    return cap;
}

template <int H>
static int stage_cap() {
    static int cap = grid_cap(sg_stage_tc_kernel<H>, StagePlan<H>::kSmem);
    return cap;
}

void sg_gru_tc_prepare(int H) {
    if (H == 64) {
        gru_cap<64>();
        stage_cap<64>();
    } else {
        gru_cap<32>();
        stage_cap<32>();
    }
}

static int persistent_grid(int A, int cap) {
    const int tiles = (A + kTileM - 1) / kTileM;
    return tiles < cap ? tiles : cap;
}

void launch_sg_gru_tc(const SgGruTcArgs &a, cudaStream_t s) {
    if (a.H == 64) {
        const int g = persistent_grid(a.A, gru_cap<64>());
        if (g > 0) sg_gru_tc_kernel<64><<<g, kThreads, Plan<64>::kSmem, s>>>(a);
    } else {
        const int g = persistent_grid(a.A, gru_cap<32>());
        if (g > 0) sg_gru_tc_kernel<32><<<g, kThreads, Plan<32>::kSmem, s>>>(a);
    }
}

void launch_sg_stage_tc(const SgStageTcArgs &a, cudaStream_t s) {
    if (a.H == 64) {
        const int g = persistent_grid(a.A, stage_cap<64>());
        if (g > 0) sg_stage_tc_kernel<64><<<g, kThreads, StagePlan<64>::kSmem, s>>>(a);
    } else {
        const int g = persistent_grid(a.A, stage_cap<32>());
        if (g > 0) sg_stage_tc_kernel<32><<<g, kThreads, StagePlan<32>::kSmem, s>>>(a);
    }
}

}  // namespace fusion
