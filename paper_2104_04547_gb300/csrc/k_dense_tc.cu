// CNN dense layer on the tcgen05 tensor cores, bf16 inputs and weights, FP32 accumulation
// (Section 3.3.1: flatten -> dense + ReLU, the 221,184 -> 256 layer of the full-size model).
//
// y[b][n] = act(bias[n] + sum_k x[b][k] W[n][k]).  At the batch sizes of a scoring call the layer
// streams 113 MB of weights for 7 GFLOP, so it is a weight-streaming split-K product: CTA
// (m-tile, split s, b-tile) computes D = W[m-tile rows][K slice s] x[b-tile][K slice s]^T as
// M = 128 output channels x N = 64 poses in tensor memory, and writes the FP32 partial; the fixed-
// order reduction over the splits (shared with the SIMT path) adds bias and ReLU.  The split
// boundaries depend on K and the output width only, so a pose's result does not depend on its batch.
//
// Operands: both matrices are K-major in global memory ([rows][K] bf16).  A 2-D tensor map with a box of
// 64 elements (128 bytes) x the tile's rows and 128-byte swizzling lands each 64-wide K stage in shared
// memory as rows of 128 bytes whose 16-byte chunks are permuted by the row index mod 8: the K-major
// 128-byte-swizzle layout of the MMA descriptors (8-row atoms of 1 KB, 1 KB apart; a K step of 16 moves the
// start address 32 bytes along the row).  Each TMA request then moves whole 128-byte rows.  Rows beyond the
// matrix and K beyond its end are zero-filled by TMA.
//
// Roles: warp 0 lane 0 issues the TMA loads into a ring of stages; warp 1 owns tensor memory and
// its lane 0 issues 4 MMAs (K = 16 each) per stage; warps 2..5 (one per tensor-memory lane quarter)
// read the accumulator and store the partial.  Every wait is bounded: one that runs out sets
// FUSION_ERR_TIMEOUT and the CTA drains and returns.
#include "fusion_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>

namespace fusion {

namespace {

constexpr int kBM = 128;                  // output channels per tile (MMA M)
constexpr int kBN = 64;                   // poses per tile (MMA N)
constexpr int kBK = 64;                   // K per stage
constexpr int kStages = 6;
constexpr uint32_t kABytes = kBM * kBK * 2;
constexpr uint32_t kBBytes = kBN * kBK * 2;
constexpr uint32_t kStageBytes = kABytes + kBBytes;
constexpr int kThreads = 192;
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s

// 2-D tiled TMA load into shared memory, completing on `bar` (coordinates: K element, row).
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            tc::smem_u32(dst)),
        "l"(tmap), "r"(tc::smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

// Shared-memory matrix descriptor, K-major with 128-byte swizzling (layout type 2 in bits 61..63): rows of
// 128 bytes, 8-row atoms 1024 bytes apart (stride byte offset), the leading byte offset unused (1); the
// tile starts on a 1024-byte boundary, so the base-offset field is 0.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

struct TcArgs {
    float *part;          // [splits][B][N]
    int B, N, K, kper;
    unsigned *err;
};

__global__ void __launch_bounds__(kThreads, 1) dense_tc_kernel(const __grid_constant__ CUtensorMap tw,
                                                               const __grid_constant__ CUtensorMap tx, TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr uint32_t IDESC = tc::idesc_bf16(kBM, kBN);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_full + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kBM, split = blockIdx.y, b0 = blockIdx.z * kBN;
    const int kbeg = split * a.kper;
    const int kend = min(a.K, kbeg + a.kper);
    const int niter = (kend - kbeg + kBK - 1) / kBK;
    const uint64_t deadline = tc::globaltimer() + kWaitNs;

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) { tc::mbar_init(&full[i], 1); tc::mbar_init(&empty[i], 1); }
        tc::mbar_init(acc_full, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, kBN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(a.err, FUSION_ERR_TIMEOUT);
    };

    int issued = 0;
    if (warp == 0 && lane == 0) {
        // ---------------- producer ----------------
        for (int it = 0; it < niter && !*abort_flag; ++it) {
            const int st = it % kStages;
            if (!tc::mbar_wait(&empty[st], ((it / kStages) & 1) ^ 1, deadline, a.err, FUSION_ERR_TIMEOUT)) { fail(); break; }
            tc::mbar_expect_tx(&full[st], kStageBytes);
            unsigned char *sa = smem + st * kStageBytes;
            const int kk = kbeg + it * kBK;
            tma_load_2d(sa, &tw, &full[st], kk, m0);
            tma_load_2d(sa + kABytes, &tx, &full[st], kk, b0);
            ++issued;
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t a0 = tc::smem_u32(smem), bofs = kABytes;
        for (int it = 0; it < niter && !*abort_flag; ++it) {
            const int st = it % kStages;
            if (!tc::mbar_wait(&full[st], (it / kStages) & 1, deadline, a.err, FUSION_ERR_TIMEOUT)) { fail(); break; }
            tc::tc_fence_after();
            const uint32_t sa = a0 + st * kStageBytes;
            // 128-byte-swizzled K-major tiles: 8-row atoms 1 KB apart; MMA j reads K 16 j .. 16 j + 15, 32 bytes
            // into each row (the start-address field counts 16-byte units)
            const uint64_t ad = desc_sw128(sa);
            const uint64_t bd = desc_sw128(sa + bofs);
#pragma unroll
            for (int j = 0; j < kBK / 16; ++j)
                tc::mma_bf16(tbase, ad + (uint64_t)(j * 2), bd + (uint64_t)(j * 2), IDESC, (it > 0 || j > 0) ? 1u : 0u);
            tc::mma_commit(&empty[st]);
        }
        tc::mma_commit(acc_full);
    } else if (warp >= 2) {
        // ---------------- epilogue: lane quarter q = warp & 3, row = output channel ----------------
        const int q = warp & 3;
        const int n = m0 + q * 32 + lane;
        const bool ok = tc::mbar_wait(acc_full, 0, deadline, a.err, FUSION_ERR_TIMEOUT);
        if (!ok) fail();
        tc::tc_fence_after();
        if (ok && !*abort_flag) {
#pragma unroll 1
            for (int cc = 0; cc < kBN / 32; ++cc) {
                uint32_t r[32];
                tc::tmem_ld32(tbase + ((uint32_t)(q * 32) << 16) + cc * 32, r);
                tc::tmem_ld_wait();
                if (n >= a.N) continue;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int b = b0 + cc * 32 + j;
                    if (b < a.B) a.part[((size_t)split * a.B + b) * a.N + n] = __uint_as_float(r[j]);
                }
            }
        }
    }
    // the final commit covers every MMA; wait for it before freeing tensor memory
    if (warp == 1) {
        if (lane == 0 && !tc::mbar_wait(acc_full, 0, deadline)) fail();
        __syncwarp();
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0 && lane == 0) {
        // make sure no copy issued by this CTA is still landing in its shared memory
        const uint64_t dl = tc::globaltimer() + 100000000ull;
        for (int i = 0; i < kStages; ++i) {
            const int cnt = issued > i ? (issued - i + kStages - 1) / kStages : 0;
            if (cnt > 0 && !tc::mbar_wait(&full[i], (cnt - 1) & 1, dl)) atomicOr(a.err, FUSION_ERR_TIMEOUT);
        }
    }
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tbase, kBN);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// [rows][K] bf16 as a 2-D map, box (64 elements, box_rows), 128-byte swizzling.
int encode_kmajor(CUtensorMap *map, const void *base, int rows, int K, int box_rows) {
    auto enc = get_encode();
    if (!enc) return -2;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)r;
}

}  // namespace

struct DenseTcPlan::Impl {
    CUtensorMap tw, tx;
    TcArgs args;
    int splits = 0;
    unsigned gx = 0, gz = 0;
};

DenseTcPlan::DenseTcPlan() : impl(new Impl()) {}
DenseTcPlan::~DenseTcPlan() { delete impl; }

// K per split: about one wave of CTAs for a 64-pose tile, a multiple of the stage K.
static int dense_tc_kper(int K, int N) {
    const int mt = (N + kBM - 1) / kBM;
    int target = 152 / mt;
    if (target < 1) target = 1;
    const int kper = (K + target - 1) / target;
    return (kper + kBK - 1) / kBK * kBK;
}

// Every split s < splits starts below K (s * kper < K), so each one has at least one stage.
int dense_tc_splits(int K, int N) {
    const int kper = dense_tc_kper(K, N);
    return (K + kper - 1) / kper;
}

int dense_tc_plan(DenseTcPlan &plan, const void *x, const void *w, int max_poses, int N, int K, unsigned *err,
                  char *why, size_t why_len) {
    DenseTcPlan::Impl &P = *plan.impl;
    if (K % 8 != 0 || K <= 0 || N <= 0) {
        snprintf(why, why_len, "tensor-core dense needs K a positive multiple of 8");
        return -1;
    }
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(w)) & 15) {
        snprintf(why, why_len, "tensor-core dense needs 16-byte aligned operands");
        return -1;
    }
    int r = encode_kmajor(&P.tw, w, N, K, kBM);
    if (!r) r = encode_kmajor(&P.tx, x, max_poses, K, kBN);
    if (r) {
        snprintf(why, why_len, "cuTensorMapEncodeTiled failed for the dense operands (%d)", r);
        return -2;
    }
    P.args.kper = dense_tc_kper(K, N);
    P.splits = dense_tc_splits(K, N);
    P.args.N = N;
    P.args.K = K;
    P.args.err = err;
    P.gx = (unsigned)((N + kBM - 1) / kBM);
    return 0;
}


void dense_tc_launch(DenseTcPlan &plan, int B, float *part, cudaStream_t s) {
    DenseTcPlan::Impl &P = *plan.impl;
    P.args.B = B;
    P.args.part = part;
    const size_t sm = (size_t)kStages * kStageBytes + (2 * kStages + 1) * 8 + 16;
    cudaFuncSetAttribute(dense_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid(P.gx, P.splits, (unsigned)((B + kBN - 1) / kBN));
    dense_tc_kernel<<<grid, kThreads, sm, s>>>(P.tw, P.tx, P.args);
}

}  // namespace fusion
