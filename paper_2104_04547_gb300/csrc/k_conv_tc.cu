// BF16 and FP8 3D convolution on the tcgen05 tensor cores (Section 3.3.1,
// Table III: the convolutions of the 3D-CNN are the one dense contraction of
// the path).
//
// Implicit GEMM: M = output voxels, N = output channels, K = input channels x
// kernel offsets.  A CTA owns T output slices of 16 x 8 voxels (T M-tiles of
// 128 rows) and all N output channels; the T accumulators (128 lanes x N fp32
// columns each) live in tensor memory.
//
// Operand A comes from an input halo in shared memory: for each 16-channel
// chunk (and, for stride 2, each of the 8 input parity phases) one TMA load
// per 8-channel plane brings the (T + k' - 1) x (16 + k' - 1) x (8 + k' - 1)
// voxel neighbourhood of the tile (zero-filled outside the grid, which is the
// convolution's zero padding; stride-2 phases use the TMA element stride).
// Every kernel offset of the chunk then reads its A operand straight from that
// halo through a shared-memory descriptor whose start address slides by the
// offset (K-major, no swizzle: an 8-row core matrix is one 8-voxel W-line of
// 8 channels, 16 bytes per row, W-lines at a stride of the halo width).  So
// each input element is fetched once per chunk, not once per offset.
//
// Channel-blocked inputs ([pose][z][y][16-byte channel block][x][16 bytes],
// written so by the previous layer or the quantizer for stride-1 layers): the
// chunk's two blocks then come in one TMA box whose rows are whole halo
// W-lines (hw x 16 bytes) instead of single voxels (16 bytes).  A TMA load
// costs about a clock per box row, so a 138 KB halo takes 1.7-2.2 us instead
// of 4.7-4.9 us (measured on all SMs at once), and the tensor pipe waits that
// much less at each chunk.  The halo buffer is then [z][y][K half][x][16 bytes]:
// the descriptor's K-half offset is hw x 16 bytes and its W-line stride 2 hw x 16.
// Parity-split inputs (stride 2, written so by the previous layer or the
// quantizer): the blocked layout of each of the 8 sub-grids of voxels of one
// coordinate parity.  Input voxel 2 o + p - pad of parity phase p is voxel
// o + ((p - pad) >> 1) of sub-grid (p - pad) & 1, so a phase's halo is one
// plain box of whole W-lines of that sub-grid instead of single voxels at the
// TMA element stride of 2, and lands in the same buffer layout.
//
// Operand B (the weights) streams through a ring of shared-memory stages with
// plain bulk copies.  The host arranges them per in-plane offset (ty, tx) as a
// group [8-channel half][tz = nz-1, .., 1, 0][co][16 bytes], so that the rows
// of consecutive entries are W(tz), W(tz - 1), ...
//
// Slice groups: an MMA may serve G adjacent output slices z .. z+G-1 (G = 1, 2
// or 4, G x N <= 256).  Input plane z + u holds, for slice z + s, the offset
// tz = u - s, so one M=128 MMA over that plane with the rows of entries
// nz-1-(u-s_lo) onward (W(u - s_lo), W(u - s_lo - 1), ...) updates slices
// s_lo .. s_hi (those with 0 <= u - s < nz) at once: N = (s_hi - s_lo + 1) x C.
// The A tile is then read from shared memory once for up to G slices.  At
// N = 64 a one-slice MMA reads 6 KB per 32 clocks against a 128 B/clock operand
// path; four slices per MMA read 12 KB per 128 clocks, so the tensor pipe, not
// shared memory, sets the pace.  The work is exactly the useful work (no zero
// weights): planes near the ends of the group feed fewer slices with narrower
// MMAs.  The accumulators are zeroed in tensor memory first and every MMA
// accumulates; slice d sits at columns [dN, dN + N) whatever G is, so the
// epilogue does not depend on it, and every output element receives its terms
// in the same order for every G (offset groups in (ty, tx) order, tz ascending).
//
// Folded first-layer input: the grid's 19 channels fill neither two 16-channel
// chunks (BF16) nor one 32-channel chunk (FP8) well, so the first layer reads a
// grid whose chunks hold some channels at several x positions (the BF16 grid's
// second chunk: channels 16..18 of voxels x-p .. x-p+4; the FP8 grid: channels
// 0..15 of voxels x-1 and x, then 16..18 of voxels x-p .. x+p).  Such a chunk
// is read at a few x-offsets (xt_start + xt_step * t) instead of k, with
// weights arranged to match (conv_tc_arrange_weights, fold modes 1 and 2).
//
// FP8 variant (E4M3 inputs, kind::f8f6f4, 32 channels per MMA): weights carry a
// per-output-channel scale and activations a per-pose scale; the epilogue
// multiplies the FP32 accumulator by both, and records the per-pose maximum
// |output| so the next layer's input can be quantized with its own scale.
//
// Persistent schedule: one CTA per multiprocessor (the tile's shared memory
// allows one); a CTA's first tile is its block index and the producer takes
// each further one from a global counter, passing the index on to the other
// roles through a small ring in shared memory.  Roles: warp 0 lane 0 issues the TMA
// loads, running ahead into the next tile while the current one finishes;
// warp 1 owns tensor memory; lane 0 of warps 1..NI issues the MMAs of its share
// of the slice groups (one issuing thread was measured to limit the MMA rate,
// so several warps issue; each commits its own MMAs and the empty barriers
// count NI arrivals); the remaining 4 x EPW warps run the epilogue (tensor
// memory -> registers, bias, ReLU, residual add, bf16 stores in NDHWC or
// channel-blocked order), EPW per
// tensor-memory lane quarter (a warp reaches only the lanes of quarter
// warp % 4), each holding up to 128 columns of a slice group: two per quarter
// when a group spans 256 columns, so a group is read in one pass.  Each
// epilogue warp reads its columns, zeroes them in tensor memory and hands them
// back on the group's barrier before any arithmetic, so the next tile's MMAs
// into the group wait only for the reads, not for the residual loads and the
// stores.  At the start of a tile the epilogue warps ask L2 for the residual
// input lines they will add, while the tile's MMAs run.  Every wait is
// bounded (re-armed per tile); a wait that runs out sets FUSION_ERR_TIMEOUT and
// the CTA drains and returns.
#include "fusion_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdio>
#include <cstring>

namespace fusion {

namespace {

constexpr int kIssReq = 4;
constexpr int kRing = 4;     // tile indices the producer publishes ahead of the issuers and the epilogue

// Warp roles of one kernel instance: warp 0 loads, warps 1..NI issue MMAs, then 4 x EPW epilogue warps
// (EPW per tensor-memory lane quarter, each holding PART columns of a slice group).
template <int N, int T, int G>
struct Roles {
    static constexpr int UNITS = T / G;                          // slice groups per tile
    static constexpr int NI = kIssReq < UNITS ? kIssReq : UNITS;  // MMA-issuing warps, each owns UNITS / NI
    static constexpr int UCOLS = G * N;                          // accumulator columns of one slice group
    static constexpr int EPW = UCOLS > 128 ? UCOLS / 128 : 1;
    static constexpr int PART = UCOLS / EPW;
    static constexpr int EPI0 = 1 + NI;                           // first epilogue warp
    static constexpr int THREADS = 32 * (EPI0 + 4 * EPW);
};
constexpr uint64_t kWaitNs = 1000000000ull;    // 1 s

struct Geo {
    int nbx, nby, nbz;     // blocks along x (8), y (16), z (T)
    int nphase;            // 1 or 8
    int ntap[2];           // taps per dim for parity 0 / 1 (stride 2), or k (stride 1)
    int hd, hh, hw;        // halo extents
    uint32_t plane_bytes;  // one 8-channel plane of the halo, 128-byte aligned (plain input)
    uint32_t a_bytes;      // one halo buffer (both K halves), 128-byte aligned
    uint32_t lbo_a;        // bytes between the two K halves of a voxel row in the buffer
    int ystep;             // 16-byte rows between consecutive y rows of the buffer
    uint32_t stage_bytes;  // one B stage
    int groups_per_stage;  // (ty, tx) offset groups per B stage
    int nbs;               // B stages
    int na;                // A buffers
    int chunks;            // 16-channel (FP8: 32-channel) chunks of the input
};

struct Args {
    const __nv_bfloat16 *xres;  // bf16 copy of the input [B][n_in]^3[cres] (residual blocks)
    int cres;                   // channels of xres
    const uint8_t *w;           // [chunk][phase][ty][tx][2 halves][tz = nz-1..0][N][16 bytes]
    const float *s_in;          // FP8: per-pose input scale [B]
    const float *s_w;           // FP8: per-output-channel weight scale [N]
    float *amax;                // FP8: per-pose max |output| [B] (atomic max; may be null)
    const float *bias;          // [N]
    __nv_bfloat16 *y;           // [B][n_out]^3[N]
    int n_in, n_out, cin, k, stride, pad, residual;
    int B;                      // poses of this launch (tiles = per-pose tiles x B)
    int stall;                  // test of the bounded waits: the producer issues nothing, so every MMA
                                // issuer's first wait runs out and the launch reports FUSION_ERR_TIMEOUT
    // x-folded input (first layer): chunk c < 2 is read at xt_n[c] x-offsets xt_start[c] + xt_step[c] * t
    // instead of 0 .. k-1, and the input's x coordinate 0 is voxel x_shift of the stored tensor
    int xpat, xt_n[2], xt_step[2], xt_start[2], x_shift;
    int blocked;                // input stored channel-blocked (ConvTcSpec::blocked): one TMA box per chunk
    int out_blocked;            // write y channel-blocked: [pose][z][y][N / 8][x][8]
    int res_blocked;            // xres is channel-blocked: [pose][z][y][cres / 8][x][8]
    Geo g;
    unsigned *err;
    int *tile_counter;          // tiles handed out beyond each CTA's first (zeroed before every launch)
};

__device__ __forceinline__ void phase_taps(const Args &a, int ph, int &pz, int &py, int &px, int &nz, int &ny,
                                           int &nx) {
    if (a.stride == 1) {
        pz = py = px = 0;
        nz = ny = nx = a.k;
    } else {
        pz = (ph >> 2) & 1;
        py = (ph >> 1) & 1;
        px = ph & 1;
        nz = a.g.ntap[pz];
        ny = a.g.ntap[py];
        nx = a.g.ntap[px];
    }
}

template <int N, int T, bool F8, int G>
__global__ void __launch_bounds__(Roles<N, T, G>::THREADS, 1) conv3d_tc_kernel(const __grid_constant__ CUtensorMap tmap, Args a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    static_assert(T % G == 0 && G * N <= 256, "a slice group divides T and spans at most 256 columns");
    constexpr uint32_t TCOLS = (T * N <= 32) ? 32 : (T * N <= 64) ? 64 : (T * N <= 128) ? 128 : (T * N <= 256) ? 256 : 512;
    // instruction descriptor without its N field (bits 17..22 = N / 8, set per MMA)
    constexpr uint32_t IDESC0 = (F8 ? tc::idesc_e4m3(128, 8) : tc::idesc_bf16(128, 8)) & ~(0x3Fu << 17);
    using R = Roles<N, T, G>;
    constexpr int UNITS = R::UNITS, NI = R::NI, UCOLS = R::UCOLS, EPW = R::EPW, PART = R::PART, EPI0 = R::EPI0;
    constexpr int DPI = UNITS / NI;
    constexpr int CPR = F8 ? 16 : 8;      // channels per 16-byte row (one core-matrix column)
    const Geo &g = a.g;
    const uint32_t a_bytes = g.a_bytes;                             // buffer stride
    const uint32_t a_tx = 2u * (uint32_t)(g.hd * g.hh * g.hw) * 16u;  // bytes the two TMA loads deliver
    unsigned char *sA = smem;
    unsigned char *sB = smem + g.na * a_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + g.nbs * g.stage_bytes);
    uint64_t *a_full = bars;            // [2]
    uint64_t *a_empty = bars + 2;       // [2]
    uint64_t *b_full = bars + 4;        // [nbs]
    uint64_t *b_empty = b_full + g.nbs; // [nbs]
    uint64_t *acc_full = b_empty + g.nbs;   // [UNITS]: the tile's MMAs of the group are complete
    uint64_t *acc_empty = acc_full + UNITS; // [UNITS]: the epilogue has read and re-zeroed the group
    uint64_t *mma_done = acc_empty + UNITS;
    uint64_t *tile_full = mma_done + 1;        // [kRing]: ring slot holds the next tile index (or -1: done)
    uint64_t *tile_empty = tile_full + kRing;  // [kRing]: every issuer and epilogue warp has read the slot
    int *tile_ring = reinterpret_cast<int *>(tile_empty + kRing);   // [kRing]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tile_ring + kRing);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = g.nbx * g.nby * g.nbz * a.B;
    auto decode = [&](int t, int &x0, int &y0, int &z0, int &b) {
        x0 = (t % g.nbx) * 8; t /= g.nbx;
        y0 = (t % g.nby) * 16; t /= g.nby;
        z0 = (t % g.nbz) * T;
        b = t / g.nbz;
    };

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) { tc::mbar_init(&a_full[i], 1); tc::mbar_init(&a_empty[i], NI); }
        for (int i = 0; i < g.nbs; ++i) { tc::mbar_init(&b_full[i], 1); tc::mbar_init(&b_empty[i], NI); }
        for (int u = 0; u < UNITS; ++u) { tc::mbar_init(&acc_full[u], 1); tc::mbar_init(&acc_empty[u], 4 * EPW); }
        tc::mbar_init(mma_done, NI);
        for (int i = 0; i < kRing; ++i) { tc::mbar_init(&tile_full[i], 1); tc::mbar_init(&tile_empty[i], NI + 4 * EPW); }
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, TCOLS);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    // the first four epilogue warps (one per tensor-memory lane quarter, warp & 3) zero the accumulators; after
    // that each group is re-zeroed by the epilogue that reads it, so every MMA accumulates
    if (warp >= EPI0 && warp < EPI0 + 4) {
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        for (uint32_t c = 0; c < TCOLS; c += 32u) tc::tmem_st32_zero(tbase + lane_base + c);
        tc::tmem_st_wait();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();

    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(a.err, FUSION_ERR_TIMEOUT);
    };

    // Tiles: a CTA's first is blockIdx.x; the producer takes each further one from a global counter (so a CTA
    // that started late, its SM still busy with another kernel, takes fewer) and publishes every tile index,
    // then -1, through the ring to the issuers and the epilogue.  Every wait's deadline is re-armed per tile.
    int prod_ai = 0, prod_bi = 0;
    if (warp == 0 && lane == 0) {
        // ---------------- producer ----------------
        int &ai = prod_ai, &bi = prod_bi;
        int tile = blockIdx.x;
        for (int k = 0;; ++k) {
            const uint64_t deadline = tc::globaltimer() + kWaitNs;
            const int slot = k % kRing;
            if (!tc::mbar_wait(&tile_empty[slot], ((k / kRing) & 1) ^ 1, deadline, a.err, FUSION_ERR_TIMEOUT)) { fail(); break; }
            const bool done = tile >= n_tiles || *abort_flag;
            tile_ring[slot] = done ? -1 : tile;
            tc::mbar_arrive(&tile_full[slot]);           // release: the ring entry is visible to the waiters
            if (done || a.stall) break;                  // stall test: publish the first tile, load nothing
            int x0, y0, z0, b;
            decode(tile, x0, y0, z0, b);
            const uint8_t *wc = a.w;     // weights are consumed in storage order: chunk, phase, (ty, tx) group
            for (int c = 0; c < g.chunks && !*abort_flag; ++c) {
                for (int ph = 0; ph < g.nphase && !*abort_flag; ++ph) {
                    int pz, py, px, nz, ny, nx;
                    phase_taps(a, ph, pz, py, px, nz, ny, nx);
                    const int buf = ai % g.na;
                    if (!tc::mbar_wait(&a_empty[buf], ((ai / g.na) & 1) ^ 1, deadline, a.err, FUSION_ERR_TIMEOUT)) { fail(); break; }
                    tc::mbar_expect_tx(&a_full[buf], a_tx);
                    const int S = a.stride;
                    if (a.blocked == 2) {
                        // parity-split input: input coordinate 2 o + p - pad = 2 (o + (p - pad) >> 1) + ((p - pad) & 1),
                        // so the phase's halo is one plain box of the parity sub-grid (p - pad) & 1 per dimension,
                        // starting (p - pad) >> 1 voxels from the tile (arithmetic shift: rounds down)
                        const int qx = px - a.pad, qy = py - a.pad, qz = pz - a.pad;
                        tc::tma_load_5d(sA + buf * a_bytes, &tmap, &a_full[buf], (x0 + (qx >> 1)) * CPR, 2 * c,
                                        y0 + (qy >> 1), z0 + (qz >> 1), b * 8 + (qz & 1) * 4 + (qy & 1) * 2 + (qx & 1));
                    } else if (a.blocked) {
                        // buffer [z][y][K half][x][16 bytes]: the chunk's two 16-byte channel blocks in one box
                        tc::tma_load_5d(sA + buf * a_bytes, &tmap, &a_full[buf], (x0 - a.pad + a.x_shift) * CPR, 2 * c,
                                        y0 - a.pad, z0 - a.pad, b);
                    } else {
                        // buffer [K half][z][y][x][16 bytes]: one box per 16-byte channel block
                        for (int j = 0; j < 2; ++j)
                            tc::tma_load_5d(sA + buf * a_bytes + j * g.plane_bytes, &tmap, &a_full[buf], c * 2 * CPR + j * CPR,
                                            x0 * S + px - a.pad + a.x_shift, y0 * S + py - a.pad, z0 * S + pz - a.pad, b);
                    }
                    ++ai;
                    if (a.xpat) nx = a.xt_n[c];
                    const int ngr = nz > 0 ? ny * nx : 0;   // a phase without z taps adds nothing
                    const uint32_t gbytes = (uint32_t)nz * N * 32;
                    for (int g0 = 0; g0 < ngr; g0 += g.groups_per_stage) {
                        const int cnt = min(g.groups_per_stage, ngr - g0);
                        const int st = bi % g.nbs;
                        if (!tc::mbar_wait(&b_empty[st], ((bi / g.nbs) & 1) ^ 1, deadline, a.err, FUSION_ERR_TIMEOUT)) { fail(); break; }
                        const uint32_t bytes = (uint32_t)cnt * gbytes;
                        tc::mbar_expect_tx(&b_full[st], bytes);
                        tc::bulk_load(sB + st * g.stage_bytes, wc + (size_t)g0 * gbytes, bytes, &b_full[st]);
                        ++bi;
                    }
                    wc += (size_t)ngr * gbytes;
                }
            }
            tile = atomicAdd(a.tile_counter, 1) + (int)gridDim.x;
        }
    } else if (warp >= 1 && warp <= NI && lane == 0) {
        const int d0 = (warp - 1) * DPI;
        // ---------------- MMA issuer ----------------
        int ai = 0, bi = 0;
        const uint32_t sbo_a = (uint32_t)g.ystep * 16;
        const uint32_t row_zy = (uint32_t)g.hh * g.ystep;
        for (int it = 0;; ++it) {
            const uint64_t deadline = tc::globaltimer() + kWaitNs;
            const int slot = it % kRing;
            if (!tc::mbar_wait(&tile_full[slot], (it / kRing) & 1, deadline, a.err, FUSION_ERR_TIMEOUT)) { fail(); break; }
            const int tile = tile_ring[slot];
            tc::mbar_arrive(&tile_empty[slot]);
            if (tile < 0 || *abort_flag) break;
            // this warp's slice groups must have been read (and re-zeroed) by the previous tile's epilogue
            bool ok = true;
            for (int dd = 0; dd < DPI && ok; ++dd)
                ok = tc::mbar_wait(&acc_empty[d0 + dd], (it & 1) ^ 1, deadline, a.err, FUSION_ERR_TIMEOUT);
            if (!ok) { fail(); break; }
            tc::tc_fence_after();
            for (int c = 0; c < g.chunks && !*abort_flag; ++c) {
                for (int ph = 0; ph < g.nphase && !*abort_flag; ++ph) {
                    int pz, py, px, nz, ny, nx;
                    phase_taps(a, ph, pz, py, px, nz, ny, nx);
                    const int buf = ai % g.na;
                    if (!tc::mbar_wait(&a_full[buf], (ai / g.na) & 1, deadline, a.err, FUSION_ERR_TIMEOUT)) { fail(); break; }
                    // descriptors advance by plain integer adds: the start-address field counts 16-byte rows
                    const uint64_t adesc0 = tc::desc_kmajor(tc::smem_u32(sA + buf * a_bytes), g.lbo_a, sbo_a);
                    const uint32_t lbo_b = (uint32_t)nz * N * 16;    // between the two 8-channel halves
                    // an x-folded chunk reads its few x-offsets at halo columns xt_start + xt_step * tx
                    int xstep = 1, xstart = 0;
                    if (a.xpat) {
                        nx = a.xt_n[c];
                        xstep = a.xt_step[c];
                        xstart = a.xt_start[c];
                    }
                    const int ngr = nz > 0 ? ny * nx : 0;   // a phase without z taps adds nothing
                    for (int g0 = 0; g0 < ngr; g0 += g.groups_per_stage) {
                        const int gend = min(g0 + g.groups_per_stage, ngr);
                        const int st = bi % g.nbs;
                        if (!tc::mbar_wait(&b_full[st], (bi / g.nbs) & 1, deadline, a.err, FUSION_ERR_TIMEOUT)) { fail(); break; }
                        tc::tc_fence_after();
                        uint64_t bgrp = tc::desc_kmajor(tc::smem_u32(sB + st * g.stage_bytes), lbo_b, 128);
                        for (int gi = g0; gi < gend; ++gi) {
                            const int ty = gi / nx, tx = gi - (gi / nx) * nx;
                            const int hx = xstart + xstep * tx;
                            const uint64_t arow = adesc0 + (uint64_t)(ty * g.ystep + hx);
                            // plane u of slice group j feeds its slices s_lo..s_hi (offset tz = u - s) in one MMA
                            for (int u = 0; u <= nz + G - 2; ++u) {
                                const int s_lo = u - (nz - 1) > 0 ? u - (nz - 1) : 0;
                                const int s_hi = u < G - 1 ? u : G - 1;
                                const uint32_t idesc = IDESC0 | ((uint32_t)((s_hi - s_lo + 1) * N) >> 3) << 17;
                                const uint64_t bd = bgrp + (uint64_t)((nz - 1 - (u - s_lo)) * N);
#pragma unroll
                                for (int dd = 0; dd < DPI; ++dd) {
                                    const int j = d0 + dd;
                                    const uint64_t ad = arow + (uint64_t)((G * j + u) * row_zy);
                                    const uint32_t dt = tbase + (uint32_t)((G * j + s_lo) * N);
                                    if constexpr (F8) tc::mma_e4m3(dt, ad, bd, idesc, 1u);
                                    else tc::mma_bf16(dt, ad, bd, idesc, 1u);
                                }
                            }
                            bgrp += (uint64_t)(nz * N * 2);   // next group: nz * N * 32 bytes
                        }
                        tc::mma_commit(&b_empty[st]);
                        ++bi;
                    }
                    tc::mma_commit(&a_empty[buf]);
                    ++ai;
                }
            }
            for (int dd = 0; dd < DPI; ++dd) tc::mma_commit(&acc_full[d0 + dd]);
        }
        tc::mma_commit(mma_done);
    } else if (warp >= EPI0) {
        // ---------------- epilogue: EPW warps per tensor-memory lane quarter ----------------
        const int q = warp & 3;                 // lane quarter
        const int half = (warp - EPI0) >> 2;    // which PART columns of a slice group this warp holds
        const int r = q * 32 + lane;            // M row = voxel of the slice
        const int h = r >> 3, w = r & 7;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        for (int it = 0;; ++it) {
            const uint64_t deadline = tc::globaltimer() + kWaitNs;
            // lane 0 takes the tile index from the ring; the warp follows its answer
            const int slot = it % kRing;
            int tile = -1;
            if (lane == 0) {
                if (tc::mbar_wait(&tile_full[slot], (it / kRing) & 1, deadline, a.err, FUSION_ERR_TIMEOUT)) {
                    tile = tile_ring[slot];
                    tc::mbar_arrive(&tile_empty[slot]);
                } else {
                    fail();
                }
            }
            tile = __shfl_sync(0xffffffffu, tile, 0);
            if (tile < 0 || __any_sync(0xffffffffu, *abort_flag != 0)) break;
            int x0, y0, z0, b;
            decode(tile, x0, y0, z0, b);
            const int yy = y0 + h, xx = x0 + w;
            const float sx = F8 ? a.s_in[b] : 1.f;
            // element offset of channel c of this thread's voxel in slice zz, NDHWC or channel-blocked
            // Both layouts are affine in (slice zz, channel c, c a multiple of 8) for this thread's voxel:
            //   NDHWC    ((b n + zz) n + yy) n + xx) C + c
            //   blocked  ((((b n + zz) n + yy) C/8 + c/8) n + xx) 8
            //   = b n^3 C + zz n^2 C + yy n C + (blocked ? xx 8 + c n : xx C + c)
            // The parity-split output (out_blocked 2, read by a stride-2 layer) is the blocked layout of each of
            // the 8 parity sub-grids of half the size, [pose][(z&1) 4 + (y&1) 2 + (x&1)][z/2][y/2][C/8][x/2][8]:
            //   b n^3 C + ((y&1) 2 + (x&1)) h^3 C + (y/2) h C + (x/2) 8 + c h  +  (z&1) 4 h^3 C + (z/2) h^2 C
            const int n = a.n_out;
            const bool split = a.out_blocked == 2;
            const int hn = n >> 1;
            const size_t hcube = (size_t)hn * hn * hn * N;
            const size_t zstep_y = split ? (size_t)hn * hn * N : (size_t)n * n * N, zstep_r = (size_t)n * n * a.cres;
            const size_t zpar_y = 4 * hcube;    // parity-split: the odd slices' sub-grids
            const size_t ybase = split ? (size_t)b * n * n * n * N + (size_t)((yy & 1) * 2 + (xx & 1)) * hcube +
                                             (size_t)(yy >> 1) * hn * N + (size_t)(xx >> 1) * 8
                                       : (size_t)b * n * zstep_y + (size_t)yy * n * N + (a.out_blocked ? xx * 8 : xx * N);
            const size_t rbase = (size_t)b * n * zstep_r + (size_t)yy * n * a.cres + (a.res_blocked ? xx * 8 : xx * a.cres);
            const int ycc = split ? hn : a.out_blocked ? n : 1, rcc = a.res_blocked ? n : 1;   // per channel
            if (a.residual && yy < a.n_out && xx < a.n_out) {
                // ask L2 for the residual input this tile's stores will add, while its MMAs run (one line per
                // voxel row of a 16-byte block when blocked, taken by the lane at the row's first voxel)
#pragma unroll 1
                for (int u = 0; u < UNITS; ++u)
#pragma unroll 1
                    for (int c32 = 0; c32 < PART / 32; ++c32) {
                        const int col = u * UCOLS + half * PART + c32 * 32;
                        const int zz = z0 + col / N, cc = col % N;
                        if (zz >= a.n_out) continue;
                        const __nv_bfloat16 *r0 = a.xres + rbase + zz * zstep_r + (size_t)cc * rcc;
                        if (!a.res_blocked) tc::prefetch_line_l2(r0);
                        else if (w == 0)
                            for (int k4 = 0; k4 < 4; ++k4) tc::prefetch_line_l2(r0 + (size_t)k4 * 8 * n);
                    }
            }
            float vmax = 0.f;
            bool ok = true;
            for (int u = 0; u < UNITS && ok; ++u) {
                // every lane waits (each acquires), and the warp goes on only if all succeeded and nobody gave up:
                // the tensor-memory loads below must be executed by all 32 lanes or by none
                ok = tc::mbar_wait(&acc_full[u], it & 1, deadline, a.err, FUSION_ERR_TIMEOUT);
                ok = __all_sync(0xffffffffu, ok) && !__any_sync(0xffffffffu, *abort_flag != 0);
                if (!ok) { if (lane == 0) fail(); break; }
                tc::tc_fence_after();
                // read this warp's columns of the group, zero them for the next tile and hand them back
                // before any arithmetic, so the next tile's MMAs into the group wait only for the reads
                const int col0 = u * UCOLS + half * PART;
                uint32_t acc[PART / 32][32];
#pragma unroll
                for (int c32 = 0; c32 < PART / 32; ++c32)
                    tc::tmem_ld32(tbase + lane_base + (uint32_t)(col0 + c32 * 32), acc[c32]);
                tc::tmem_ld_wait();
#pragma unroll
                for (int c32 = 0; c32 < PART / 32; ++c32) tc::tmem_st32_zero(tbase + lane_base + (uint32_t)(col0 + c32 * 32));
                tc::tmem_st_wait();
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&acc_empty[u]);
#pragma unroll
                for (int c32 = 0; c32 < PART / 32; ++c32) {
                    const int col = col0 + c32 * 32;     // slice d = col / N, channels col % N ..
                    const int d = col / N, cc = col % N;
                    const int zz = z0 + d;
                    if (zz >= a.n_out || yy >= a.n_out || xx >= a.n_out) continue;
                    uint32_t *v = acc[c32];      // the arithmetic happens in place (float bits)
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float t = __uint_as_float(v[j]);
                        if constexpr (F8) t *= sx * a.s_w[cc + j];
                        v[j] = __float_as_uint(fmaxf(t + a.bias[cc + j], 0.f));
                    }
                    if (a.residual) {
                        // the input is read-only for the whole launch (the output is another buffer)
                        // 8-channel blocks k4 = 0..3: contiguous (NDHWC) or n_out voxels apart (blocked)
                        const __nv_bfloat16 *rsrc = a.xres + rbase + zz * zstep_r + (size_t)cc * rcc;
                        const int rstep = 8 * rcc;
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4) {
                            const uint4 t4 = __ldg(reinterpret_cast<const uint4 *>(rsrc + k4 * rstep));
                            const __nv_bfloat162 *hp = reinterpret_cast<const __nv_bfloat162 *>(&t4);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float2 f = __bfloat1622float2(hp[e]);
                                v[k4 * 8 + 2 * e] = __float_as_uint(__uint_as_float(v[k4 * 8 + 2 * e]) + f.x);
                                v[k4 * 8 + 2 * e + 1] = __float_as_uint(__uint_as_float(v[k4 * 8 + 2 * e + 1]) + f.y);
                            }
                        }
                    }
                    const size_t zoff = split ? (size_t)(zz & 1) * zpar_y + (size_t)(zz >> 1) * zstep_y : zz * zstep_y;
                    __nv_bfloat16 *const ydst = a.y + ybase + zoff + (size_t)cc * ycc;
                    const int ystep = 8 * ycc;
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        uint4 t4;
                        __nv_bfloat162 *hp = reinterpret_cast<__nv_bfloat162 *>(&t4);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            hp[e] = __floats2bfloat162_rn(__uint_as_float(v[k4 * 8 + 2 * e]),
                                                          __uint_as_float(v[k4 * 8 + 2 * e + 1]));
                            if constexpr (F8) {
                                const float2 rr = __bfloat1622float2(hp[e]);
                                vmax = fmaxf(vmax, fmaxf(fabsf(rr.x), fabsf(rr.y)));
                            }
                        }
                        *reinterpret_cast<uint4 *>(ydst + k4 * ystep) = t4;
                    }
                }
            }
            if constexpr (F8) {
                for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
                if (lane == 0 && a.amax && vmax > 0.f)
                    atomicMax(reinterpret_cast<unsigned *>(a.amax + b), __float_as_uint(vmax));
            }
            if (!ok) break;
        }
    }
    // every MMA must be complete before tensor memory is freed: each issuer's last commit covers its MMAs
    if (warp == 1) {
        if (lane == 0 && !tc::mbar_wait(mma_done, 0, tc::globaltimer() + kWaitNs)) fail();
        __syncwarp();
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0 && lane == 0) {
        // make sure no copy issued by this CTA is still landing in its shared memory
        const uint64_t dl = tc::globaltimer() + 100000000ull;
        for (int i = 0; i < g.na; ++i) {
            const int n = prod_ai > i ? (prod_ai - i + g.na - 1) / g.na : 0;
            if (n > 0 && !tc::mbar_wait(&a_full[i], (n - 1) & 1, dl)) atomicOr(a.err, FUSION_ERR_TIMEOUT);
        }
        for (int i = 0; i < g.nbs; ++i) {
            const int n = prod_bi > i ? (prod_bi - i + g.nbs - 1) / g.nbs : 0;
            if (n > 0 && !tc::mbar_wait(&b_full[i], (n - 1) & 1, dl)) atomicOr(a.err, FUSION_ERR_TIMEOUT);
        }
    }
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tbase, TCOLS);
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

}  // namespace

struct ConvTcPlan::Impl {
    CUtensorMap tmap;
    Args args;
    int *counter = nullptr;     // device: the launch's tile counter
    ~Impl() { if (counter) cudaFree(counter); }
    int N = 0, T = 0;
    bool f8 = false;
    int group = 1;          // output slices per MMA
    int sms = 1;            // multiprocessors of the device (persistent grid size)
    size_t smem = 0;
    unsigned grid = 0;
};

ConvTcPlan::ConvTcPlan() : impl(new Impl()) {}
ConvTcPlan::~ConvTcPlan() { delete impl; }

int conv_tc_tile_slices(int c_out) { return c_out >= 256 ? 2 : c_out >= 128 ? 4 : 8; }

// 32-output-channel layers can take 16 slices per CTA (16 x 32 = 512 tensor-memory columns) and serve 8 of
// them per MMA (N = 256, the width that keeps the MMA above the operand path's rate) with two slice groups,
// hence two issuers.  Chosen by default where the halo fits and the z extent wastes no more slices than 8
// per CTA would.
static bool wide_tiles_ok(int c_out, int n_out) {
    const int w16 = (n_out + 15) / 16 * 16, w8 = (n_out + 7) / 8 * 8;
    return c_out <= 32 && w16 <= w8;
}

// Taps per dimension of parity phase ph: k at stride 1; (k + 1) / 2 and k / 2 for parities 0 / 1 at stride 2.
static void phase_ntaps(int k, int stride, int ph, int &nz, int &ny, int &nx) {
    if (stride == 1) {
        nz = ny = nx = k;
        return;
    }
    const int n[2] = {(k + 1) / 2, k / 2};
    nz = n[(ph >> 2) & 1];
    ny = n[(ph >> 1) & 1];
    nx = n[ph & 1];
}

// Arranged bytes of one channel chunk: every phase's (ty, tx) groups of nz x 2 x c_out 16-byte rows.
static size_t chunk_weight_bytes(int c_out, int k, int stride) {
    size_t rows = 0;
    for (int ph = 0; ph < (stride == 1 ? 1 : 8); ++ph) {
        int nz, ny, nx;
        phase_ntaps(k, stride, ph, nz, ny, nx);
        rows += (size_t)ny * nx * nz * 2 * c_out;
    }
    return rows * 16;
}

// x-folded first-layer inputs (3 channels beyond the first 16; see VoxArgs::fold_pad and
// launch_quantize_fold_fp8).  Mode 1 (bf16, two 16-channel chunks): chunk 0 plain; chunk 1 holds
// channels 16..18 of voxels x-p .. x-p+4 and is read at halo columns p and p + 2 (kernel columns 0..4
// and, for k = 7, 5..6 from slots 3, 4).  Mode 2 (FP8, two 32-channel chunks, stored from x = -1):
// chunk 0 holds channels 0..15 of voxels x-1 and x and is read at halo columns 0, 2, 4, .. (kernel
// columns 2t, 2t+1); chunk 1 holds channels 16..18 of voxels x-p .. x+p and is read at column p.
static int fold_nx(int k) { return k <= 5 ? 1 : 2; }

bool conv_tc_fold_ok(int c_in, int cin_pad, int k, int stride, int elem) {
    return stride == 1 && (k == 3 || k == 5 || k == 7) && c_in == 19 && cin_pad == 32 && (elem == 1 || elem == 2);
}

static void fold_pattern(int mode, int k, int n[2], int step[2], int start[2]) {
    const int p = k / 2;
    if (mode == 1) {
        n[0] = k; step[0] = 1; start[0] = 0;
        n[1] = fold_nx(k); step[1] = 2; start[1] = p;
    } else {
        n[0] = (k + 1) / 2; step[0] = 2; start[0] = 0;
        n[1] = 1; step[1] = 1; start[1] = p;
    }
}

size_t conv_tc_weight_bytes(int cin_pad, int c_out, int k, int stride, int elem, int fold) {
    const int chunk_bytes_in = 32;                         // one chunk = 32 bytes of channels per voxel
    const int chunks = cin_pad * elem / chunk_bytes_in;
    if (!fold) return (size_t)chunks * chunk_weight_bytes(c_out, k, stride);
    int n[2], st[2], s0[2];
    fold_pattern(fold, k, n, st, s0);
    return (size_t)k * (n[0] + n[1]) * k * 2 * c_out * 16;
}

// float -> E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; largest finite 448, no
// infinities), round to nearest even, saturating to +-448.
static uint8_t e4m3_from_float(float x) {
    const uint8_t sign = (x < 0.f) ? 0x80 : 0x00;
    double a = std::fabs((double)x);
    if (!(a > 0.0)) return sign;
    if (a >= 448.0) return sign | 0x7E;
    int e;
    std::frexp(a, &e);                     // a = f * 2^e, f in [0.5, 1)
    int E = e - 1;                         // a in [2^E, 2^(E+1))
    if (E < -6) E = -6;                    // subnormal range shares the 2^-9 quantum
    const double quantum = std::ldexp(1.0, E - 3);
    double r = std::nearbyint(a / quantum) * quantum;   // default rounding mode: ties to even
    if (r > 448.0) r = 448.0;
    if (r == 0.0) return sign;
    if (r < std::ldexp(1.0, -6)) {         // subnormal: mantissa m in 1..7, value m * 2^-9
        const int m = (int)std::lround(r / std::ldexp(1.0, -9));
        return sign | (uint8_t)m;
    }
    int er;
    std::frexp(r, &er);
    const int Er = er - 1;
    const int m = (int)std::lround((r / std::ldexp(1.0, Er) - 1.0) * 8.0);
    return sign | (uint8_t)(((Er + 7) << 3) | m);
}

static uint16_t bf16_from_float(float v) {
    uint32_t u;
    memcpy(&u, &v, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);       // round to nearest even
    return (uint16_t)(u >> 16);
}

void conv_tc_arrange_weights(const float *w, int c_out, int c_in, int cin_pad, int k, int stride, int elem,
                             int fold, uint8_t *out, float *s_w) {
    // blob layout w[co][ci][kd][kh][kw] ->
    //   [chunk][phase][ty][tx][8/16-channel half][tz = nz-1 .. 0][co][16 bytes]
    const int cpr = elem == 2 ? 8 : 16;                // channels per 16-byte row
    const int nph = stride == 1 ? 1 : 8;
    const int k3 = k * k * k;
    if (elem == 1) {
        for (int co = 0; co < c_out; ++co) {
            float mx = 0.f;
            for (int q = 0; q < c_in * k3; ++q) mx = std::fmax(mx, std::fabs(w[(size_t)co * c_in * k3 + q]));
            s_w[co] = mx > 0.f ? mx / 448.f : 1.f;
        }
    }
    size_t idx = 0;
    auto put = [&](float v, int co) {
        if (elem == 2) {
            const uint16_t h = bf16_from_float(v);
            memcpy(out + idx, &h, 2);
            idx += 2;
        } else {
            out[idx++] = e4m3_from_float(v / s_w[co]);
        }
    };
    if (fold) {
        // folded first-layer input: two chunks of 2 x cpr slots; slot q of chunk c at x-offset t reads
        // channel ch and kernel column kw, or nothing
        int nt[2], st[2], s0[2];
        fold_pattern(fold, k, nt, st, s0);
        for (int c = 0; c < 2; ++c)
            for (int ty = 0; ty < k; ++ty)
                for (int t = 0; t < nt[c]; ++t)
                    for (int half = 0; half < 2; ++half)
                        for (int e = 0; e < k; ++e) {
                            const int tz = k - 1 - e;
                            for (int co = 0; co < c_out; ++co)
                                for (int el = 0; el < cpr; ++el) {
                                    const int q = half * cpr + el;
                                    int ch = -1, kw = -1;
                                    if (fold == 1 && c == 0) { ch = q; kw = t; }
                                    else if (fold == 1) {
                                        const int sl = q / 3;
                                        if (q < 15 && (t == 0 ? sl < 5 : sl >= 3)) { ch = 16 + q % 3; kw = 2 * t + sl; }
                                    } else if (c == 0) { ch = el; kw = 2 * t + half; }
                                    else if (q < 3 * k) { ch = 16 + q % 3; kw = q / 3; }
                                    const bool used = ch >= 0 && ch < c_in && kw >= 0 && kw < k;
                                    put(used ? w[((((size_t)co * c_in + ch) * k + tz) * k + ty) * k + kw] : 0.f, co);
                                }
                        }
        return;
    }
    for (int c = 0; c < cin_pad / (2 * cpr); ++c) {
        for (int ph = 0; ph < nph; ++ph) {
            const int pz = stride == 1 ? 0 : (ph >> 2) & 1, py = stride == 1 ? 0 : (ph >> 1) & 1,
                      px = stride == 1 ? 0 : ph & 1;
            int nz, ny, nx;
            phase_ntaps(k, stride, ph, nz, ny, nx);
            for (int ty = 0; ty < ny; ++ty)
                for (int tx = 0; tx < nx; ++tx)
                    for (int half = 0; half < 2; ++half)
                        for (int e = 0; e < nz; ++e) {
                            const int tz = nz - 1 - e;
                            const int kd = pz + stride * tz, kh = py + stride * ty, kw = px + stride * tx;
                            for (int co = 0; co < c_out; ++co)
                                for (int el = 0; el < cpr; ++el) {
                                    const int ci = c * 2 * cpr + half * cpr + el;
                                    float v = 0.f;
                                    if (ci < c_in) v = w[((((size_t)co * c_in + ci) * k + kd) * k + kh) * k + kw];
                                    if (elem == 2) {
                                        const uint16_t h = bf16_from_float(v);
                                        memcpy(out + idx, &h, 2);
                                        idx += 2;
                                    } else {
                                        out[idx++] = e4m3_from_float(v / s_w[co]);
                                    }
                                }
                        }
        }
    }
}

int conv_tc_plan(ConvTcPlan &plan, const ConvTcSpec &sp, char *why, size_t why_len) {
    ConvTcPlan::Impl &P = *plan.impl;
    const int c_out = sp.c_out, k = sp.k, stride = sp.stride;
    if (sp.T <= 0 && stride == 1 && wide_tiles_ok(c_out, sp.n_out)) {
        ConvTcSpec wide = sp;
        wide.T = 16;
        if (conv_tc_plan(plan, wide, why, why_len) == 0) return 0;   // else the default below
    }
    const int T = sp.T > 0 ? sp.T : conv_tc_tile_slices(c_out);
    const int chunk_ch = sp.elem == 2 ? 16 : 32;
    // 16 slices per CTA only at stride 1 (the strided phases are built and checked for at most 8)
    const bool t_ok = (c_out <= 64 && (T == 4 || T == 8)) || (c_out <= 32 && T == 16 && stride == 1) ||
                      (c_out == 128 && (T == 2 || T == 4)) ||
                      (c_out == 256 && T == 2);
    if (!t_ok) {
        snprintf(why, why_len, "unsupported output slices per CTA (%d) for %d output channels at stride %d", T, c_out,
                 stride);
        return -1;
    }
    if (c_out != 32 && c_out != 64 && c_out != 128 && c_out != 256) {
        snprintf(why, why_len, "tensor-core conv needs c_out in {32, 64, 128, 256}");
        return -1;
    }
    if (sp.cin_pad % chunk_ch != 0 || (stride != 1 && stride != 2) || (sp.elem != 1 && sp.elem != 2)) {
        snprintf(why, why_len, "tensor-core conv needs input channels padded to %d and stride 1 or 2", chunk_ch);
        return -1;
    }
    if (sp.fold && (sp.residual || !conv_tc_fold_ok(19, 32, k, stride, sp.elem) ||
                    (sp.fold == 1 && (sp.elem != 2 || sp.cin_pad != 32)) ||
                    (sp.fold == 2 && (sp.elem != 1 || sp.cin_pad != 64)) || sp.fold > 2)) {
        snprintf(why, why_len, "an x-folded input needs 19 channels, stride 1, k in {3, 5, 7}, no residual, and "
                 "32 bf16 (mode 1) or 64 FP8 (mode 2) stored channels");
        return -1;
    }
    Geo g{};
    g.nbx = (sp.n_out + 7) / 8;
    g.nby = (sp.n_out + 15) / 16;
    g.nbz = (sp.n_out + T - 1) / T;
    g.nphase = stride == 1 ? 1 : 8;
    g.ntap[0] = stride == 1 ? k : (k + 1) / 2;
    g.ntap[1] = stride == 1 ? k : k / 2;
    const int ntmax = g.ntap[0];
    g.hd = T + ntmax - 1;
    g.hh = 16 + ntmax - 1;
    g.hw = 8 + ntmax - 1;
    if ((sp.blocked == 1 && stride != 1) || (sp.blocked == 2 && (stride != 2 || sp.n_in % 2 != 0 || sp.fold)) ||
        sp.blocked < 0 || sp.blocked > 2) {
        snprintf(why, why_len, "a channel-blocked input needs stride 1, a parity-split one stride 2 and an even size");
        return -1;
    }
    if (sp.out_blocked < 0 || sp.out_blocked > 2 || (sp.out_blocked == 2 && sp.n_out % 2 != 0)) {
        snprintf(why, why_len, "a parity-split output needs an even size");
        return -1;
    }
    g.plane_bytes = ((uint32_t)(g.hd * g.hh * g.hw) * 16 + 127) / 128 * 128;
    if (sp.blocked) {
        // [z][y][K half][x][16 bytes]: K halves hw rows apart, y rows 2 hw apart
        g.a_bytes = ((uint32_t)(g.hd * g.hh * g.hw) * 32 + 127) / 128 * 128;
        g.lbo_a = (uint32_t)g.hw * 16;
        g.ystep = 2 * g.hw;
    } else {
        // [K half][z][y][x][16 bytes]
        g.a_bytes = 2 * g.plane_bytes;
        g.lbo_a = g.plane_bytes;
        g.ystep = g.hw;
    }
    // about 48 KB of weights per stage in a ring of two: each stage hand-off costs a fixed few
    // hundred cycles, and fewer, larger stages measured faster than deeper rings of smaller ones
    const uint32_t gbytes_max = (uint32_t)ntmax * c_out * 32;
    // stride 2: about 72 KB per stage, at most one parity phase's groups (a stage never spans phases).  Its
    // small halos leave the room, and fewer weight copies per phase measured faster (full-size conv3, 64
    // poses: 1.47 -> 1.39-1.40 ms BF16, 1.04 -> 1.00-1.01 ms FP8 with 6 groups instead of 4)
    const uint32_t stage_target = stride == 2 ? 73728u : 49152u;
    g.groups_per_stage = sp.groups_per_stage > 0 ? sp.groups_per_stage : (int)(stage_target / gbytes_max);
    if (sp.groups_per_stage <= 0 && stride == 2 && g.groups_per_stage > ntmax * ntmax) g.groups_per_stage = ntmax * ntmax;
    if (g.groups_per_stage < 1) g.groups_per_stage = 1;
    g.stage_bytes = ((uint32_t)g.groups_per_stage * gbytes_max + 127) / 128 * 128;
    // output slices per MMA: by default the most (4, else 2) that fit, for stride 1.  Measured on the
    // 64-channel layers (64 poses, BF16, persistent kernel): 2 slices 10.4-10.5 ms, 4 slices 10.1-10.3 ms per
    // residual layer.  (Before the epilogue had warps of its own, 4 lost to 2: one thread issues an MMA
    // about every 80-100 clocks, and 4 slices per MMA leave two accumulator sets, hence two issuers, whose
    // warps also ran the epilogue.)  At stride 2 each phase has only 2-3 z offsets, so a slice group
    // shares little: 1.
    auto group_ok = [&](int G) {
        return (G == 1 || G == 2 || G == 4 || G == 8) && T % G == 0 && G * c_out <= 256 && T / G >= (G == 8 ? 2 : 1);
    };
    int group = sp.group;
    if (group <= 0) group = stride != 1 ? 1 : (T == 16 && group_ok(8)) ? 8 : group_ok(4) ? 4 : group_ok(2) ? 2 : 1;
    if (!group_ok(group)) {
        snprintf(why, why_len, "%d slices per MMA: must be 1, 2, 4 or 8 (8: with 16 slices per CTA), divide the %d "
                 "slices per CTA and span <= 256 columns", group, T);
        return -1;
    }
    g.nbs = sp.nbs > 0 ? sp.nbs : 2;
    if (g.nbs < 2 || g.nbs > 8) {
        snprintf(why, why_len, "weight stages must be in [2, 8]");
        return -1;
    }
    g.chunks = sp.cin_pad / chunk_ch;
    // a_full/a_empty [2] each, b_full/b_empty [nbs] each, acc_full/acc_empty [T / group] each, mma_done,
    // tile_full/tile_empty [kRing] each, the tile ring, then the tensor-memory slot and the abort flag
    const size_t bar_bytes = (size_t)(4 + 2 * g.nbs + 2 * (T / group) + 1 + 2 * kRing) * 8 + kRing * 4 + 16;
    const size_t limit = 227 * 1024;
    const size_t a1 = g.a_bytes;
    // a larger halo (16 slices per CTA) leaves less room for weights: shrink the default stages to fit
    while (sp.groups_per_stage <= 0 && g.groups_per_stage > 1 &&
           a1 + (size_t)g.nbs * g.stage_bytes + bar_bytes > limit) {
        --g.groups_per_stage;
        g.stage_bytes = ((uint32_t)g.groups_per_stage * gbytes_max + 127) / 128 * 128;
    }
    const size_t b_total = (size_t)g.nbs * g.stage_bytes;
    g.na = (2 * a1 + b_total + bar_bytes <= limit) ? 2 : 1;
    P.smem = g.na * a1 + b_total + bar_bytes;
    if (P.smem > limit) {
        snprintf(why, why_len, "tensor-core conv tile needs %zu bytes of shared memory", P.smem);
        return -1;
    }
    if (g.hw * stride > 256 || g.hh * stride > 256 || g.hd * stride > 256 || (sp.blocked && g.hw * 16 / sp.elem > 256)) {
        snprintf(why, why_len, "halo box too large for a TMA load");
        return -1;
    }
    auto enc = get_encode();
    if (!enc) {
        snprintf(why, why_len, "cuTensorMapEncodeTiled is not available");
        return -2;
    }
    const cuuint64_t rowb = (cuuint64_t)sp.cin_pad * sp.elem;   // bytes per voxel
    const cuuint64_t n = (cuuint64_t)sp.n_in;
    const cuuint64_t nx_in = n + (sp.fold == 2 ? 1 : 0);          // FP8-folded input is stored from x = -1
    const cuuint64_t cpr = (cuuint64_t)(16 / sp.elem);              // elements per 16-byte channel block
    cuuint64_t dims[5] = {(cuuint64_t)sp.cin_pad, nx_in, n, n, (cuuint64_t)sp.max_poses};
    cuuint64_t strides[4] = {rowb, rowb * nx_in, rowb * nx_in * n, rowb * nx_in * n * n};
    cuuint32_t box[5] = {(cuuint32_t)cpr, (cuuint32_t)(g.hw * stride), (cuuint32_t)(g.hh * stride),
                         (cuuint32_t)(g.hd * stride), 1};
    cuuint32_t estr[5] = {1, (cuuint32_t)stride, (cuuint32_t)stride, (cuuint32_t)stride, 1};
    if (sp.blocked == 2) {
        // parity-split: dims (x' * cpr + channel in block, block, y', z', pose * 8 + parity), x' y' z' < n / 2;
        // a box row is hw voxels x 16 bytes, and the element strides are 1
        const cuuint64_t blocks = (cuuint64_t)sp.cin_pad / cpr, h = n / 2;
        dims[0] = h * cpr; dims[1] = blocks; dims[2] = h; dims[3] = h; dims[4] = (cuuint64_t)sp.max_poses * 8;
        strides[0] = h * 16; strides[1] = blocks * h * 16; strides[2] = strides[1] * h; strides[3] = strides[2] * h;
        box[0] = (cuuint32_t)(g.hw * cpr); box[1] = 2; box[2] = (cuuint32_t)g.hh; box[3] = (cuuint32_t)g.hd; box[4] = 1;
        for (int i = 0; i < 5; ++i) estr[i] = 1;
    } else if (sp.blocked) {
        // dims (x * cpr + channel in block, block, y, z, pose); a box row is hw voxels x 16 bytes
        const cuuint64_t blocks = (cuuint64_t)sp.cin_pad / cpr;
        dims[0] = nx_in * cpr; dims[1] = blocks; dims[2] = n; dims[3] = n; dims[4] = (cuuint64_t)sp.max_poses;
        strides[0] = nx_in * 16; strides[1] = blocks * nx_in * 16; strides[2] = strides[1] * n; strides[3] = strides[2] * n;
        box[0] = (cuuint32_t)(g.hw * cpr); box[1] = 2; box[2] = (cuuint32_t)g.hh; box[3] = (cuuint32_t)g.hd; box[4] = 1;
    }
    CUresult r = enc(&P.tmap, sp.elem == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 5,
                     const_cast<void *>(sp.x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(why, why_len, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        return -2;
    }
    Args &A = P.args;
    A.xres = static_cast<const __nv_bfloat16 *>(sp.xres);
    A.cres = sp.cres;
    A.w = static_cast<const uint8_t *>(sp.w);
    A.s_in = sp.s_in;
    A.s_w = sp.s_w;
    A.amax = sp.amax;
    A.bias = sp.bias;
    A.y = static_cast<__nv_bfloat16 *>(sp.y);
    A.n_in = sp.n_in;
    A.n_out = sp.n_out;
    A.cin = sp.cin_pad;
    A.k = k;
    A.stride = stride;
    A.pad = k / 2;
    A.residual = sp.residual;
    A.xpat = sp.fold ? 1 : 0;
    A.x_shift = sp.fold == 2 ? 1 : 0;
    if (sp.fold) fold_pattern(sp.fold, k, A.xt_n, A.xt_step, A.xt_start);
    A.blocked = sp.blocked;
    A.out_blocked = sp.out_blocked;
    A.res_blocked = sp.res_blocked;
    A.g = g;
    A.err = sp.err;
    P.N = c_out;
    P.T = T;
    P.f8 = sp.elem == 1;
    P.group = group;
    P.grid = (unsigned)(g.nbx * g.nby * g.nbz);   // tiles per pose; times B at launch
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms <= 0) {
        snprintf(why, why_len, "cannot read the multiprocessor count");
        return -2;
    }
    P.sms = sms;
    if (!P.counter && cudaMalloc(&P.counter, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        snprintf(why, why_len, "cannot allocate the tile counter");
        return -2;
    }
    A.tile_counter = P.counter;
    return 0;
}

template <int N, int T, bool F8, int G>
static void launch_t(ConvTcPlan::Impl &P, int B, cudaStream_t s) {
    cudaFuncSetAttribute(conv3d_tc_kernel<N, T, F8, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
    // persistent: one CTA per multiprocessor (one fits at this shared-memory size); tiles from the counter
    P.args.B = B;
    const unsigned tiles = P.grid * (unsigned)B;
    const unsigned grid = tiles < (unsigned)P.sms ? tiles : (unsigned)P.sms;
    cudaMemsetAsync(P.counter, 0, sizeof(int), s);
    conv3d_tc_kernel<N, T, F8, G><<<grid, Roles<N, T, G>::THREADS, P.smem, s>>>(P.tmap, P.args);
}

template <int N, int T, bool F8>
static void launch_g(ConvTcPlan::Impl &P, int B, cudaStream_t s) {
    if constexpr (T == 16 && 8 * N <= 256) {
        if (P.group == 8) return launch_t<N, T, F8, 8>(P, B, s);
    }
    if constexpr (T % 4 == 0 && 4 * N <= 256) {
        if (P.group == 4) return launch_t<N, T, F8, 4>(P, B, s);
    }
    if constexpr (T % 2 == 0 && 2 * N <= 256) {
        if (P.group == 2) return launch_t<N, T, F8, 2>(P, B, s);
    }
    launch_t<N, T, F8, 1>(P, B, s);
}

template <bool F8>
static void launch_n(ConvTcPlan::Impl &P, int B, cudaStream_t s) {
    switch (P.N * 16 + P.T) {
    case 32 * 16 + 4: launch_g<32, 4, F8>(P, B, s); break;
    case 32 * 16 + 8: launch_g<32, 8, F8>(P, B, s); break;
    case 32 * 16 + 16: launch_g<32, 16, F8>(P, B, s); break;
    case 64 * 16 + 4: launch_g<64, 4, F8>(P, B, s); break;
    case 64 * 16 + 8: launch_g<64, 8, F8>(P, B, s); break;
    case 128 * 16 + 2: launch_g<128, 2, F8>(P, B, s); break;
    case 128 * 16 + 4: launch_g<128, 4, F8>(P, B, s); break;
    default: launch_g<256, 2, F8>(P, B, s); break;
    }
}

void conv_tc_describe(const ConvTcPlan &plan, int *T, int *groups_per_stage, int *nbs, size_t *smem, int *group) {
    *T = plan.impl->T;
    *groups_per_stage = plan.impl->args.g.groups_per_stage;
    *nbs = plan.impl->args.g.nbs;
    *smem = plan.impl->smem;
    *group = plan.impl->group;
}

void conv_tc_stall_next(ConvTcPlan &plan) { plan.impl->args.stall = 1; }

void conv_tc_launch(ConvTcPlan &plan, int B, cudaStream_t s) {
    ConvTcPlan::Impl &P = *plan.impl;
    if (P.f8) launch_n<true>(P, B, s);
    else launch_n<false>(P, B, s);
    P.args.stall = 0;   // one launch only
}

}  // namespace fusion
