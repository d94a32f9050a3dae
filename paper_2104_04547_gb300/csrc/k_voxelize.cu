// Pose preparation, the voxel-cell list, and gather-form voxelization (Section 1
// and Section 3.3: atoms become a multi-channel density grid; the paper keeps the
// FAST grid sizing and atom propagation, read here as a voxel-integrated
// isotropic Gaussian over the cube of voxels within +-k of the atom's own voxel).
//
// prep_kernel (four CTAs per pose): validates the pose, computes the grid origin
// (ligand centroid summed left to right in float32, minus half a grid edge)
// and, per atom, its containing voxel and the 3 x (2k+1) per-axis weights
//   w_d(i) = 1/2 [erf((u_i + h - x_d)/(sigma sqrt 2)) - erf((u_i - x_d)/(sigma sqrt 2))].
// It then counting-sorts the pose's atoms into a list of 1 A cells (a cell is a
// voxel of the extended range [-k, n-1+k]^3, so exactly the atoms whose support
// cube meets the grid are listed): atoms ordered by cell (z, y, x) and, within a
// cell, by atom index, with an index of where each (z, y) row of cells starts.
// The row sorts make the order independent of the atomics that place atoms.  Each
// of a pose's CTAs builds the same list and writes a quarter of its records (the
// per-axis weights are most of the work).
//
// voxelize_kernel (one CTA per tile of 4 y-rows x 2 z-slices x all n x-voxels
// of a pose): the atoms whose support meets the tile are, for each z-row of
// cells in reach, one contiguous run of the cell list (cells (cz, cy_lo..cy_hi,
// all x) are consecutive), so the tile's candidates come from at most 2 + 2k
// runs, read in cell order.  They are staged in shared memory in chunks; each
// warp owns a 4 (x) x 4 (y) x 2 (z) voxel box (a lane per voxel), tests 32
// staged atoms at a time against its box by ballot, and accumulates all channels
// of its voxels over the atoms that reach it in cell-list order (deterministic,
// no atomics).  A tile with no candidate stores zeros without staging anything.
//
// Stores: one contiguous vector per voxel (16-byte stores) in the NDHWC layout
// (float32, or bf16 for the FP8 path's quantizer) or, for the bf16 tensor-core
// conv, channel-blocked with the 3 channels beyond the first 16 folded along x
// (fold_pad = p >= 0): the second 16-channel chunk of voxel x holds features
// 16..18 of voxels x - p .. x - p + 4, so that chunk needs 2 x-offsets of a 7^3
// kernel instead of 7 (it would otherwise be 13/16 zero padding).  A tile spans
// whole x-rows, so the fold reads its neighbours from shared memory and the grid
// is written once.
#include "fusion_internal.cuh"

#include <math.h>

namespace fusion {

namespace {

constexpr int kPrepThreads = 256;
constexpr int kPrepSplit = 4;     // CTAs per pose: each builds the pose's cell list, a quarter of its records

// erf(b) - erf(a) for a < b, through erfc in the tails to keep relative accuracy.
__device__ __forceinline__ float erf_diff(float a, float b) {
    if (a >= 0.f) return erfcf(a) - erfcf(b);
    if (b <= 0.f) return erfcf(-b) - erfcf(-a);
    return erff(b) - erff(a);
}

// In-place exclusive scan of d[0..n) by the whole block (blockDim.x a multiple of 32, at most 1024).
__device__ void block_exscan(int *d, int n, int *s_tmp /* [33] */) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int beg = min(tid * per, n), end = min(beg + per, n);
    int sum = 0;
    for (int i = beg; i < end; ++i) sum += d[i];
    int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        const int v = lane < nw ? s_tmp[lane] : 0;
        int wi = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < nw) s_tmp[lane] = wi - v;
    }
    __syncthreads();
    int run = s_tmp[warp] + incl - sum;
    for (int i = beg; i < end; ++i) {
        const int v = d[i];
        d[i] = run;
        run += v;
    }
    __syncthreads();
}

// The containing voxel of coordinate x on one axis, floor(fl32(fl32(x - o) / h)), clamped far outside the grid.
__device__ __forceinline__ int containing_voxel(float x, float o, float h, float *t_out) {
    const float t = __fsub_rn(x, o);
    float q = floorf(__fdiv_rn(t, h));
    q = fminf(fmaxf(q, -1.0e6f), 1.0e6f);      // far outside the grid: contributes nothing
    if (!isfinite(t)) q = -1.0e6f;
    *t_out = t;
    return (int)q;
}

__global__ void __launch_bounds__(kPrepThreads) prep_kernel(PrepArgs a) {
    extern __shared__ __align__(16) int psm[];
    const int p = blockIdx.x;
    const int part = blockIdx.y;                     // kPrepSplit CTAs per pose share the record writing
    const int K = a.k, KW = 2 * a.k + 1;
    const int R = a.grid_n + 2 * K, RR = R * R;
    int *s_start = psm;                  // [RR + 1] row starts (counts first)
    int *s_cur = s_start + RR + 1;       // [RR] fill cursors
    int *s_row = s_cur + RR;             // [max_atoms] row of atom i, or -1 (support misses the grid)
    int *s_key = s_row + a.max_atoms;    // [max_atoms] (cx + k) << 16 | i
    int *s_list = s_key + a.max_atoms;   // [max_atoms] keys in cell order
    float *s_xyz = reinterpret_cast<float *>(s_list + a.max_atoms);   // [max_atoms][3] the pose's coordinates
    __shared__ float s_org[3];
    __shared__ int s_tmp[33];
    int32_t *row_out = a.cell_row + (size_t)p * (RR + 1);
    for (int r = threadIdx.x; r <= RR; r += blockDim.x) s_start[r] = 0;
    const int a0 = a.atom_off[p];
    const int N = a.atom_off[p + 1] - a0;
    const int nl = a.n_lig[p];
    if (N < 1 || N > a.max_atoms || nl < 1 || nl > N || a0 < 0) {
        // an empty cell list keeps the voxelize kernel's reads in bounds; the call fails on the flag
        if (part == 0) {
            for (int r = threadIdx.x; r <= RR; r += blockDim.x) row_out[r] = 0;
            if (threadIdx.x == 0) atomicOr(a.err, FUSION_ERR_INPUT);
        }
        return;
    }
    for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) s_xyz[e] = a.xyz[(size_t)a0 * 3 + e];
    __syncthreads();
    if (threadIdx.x < 3) {
        // the ligand centroid, summed left to right (a float32 decision both sides make the same way)
        const int d = threadIdx.x;
        float s = 0.f;
        for (int i = 0; i < nl; ++i) s = __fadd_rn(s, s_xyz[i * 3 + d]);
        const float c = __fdiv_rn(s, (float)nl);
        const float half = __fmul_rn(__fmul_rn((float)a.grid_n, a.h), 0.5f);
        const float o = __fsub_rn(c, half);
        s_org[d] = o;
        if (part == 0) a.origin[p * 3 + d] = o;
    }
    __syncthreads();
    // 1. each atom's cell: its containing voxel, if that lies in the extended range (its support meets the grid)
    bool bad = false;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        int c3[3];
        bool in = true;
        for (int d = 0; d < 3; ++d) {
            const float x = s_xyz[i * 3 + d];
            if (!isfinite(x)) bad = true;
            float t;
            c3[d] = containing_voxel(x, s_org[d], a.h, &t);
            in = in && c3[d] >= -K && c3[d] <= a.grid_n - 1 + K;
        }
        const int r = in ? (c3[2] + K) * R + (c3[1] + K) : -1;
        s_row[i] = r;
        s_key[i] = ((c3[0] + K) << 16) | i;
        if (r >= 0) atomicAdd(&s_start[r], 1);
    }
    if (bad && part == 0) atomicOr(a.err, FUSION_ERR_INPUT);
    __syncthreads();
    // 2. counting sort by row, then each row's entries by (cx, atom index): insertion sort, rows hold a few atoms
    block_exscan(s_start, RR + 1, s_tmp);              // s_start[RR] = atoms listed
    for (int r = threadIdx.x; r < RR; r += blockDim.x) s_cur[r] = s_start[r];
    if (part == 0)
        for (int r = threadIdx.x; r <= RR; r += blockDim.x) row_out[r] = s_start[r];
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int r = s_row[i];
        if (r >= 0) s_list[atomicAdd(&s_cur[r], 1)] = s_key[i];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < RR; r += blockDim.x) {
        const int b = s_start[r], e = s_start[r + 1];
        for (int j = b + 1; j < e; ++j) {
            const int v = s_list[j];
            int q = j - 1;
            while (q >= b && s_list[q] > v) {
                s_list[q + 1] = s_list[q];
                --q;
            }
            s_list[q + 1] = v;
        }
    }
    __syncthreads();
    // 3. the records in cell order: voxel and pose, per-axis weights
    //      w_d(m) = 1/2 [erf((u + h - x_d) / (sigma sqrt 2)) - erf((u - x_d) / (sigma sqrt 2))], u = (c_d - k + m) h,
    //    and the features
    const float inv = 1.0f / (a.sigma * 1.41421356237309515f);
    const int WP = atom_rec_wpad(K), RECF = atom_rec_floats(K);
    const int listed = s_start[RR];
    // every CTA of the pose sorted the same list; CTA `part` writes records part, part + kPrepSplit, ...
    for (int j = part + kPrepSplit * threadIdx.x; j < listed; j += kPrepSplit * blockDim.x) {
        const int i = s_list[j] & 0xFFFF;
        const size_t ai = (size_t)a0 + i;
        float *rec = a.atom_rec + ((size_t)a0 + j) * RECF;
        // the features first, all loads in flight together (the record stores below could alias them)
        float f[kFeat];
#pragma unroll
        for (int c = 0; c < kFeat; ++c) f[c] = __ldg(&a.feat[ai * kFeat + c]);
        int c3[3];
        for (int d = 0; d < 3; ++d) {
            float t;
            const int ci = containing_voxel(s_xyz[i * 3 + d], s_org[d], a.h, &t);
            c3[d] = ci;
            float *w = rec + 4 + (2 - d) * KW;          // slots: 0 z, 1 y, 2 x
            for (int m = 0; m < KW; ++m) {
                const int idx = ci - K + m;
                const float lo = __fsub_rn((float)idx * a.h, t);
                const float hi = __fsub_rn((float)(idx + 1) * a.h, t);
                w[m] = 0.5f * erf_diff(lo * inv, hi * inv);
            }
        }
        *reinterpret_cast<int4 *>(rec) = make_int4(c3[2], c3[1], c3[0], p);
        for (int q = 3 * KW; q < WP; ++q) rec[4 + q] = 0.f;
        float4 *rf = reinterpret_cast<float4 *>(rec + 4 + WP);     // 16-byte aligned (WP a multiple of 4)
#pragma unroll
        for (int c4 = 0; c4 < 5; ++c4)
            rf[c4] = make_float4(f[4 * c4], f[4 * c4 + 1], f[4 * c4 + 2], 4 * c4 + 3 < kFeat ? f[4 * c4 + 3] : 0.f);
    }
}

constexpr int kVoxWarps = 6;              // a warp per 4 (x) x 4 (y) x 2 (z) voxel box, BPW boxes each
constexpr int kVoxThreads = 32 * kVoxWarps;
constexpr int kTileY = 4;                 // y-rows per tile
constexpr int kTileZ = 2;                 // z-slices per tile
constexpr int kStage = 128;               // candidate records staged at a time
constexpr int kMaxRuns = 32;              // candidate runs per tile: kTileZ + 2k <= 12

// Element offset of 8-channel block c0 / 8 of voxel (z, y, x) of pose p, 32 bf16 channels per voxel:
// NDHWC, or channel-blocked [p][z][y][4][x][8].
__device__ __forceinline__ size_t bf16_block_off(int p, int z, int y, int x, int c0, int n, int blocked) {
    const size_t row = ((size_t)p * n + z) * n + y;
    return blocked ? ((row * 4 + c0 / 8) * n + x) * 8 : (row * n + x) * 32 + c0;
}

// BPW: x-boxes per warp (a tile spans whole x-rows: ceil(n / 4) boxes; warp w takes boxes w, w + 6, ..., so
// each warp holds boxes from both halves of the row and the warps' work evens out).
// AMAX: also reduce the pose's max |stored value| (the FP8 path's first input scale).
template <bool BF16, int CX, bool AMAX, int BPW>
__global__ void __launch_bounds__(kVoxThreads, 6) voxelize_kernel(VoxArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.grid_n;
    const int K = a.k, KW = 2 * a.k + 1, R = n + 2 * K;
    const int WP = atom_rec_wpad(K), RECF = atom_rec_floats(K);
    const int RW = WP + 20;                            // staged floats per record (weights + features)
    const int nxb = (n + 3) / 4;                       // x-boxes of a row
    const int tiles_y = (n + kTileY - 1) / kTileY;
    const int t = blockIdx.x, p = blockIdx.y;
    const int y0 = (t % tiles_y) * kTileY, z0 = (t / tiles_y) * kTileZ;
    const int a0 = a.atom_off[p];
    const int N = a.atom_off[p + 1] - a0;
    if (N < 1 || N > a.max_atoms) return;

    int4 *s_v = reinterpret_cast<int4 *>(smem);                      // [kStage] (cz, cy, cx, pose)
    float *s_r = reinterpret_cast<float *>(s_v + kStage);            // [kStage][RW] weights, then features
    float *s_wzy = s_r + kStage * RW;                                // [kStage][8] wz(z) wy(y) of the tile's rows
    int *s_list = reinterpret_cast<int *>(s_wzy + kStage * 8);       // [max_atoms] record positions
    __nv_bfloat16 *s_hi = reinterpret_cast<__nv_bfloat16 *>(s_list + a.max_atoms);   // [2][4][nxb * 4][3]
    __shared__ int s_rb[kMaxRuns], s_ro[kMaxRuns + 1];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nruns = kTileZ + 2 * K;
    // this lane's voxel within a box: x = lane & 3, y = (lane >> 2) & 3, z = lane >> 4
    const int lx = lane & 3, ly = (lane >> 2) & 3, lz = lane >> 4;
    const int vy = y0 + ly, vz = z0 + lz;

    // 1. the candidate runs: for z-row cz of the tile's reach, cells (cz, cy_lo..cy_hi, every x) are consecutive
    if (warp == 0) {
        int beg = 0, len = 0;
        const int cz = z0 - K + lane;
        if (lane < nruns && cz <= n - 1 + K) {
            const int32_t *rs = a.cell_row + (size_t)p * (R * R + 1);
            const int cy_lo = max(y0 - K, -K), cy_hi = min(y0 + kTileY - 1 + K, n - 1 + K);
            beg = rs[(cz + K) * R + cy_lo + K];
            len = rs[(cz + K) * R + cy_hi + K + 1] - beg;
        }
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        s_rb[lane] = beg;
        s_ro[lane] = incl - len;
        if (lane == 31) s_ro[kMaxRuns] = incl;
    }
    __syncthreads();
    const int M = min(s_ro[kMaxRuns], N);

    if (M == 0) {
        // no atom reaches the tile: zeros (the folded channels too), nothing staged
#pragma unroll
        for (int j = 0; j < BPW; ++j) {
            const int vx = (warp + kVoxWarps * j) * 4 + lx;
            if (vx >= n || vy >= n || vz >= n) continue;
            if constexpr (BF16) {
                __nv_bfloat16 *const out = reinterpret_cast<__nv_bfloat16 *>(a.out);
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    *reinterpret_cast<uint4 *>(out + bf16_block_off(p, vz, vy, vx, 8 * b, n, a.blocked)) =
                        make_uint4(0u, 0u, 0u, 0u);
            } else {
                float4 *out = reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.out) +
                                                         ((((size_t)p * n + vz) * n + vy) * n + vx) * CX);
#pragma unroll
                for (int c4 = 0; c4 < CX / 4; ++c4) out[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        return;
    }

    // 2. the positions of the tile's candidates in the cell-ordered records
    for (int i = tid; i < M; i += kVoxThreads) {
        int r = 0;
        while (r + 1 < nruns && s_ro[r + 1] <= i) ++r;
        s_list[i] = a0 + s_rb[r] + (i - s_ro[r]);
    }
    // stage candidates r0 .. r0 + nr: records copied 16 bytes at a time (whole rows are contiguous in memory)
    const int q4 = RECF / 4;
    const unsigned mq = ((1u << 20) + q4 - 1) / q4;    // e / q4 = (e mq) >> 20 for e < 2^16
    // then, per staged atom and tile row (z0 + lz, y0 + ly), the product wz * wy (zero outside its support), so a
    // visit needs only the x weight
    auto stage = [&](int r0, int nr) {
        for (int e = tid; e < nr * q4; e += kVoxThreads) {
            const int c = (int)(((unsigned)e * mq) >> 20), part = e - c * q4;
            const float4 v = reinterpret_cast<const float4 *>(a.atom_rec + (size_t)s_list[r0 + c] * RECF)[part];
            if (part == 0) s_v[c] = make_int4(__float_as_int(v.x), __float_as_int(v.y), __float_as_int(v.z), 0);
            else reinterpret_cast<float4 *>(s_r + c * RW)[part - 1] = v;
        }
        __syncthreads();
        for (int e = tid; e < nr * 8; e += kVoxThreads) {
            const int c = e >> 3, rz = (e >> 2) & 1, ry = e & 3;
            const int4 v = s_v[c];
            const unsigned dz = (unsigned)(z0 + rz - (v.x - K)), dy = (unsigned)(y0 + ry - (v.y - K));
            const float *w = s_r + c * RW;
            s_wzy[e] = dz < (unsigned)KW && dy < (unsigned)KW ? w[dz] * w[KW + dy] : 0.f;
        }
    };
    const bool single = M <= kStage;
    if (single) {
        __syncthreads();
        stage(0, M);
        __syncthreads();
    }

    float vmax = 0.f;                                  // max |stored bf16 value| of this thread's voxels
    const bool fold = BF16 && a.fold_pad >= 0;
    const int W = nxb * 4;
#pragma unroll 1
    for (int j = 0; j < BPW; ++j) {
        const int bx = warp + kVoxWarps * j;
        const bool busy = bx < nxb;                    // warp-uniform (the ballots below need every lane)
        const int bx0 = bx * 4;
        const int vx = bx0 + lx;
        float acc[kFeat];
#pragma unroll
        for (int c = 0; c < kFeat; ++c) acc[c] = 0.f;

        // 3. accumulate over the candidates (staged once when they fit, else chunk by chunk per box)
        for (int r0 = 0; r0 < M; r0 += kStage) {
            const int nr = min(kStage, M - r0);
            if (!single) {
                __syncthreads();
                stage(r0, nr);
                __syncthreads();
            }
            if (!busy) continue;
            // 32 staged atoms at a time: each lane tests one against the warp's box (a candidate's y-support
            // always meets the tile's rows), then the warp visits the ones that reach it in list order
            for (int base = 0; base < nr; base += 32) {
                const int sl = base + lane;
                bool rel = false;
                if (sl < nr) {
                    const int4 v = s_v[sl];
                    rel = v.x - K <= z0 + 1 && v.x + K >= z0 && v.z - K <= bx0 + 3 && v.z + K >= bx0;
                }
                unsigned todo = __ballot_sync(0xffffffffu, rel);
                while (todo) {
                    const int s = base + __ffs(todo) - 1;
                    todo &= todo - 1;
                    // the lane's weight: (wz wy) wx, zero outside the atom's support cube, and a zero weight adds
                    // exactly nothing (fmaf(0, f, acc) == acc for the finite features), so no lane branches off
                    const float *w = s_r + s * RW;
                    const unsigned dx = (unsigned)(vx - (s_v[s].z - K));
                    const float wx = dx < (unsigned)KW ? w[2 * KW + dx] : 0.f;
                    const float wv = s_wzy[s * 8 + lz * 4 + ly] * wx;
                    const float4 *f4 = reinterpret_cast<const float4 *>(w + WP);
#pragma unroll
                    for (int c4 = 0; c4 < 5; ++c4) {
                        const float4 f = f4[c4];
                        acc[4 * c4] = fmaf(wv, f.x, acc[4 * c4]);
                        acc[4 * c4 + 1] = fmaf(wv, f.y, acc[4 * c4 + 1]);
                        acc[4 * c4 + 2] = fmaf(wv, f.z, acc[4 * c4 + 2]);
                        if (4 * c4 + 3 < kFeat) acc[4 * c4 + 3] = fmaf(wv, f.w, acc[4 * c4 + 3]);
                    }
                }
            }
        }

        // 4. stores (channels >= 19 are zero padding)
        const bool in = busy && vx < n && vy < n && vz < n;
        if constexpr (BF16) {
            __nv_bfloat16 *const out = reinterpret_cast<__nv_bfloat16 *>(a.out);
            if (in) {
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    if (fold && b >= 2) break;         // folded: blocks 2 and 3 after the fold below
                    __align__(16) __nv_bfloat16 v8[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int c = 8 * b + q;       // a constant after unrolling: acc stays in registers
                        v8[q] = __float2bfloat16_rn(c < kFeat ? acc[c < kFeat ? c : 0] : 0.f);
                        if (AMAX) vmax = fmaxf(vmax, fabsf(__bfloat162float(v8[q])));
                    }
                    *reinterpret_cast<uint4 *>(out + bf16_block_off(p, vz, vy, vx, 8 * b, n, a.blocked)) =
                        *reinterpret_cast<const uint4 *>(v8);
                }
            }
            if (fold && busy) {
                // features 16..18 of the tile's rows go through shared memory for the fold
                __nv_bfloat16 *h = s_hi + ((size_t)(lz * kTileY + ly) * W + vx) * 3;
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    h[f] = __float2bfloat16_rn(acc[16 + f]);
                    if (AMAX && in) vmax = fmaxf(vmax, fabsf(__bfloat162float(h[f])));
                }
            }
        } else {
            if (in) {
                const size_t vox = (((size_t)p * n + vz) * n + vy) * n + vx;
                float *out = reinterpret_cast<float *>(a.out) + vox * CX;
#pragma unroll
                for (int c0 = 0; c0 < CX; c0 += 4) {
                    float4 v4;
                    v4.x = c0 + 0 < kFeat ? acc[c0 + 0 < kFeat ? c0 + 0 : 0] : 0.f;
                    v4.y = c0 + 1 < kFeat ? acc[c0 + 1 < kFeat ? c0 + 1 : 0] : 0.f;
                    v4.z = c0 + 2 < kFeat ? acc[c0 + 2 < kFeat ? c0 + 2 : 0] : 0.f;
                    v4.w = c0 + 3 < kFeat ? acc[c0 + 3 < kFeat ? c0 + 3 : 0] : 0.f;
                    *reinterpret_cast<float4 *>(out + c0) = v4;
                }
            }
        }
    }

    if (fold) {
        // each voxel's second chunk: slot 16 + 3 s + f = feature 16 + f of voxel x - p + s (zero outside the grid)
        __syncthreads();
        __nv_bfloat16 *const out = reinterpret_cast<__nv_bfloat16 *>(a.out);
        const __nv_bfloat16 *h = s_hi + (size_t)(lz * kTileY + ly) * W * 3;
#pragma unroll
        for (int j = 0; j < BPW; ++j) {
            const int vx = (warp + kVoxWarps * j) * 4 + lx;
            if (vx >= n || vy >= n || vz >= n) continue;
            __align__(16) __nv_bfloat16 v16[16];
#pragma unroll
            for (int sl = 0; sl < 5; ++sl) {
                const int xs = vx - a.fold_pad + sl;
                const bool ok = xs >= 0 && xs < n;
#pragma unroll
                for (int f = 0; f < 3; ++f) v16[3 * sl + f] = ok ? h[xs * 3 + f] : __float2bfloat16_rn(0.f);
            }
            v16[15] = __float2bfloat16_rn(0.f);
            *reinterpret_cast<uint4 *>(out + bf16_block_off(p, vz, vy, vx, 16, n, a.blocked)) =
                reinterpret_cast<const uint4 *>(v16)[0];
            *reinterpret_cast<uint4 *>(out + bf16_block_off(p, vz, vy, vx, 24, n, a.blocked)) =
                reinterpret_cast<const uint4 *>(v16)[1];
        }
    }
    if constexpr (AMAX) {
        // the pose's max |grid value| for the FP8 input scale: warps, then one atomic per CTA
        __shared__ float s_wmax[kVoxWarps];
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if (lane == 0) s_wmax[warp] = vmax;
        __syncthreads();
        if (tid == 0) {
            float m = 0.f;
            for (int w = 0; w < kVoxWarps; ++w) m = fmaxf(m, s_wmax[w]);
            if (m > 0.f) atomicMax(reinterpret_cast<unsigned *>(a.amax + p), __float_as_uint(m));
        }
    }
}

int vox_boxes_per_warp(int n) {
    const int nxb = (n + 3) / 4;
    const int b = (nxb + kVoxWarps - 1) / kVoxWarps;
    return b <= 1 ? 1 : b <= 2 ? 2 : 4;
}

size_t vox_smem(int n, int k, int max_atoms) {
    const int RW = atom_rec_wpad(k) + 20;
    return (size_t)kStage * sizeof(int4) + (size_t)kStage * RW * 4 + (size_t)kStage * 8 * 4 + (size_t)max_atoms * 4 +
           (size_t)kTileZ * kTileY * ((n + 3) / 4) * 4 * 3 * sizeof(__nv_bfloat16);
}

size_t prep_smem(int n, int k, int max_atoms) {
    const size_t RR = (size_t)(n + 2 * k) * (n + 2 * k);
    return (2 * RR + 1 + 6 * (size_t)max_atoms) * sizeof(int);
}

template <bool BF16, int CX, bool AMAX, int BPW>
void launch_vox_t(const VoxArgs &a, cudaStream_t s) {
    const int n = a.grid_n;
    const int tiles = ((n + kTileY - 1) / kTileY) * ((n + kTileZ - 1) / kTileZ);
    const size_t sm = vox_smem(n, a.k, a.max_atoms);
    auto kern = voxelize_kernel<BF16, CX, AMAX, BPW>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    dim3 grid(tiles, a.n_poses);
    kern<<<grid, kVoxThreads, sm, s>>>(a);
}

template <bool BF16, int CX, bool AMAX>
void launch_vox_p(const VoxArgs &a, cudaStream_t s) {
    switch (vox_boxes_per_warp(a.grid_n)) {
    case 1: launch_vox_t<BF16, CX, AMAX, 1>(a, s); break;
    case 2: launch_vox_t<BF16, CX, AMAX, 2>(a, s); break;
    default: launch_vox_t<BF16, CX, AMAX, 4>(a, s); break;
    }
}

}  // namespace

void launch_prep(const PrepArgs &a, cudaStream_t s) {
    const size_t sm = prep_smem(a.grid_n, a.k, a.max_atoms);
    cudaFuncSetAttribute(prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    prep_kernel<<<dim3(a.n_poses, kPrepSplit), kPrepThreads, sm, s>>>(a);
}

void launch_voxelize(const VoxArgs &a, cudaStream_t s) {
    if (a.out_bf16) {
        if (a.amax) launch_vox_p<true, 32, true>(a, s);
        else launch_vox_p<true, 32, false>(a, s);
    } else if (a.cx == 24) {
        launch_vox_p<false, 24, false>(a, s);
    } else {
        launch_vox_p<false, 20, false>(a, s);
    }
}

}  // namespace fusion
