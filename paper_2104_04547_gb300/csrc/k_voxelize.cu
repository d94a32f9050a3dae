// Pose preparation and gather-form voxelization (Section 1 and Section 3.3:
// atoms become a multi-channel density grid; the paper keeps the FAST grid
// sizing and atom propagation, read here as a voxel-integrated isotropic
// Gaussian over the cube of voxels within +-k of the atom's own voxel).
//
// prep_kernel (one CTA per pose): validates the pose, computes the grid origin
// (ligand centroid summed left to right in float32, minus half a grid edge)
// and, per atom, its containing voxel and the 3 x (2k+1) per-axis weights
//   w_d(i) = 1/2 [erf((u_i + h - x_d)/(sigma sqrt 2)) - erf((u_i - x_d)/(sigma sqrt 2))].
//
// prep_kernel also marks, per pose, the 8^3 tiles that some atom's support cube
// meets.  voxelize_kernel (one CTA per 8^3 voxel tile of a pose) stores zeros at
// once for an unmarked tile (on docked poses about 70% of a 48^3 grid's tiles
// hold no atom); otherwise it compacts, in atom
// order, the atoms whose support cube meets the tile, stages them in shared
// memory and accumulates all channels of each voxel in registers in atom-index
// order (deterministic, no atomics), then stores the voxel's channels as one
// contiguous vector (16-byte stores) in the NDHWC layout the first conv reads.
// For the bf16 tensor-core conv the 3 channels beyond the first 16 are stored
// folded along x (fold_pad >= 0): the second 16-channel chunk of voxel x holds
// features 16..18 of voxels x - p .. x - p + 4, so that chunk needs 2 x-offsets
// of the 7^3 kernel instead of 7 (it would otherwise be 13/16 zero padding).
// voxelize_kernel stores each voxel's own features 16..18 at slot s = p, and
// fold_grid_kernel then builds the folded chunks row by row.
#include "fusion_internal.cuh"

#include <math.h>

namespace fusion {

namespace {

constexpr int kTile = 8;      // voxelize tiles are kTile^3 voxels

// erf(b) - erf(a) for a < b, through erfc in the tails to keep relative accuracy.
__device__ __forceinline__ float erf_diff(float a, float b) {
    if (a >= 0.f) return erfcf(a) - erfcf(b);
    if (b <= 0.f) return erfcf(-b) - erfcf(-a);
    return erff(b) - erff(a);
}

__global__ void __launch_bounds__(256) prep_kernel(PrepArgs a) {
    const int p = blockIdx.x;
    const int a0 = a.atom_off[p];
    const int N = a.atom_off[p + 1] - a0;
    const int nl = a.n_lig[p];
    __shared__ float s_org[3];
    __shared__ uint32_t s_mask[kTileMaskWords];
    if (N < 1 || N > a.max_atoms || nl < 1 || nl > N || a0 < 0) {
        if (threadIdx.x == 0) atomicOr(a.err, FUSION_ERR_INPUT);
        return;
    }
    for (int w = threadIdx.x; w < kTileMaskWords; w += blockDim.x) s_mask[w] = 0u;
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        float s = 0.f;
        for (int i = 0; i < nl; ++i) s = __fadd_rn(s, a.xyz[(size_t)(a0 + i) * 3 + d]);
        const float c = __fdiv_rn(s, (float)nl);
        const float half = __fmul_rn(__fmul_rn((float)a.grid_n, a.h), 0.5f);
        const float o = __fsub_rn(c, half);
        s_org[d] = o;
        a.origin[p * 3 + d] = o;
    }
    __syncthreads();
    const int K = a.k, KW = 2 * a.k + 1;
    const float inv = 1.0f / (a.sigma * 1.41421356237309515f);
    bool bad = false;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const size_t ai = (size_t)a0 + i;
        int c3[3];
        for (int d = 0; d < 3; ++d) {
            const float x = a.xyz[ai * 3 + d];
            if (!isfinite(x)) bad = true;
            const float t = __fsub_rn(x, s_org[d]);
            float q = floorf(__fdiv_rn(t, a.h));
            q = fminf(fmaxf(q, -1.0e6f), 1.0e6f);      // far outside the grid: contributes nothing
            if (!isfinite(t)) q = -1.0e6f;
            const int ci = (int)q;
            c3[d] = ci;
            float *w = a.atom_w + (ai * 3 + (2 - d)) * KW;   // slots: 0 z, 1 y, 2 x
            for (int m = 0; m < KW; ++m) {
                const int idx = ci - K + m;
                const float lo = __fsub_rn((float)idx * a.h, t);
                const float hi = __fsub_rn((float)(idx + 1) * a.h, t);
                w[m] = 0.5f * erf_diff(lo * inv, hi * inv);
            }
        }
        a.atom_vox[ai] = make_int4(c3[2], c3[1], c3[0], p);
        // the 8^3 tiles (of the tiles^3 that cover the grid) that the support cube c +- K meets: the same
        // test voxelize_kernel's compaction makes, so a tile with a clear bit has no candidate atom
        const int tiles = (a.grid_n + kTile - 1) / kTile, last = tiles * kTile - 1;
        int lo[3], hi[3];
        bool meets = true;
        for (int d = 0; d < 3; ++d) {
            const int c = c3[2 - d];                     // z, y, x
            if (c + K < 0 || c - K > last) meets = false;
            lo[d] = max(c - K, 0) / kTile;
            hi[d] = min(c + K, last) / kTile;
        }
        if (meets)
            for (int tz = lo[0]; tz <= hi[0]; ++tz)
                for (int ty = lo[1]; ty <= hi[1]; ++ty)
                    for (int tx = lo[2]; tx <= hi[2]; ++tx) {
                        const int t = (tz * tiles + ty) * tiles + tx;
                        atomicOr(&s_mask[t >> 5], 1u << (t & 31));
                    }
    }
    if (bad) atomicOr(a.err, FUSION_ERR_INPUT);
    __syncthreads();
    for (int w = threadIdx.x; w < kTileMaskWords; w += blockDim.x) a.tile_mask[(size_t)p * kTileMaskWords + w] = s_mask[w];
}

constexpr int kStage = 256;
constexpr int kFeatPad = 20;   // staged features per atom: 19 + 1 zero, so a thread reads them as 5 float4

template <bool BF16, int CX>
__global__ void __launch_bounds__(512, 3) voxelize_kernel(VoxArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.grid_n;
    const int K = a.k, KW = 2 * a.k + 1;
    const int tiles = (n + kTile - 1) / kTile;
    const int t = blockIdx.x;
    const int p = blockIdx.y;
    const int t0x = (t % tiles) * kTile;
    const int t0y = ((t / tiles) % tiles) * kTile;
    const int t0z = (t / (tiles * tiles)) * kTile;
    const int a0 = a.atom_off[p];
    const int N = a.atom_off[p + 1] - a0;
    if (N < 1 || N > a.max_atoms) return;

    // 0. a tile that no atom's support meets holds zeros: store them without scanning the atoms
    const bool empty = !((a.tile_mask[(size_t)p * kTileMaskWords + (t >> 5)] >> (t & 31)) & 1u);

    int4 *s_v = reinterpret_cast<int4 *>(smem);                  // [kStage]
    float *s_w = reinterpret_cast<float *>(s_v + kStage);        // [kStage][3*KW]
    float *s_f = s_w + kStage * 3 * KW;                          // [kStage][20], 16-byte aligned rows
    int *s_list = reinterpret_cast<int *>(s_f + kStage * kFeatPad); // [max_atoms]
    __shared__ int s_wsum[16];
    __shared__ int s_total;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // 1. ordered compaction of the atoms whose support cube meets this tile
    int count = 0;
    for (int base = 0; base < (empty ? 0 : N); base += 512) {
        const int i = base + tid;
        bool hit = false;
        if (i < N) {
            const int4 v = a.atom_vox[a0 + i];
            hit = (v.x - K <= t0z + kTile - 1) && (v.x + K >= t0z) &&
                  (v.y - K <= t0y + kTile - 1) && (v.y + K >= t0y) &&
                  (v.z - K <= t0x + kTile - 1) && (v.z + K >= t0x);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        const int lp = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) s_wsum[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            int v = lane < 16 ? s_wsum[lane] : 0;
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (lane < 16) s_wsum[lane] = incl - v;
            if (lane == 15) s_total = incl;
        }
        __syncthreads();
        if (hit) s_list[count + s_wsum[warp] + lp] = i;
        count += s_total;
        __syncthreads();
    }

    // 2. accumulate the voxel's channels over the staged atoms, in atom order
    const int vx = t0x + (tid & 7);
    const int vy = t0y + ((tid >> 3) & 7);
    const int vz = t0z + (tid >> 6);
    const int wz = vz;                                  // this warp's z-slice and y-rows
    const int wy0 = t0y + ((tid >> 3) & 4), wy1 = wy0 + 3;
    float acc[kFeat];
#pragma unroll
    for (int c = 0; c < kFeat; ++c) acc[c] = 0.f;

    for (int r = 0; r < count; r += kStage) {
        const int nr = min(kStage, count - r);
        for (int s = tid; s < nr; s += 512) s_v[s] = a.atom_vox[a0 + s_list[r + s]];
        for (int e = tid; e < nr * 3 * KW; e += 512) {
            const int s = e / (3 * KW), q = e - s * 3 * KW;
            s_w[e] = a.atom_w[(size_t)(a0 + s_list[r + s]) * 3 * KW + q];
        }
        for (int e = tid; e < nr * kFeatPad; e += 512) {
            const int s = e / kFeatPad, q = e - s * kFeatPad;
            s_f[e] = q < kFeat ? a.feat[(size_t)(a0 + s_list[r + s]) * kFeat + q] : 0.f;
        }
        __syncthreads();
        // A warp covers one z-slice, 4 y-rows and the 8 x-columns of the tile: 32 staged atoms at a time,
        // each lane tests one against that box and the warp then visits only the atoms that can reach it,
        // in ascending order (so every voxel still sums its atoms in atom-index order).
        for (int base = 0; base < nr; base += 32) {
            const int sl = base + lane;
            bool rel = false;
            if (sl < nr) {
                const int4 v = s_v[sl];
                rel = v.x - K <= wz && v.x + K >= wz && v.y - K <= wy1 && v.y + K >= wy0 && v.z - K <= t0x + 7 &&
                      v.z + K >= t0x;
            }
            unsigned todo = __ballot_sync(0xffffffffu, rel);
            while (todo) {
                const int s = base + __ffs(todo) - 1;
                todo &= todo - 1;
                const int4 v = s_v[s];
                const unsigned dz = (unsigned)(vz - (v.x - K));
                const unsigned dy = (unsigned)(vy - (v.y - K));
                const unsigned dx = (unsigned)(vx - (v.z - K));
                if (dz < (unsigned)KW && dy < (unsigned)KW && dx < (unsigned)KW) {
                    const float *w = s_w + s * 3 * KW;
                    const float wv = (w[dz] * w[KW + dy]) * w[2 * KW + dx];
                    const float4 *f4 = reinterpret_cast<const float4 *>(s_f + s * kFeatPad);
#pragma unroll
                    for (int c4 = 0; c4 < kFeatPad / 4; ++c4) {
                        const float4 f = f4[c4];
                        acc[4 * c4] = fmaf(wv, f.x, acc[4 * c4]);
                        acc[4 * c4 + 1] = fmaf(wv, f.y, acc[4 * c4 + 1]);
                        acc[4 * c4 + 2] = fmaf(wv, f.z, acc[4 * c4 + 2]);
                        if (4 * c4 + 3 < kFeat) acc[4 * c4 + 3] = fmaf(wv, f.w, acc[4 * c4 + 3]);
                    }
                }
            }
        }
        __syncthreads();
    }

    // 3. store the voxel's channel vector (channels >= 19 are zero padding)
    float vmax = 0.f;                                   // max |stored bf16 value| of this voxel
    if (vx < n && vy < n && vz < n) {
        const size_t vox = (((size_t)p * n + vz) * n + vy) * n + vx;
        if constexpr (BF16) {
            // 8-channel block c0 / 8 of the voxel: NDHWC, or channel-blocked [row][CX / 8][x][8]
            const size_t row = ((size_t)p * n + vz) * n + vy;
            __nv_bfloat16 *const base = reinterpret_cast<__nv_bfloat16 *>(a.out);
            auto blk = [&](int c0) { return a.blocked ? base + ((row * (CX / 8) + c0 / 8) * n + vx) * 8 : base + vox * CX + c0; };
            if (a.fold_pad < 0) {
#pragma unroll
                for (int c0 = 0; c0 < CX; c0 += 8) {
                    __align__(16) __nv_bfloat16 v8[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        v8[j] = __float2bfloat16_rn(c0 + j < kFeat ? acc[c0 + j] : 0.f);
                        vmax = fmaxf(vmax, fabsf(__bfloat162float(v8[j])));
                    }
                    *reinterpret_cast<uint4 *>(blk(c0)) = *reinterpret_cast<const uint4 *>(v8);
                }
            } else {
                // folded layout, first pass: features 16..18 at slot s = p of the voxel's own second chunk
                // (where the fold keeps them), the rest of that chunk zero; fold_grid_kernel fills it in
                const int sp = 16 + 3 * a.fold_pad;
#pragma unroll
                for (int c0 = 0; c0 < CX; c0 += 8) {
                    __align__(16) __nv_bfloat16 v8[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int c = c0 + j;
                        // constant register indices only (sp is a runtime value)
                        const int d = c - sp;
                        const float v = c < 16 ? acc[c < 16 ? c : 0]
                                               : d == 0 ? acc[16] : d == 1 ? acc[17] : d == 2 ? acc[18] : 0.f;
                        v8[j] = __float2bfloat16_rn(v);
                        vmax = fmaxf(vmax, fabsf(__bfloat162float(v8[j])));
                    }
                    *reinterpret_cast<uint4 *>(blk(c0)) = *reinterpret_cast<const uint4 *>(v8);
                }
            }
        } else {
            float *out = reinterpret_cast<float *>(a.out) + vox * CX;
#pragma unroll
            for (int c0 = 0; c0 < CX; c0 += 4) {
                float4 v4;
                v4.x = c0 + 0 < kFeat ? acc[c0 + 0] : 0.f;
                v4.y = c0 + 1 < kFeat ? acc[c0 + 1] : 0.f;
                v4.z = c0 + 2 < kFeat ? acc[c0 + 2] : 0.f;
                v4.w = c0 + 3 < kFeat ? acc[c0 + 3] : 0.f;
                *reinterpret_cast<float4 *>(out + c0) = v4;
            }
        }
    }
    if (a.amax) {
        // the pose's max |grid value| for the FP8 input scale: warps, then one atomic per CTA
        __shared__ float s_wmax[16];
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if (lane == 0) s_wmax[warp] = vmax;
        __syncthreads();
        if (tid == 0) {
            float m = 0.f;
            for (int w = 0; w < 16; ++w) m = fmaxf(m, s_wmax[w]);
            if (m > 0.f) atomicMax(reinterpret_cast<unsigned *>(a.amax + p), __float_as_uint(m));
        }
    }
}


// Channels 16 + 8 j .. 23 + 8 j (j = 0, 1) of voxel x of grid row `row` (pose, z, y), 32 channels per voxel.
__device__ __forceinline__ __nv_bfloat16 *hi_block(__nv_bfloat16 *grid, int row, int x, int j, int n, int blocked) {
    return blocked ? grid + (((size_t)row * 4 + 2 + j) * n + x) * 8 : grid + ((size_t)row * n + x) * 32 + 16 + 8 * j;
}

// Second pass of the folded layout: one CTA per 8 x-rows (all poses, z, y); each row's features
// 16..18 (at slot 16 + 3p) are staged in shared memory first, then every voxel's second chunk is
// rewritten as slot 16 + 3 s + f = feature 16 + f of voxel x - p + s (zero outside the grid) with
// 16-byte stores.  Rows are independent, and a row is read completely before any of it is written.
__global__ void __launch_bounds__(256) fold_grid_kernel(__nv_bfloat16 *grid, int rows, int n, int p, int blocked) {
    extern __shared__ __align__(16) __nv_bfloat16 s_r[];     // [8][n][3]
    const int r0 = blockIdx.x * 8;
    const int nr = min(8, rows - r0);
    const int sp = 16 + 3 * p;
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        // the voxel's channels 16..31 in two 16-byte loads (one 32-byte sector), then the 3 at slot sp
        const int r = e / n, x = e - r * n;
        const uint4 a0 = *reinterpret_cast<const uint4 *>(hi_block(grid, r0 + r, x, 0, n, blocked));
        const uint4 a1 = *reinterpret_cast<const uint4 *>(hi_block(grid, r0 + r, x, 1, n, blocked));
        const uint32_t wd[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        // select with constant indices (sp is a runtime value; a runtime index would go to local memory)
        const int o = sp - 16;
        unsigned short v0 = 0, v1 = 0, v2 = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const unsigned short hv = (unsigned short)((i & 1) ? (wd[i >> 1] >> 16) : (wd[i >> 1] & 0xFFFFu));
            if (i == o) v0 = hv;
            if (i == o + 1) v1 = hv;
            if (i == o + 2) v2 = hv;
        }
        s_r[e * 3 + 0] = __ushort_as_bfloat16(v0);
        s_r[e * 3 + 1] = __ushort_as_bfloat16(v1);
        s_r[e * 3 + 2] = __ushort_as_bfloat16(v2);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        const int r = e / n, x = e - r * n;
        __align__(16) __nv_bfloat16 v16[16];
#pragma unroll
        for (int sl = 0; sl < 5; ++sl) {
            const int xs = x - p + sl;
            const bool in = xs >= 0 && xs < n;
#pragma unroll
            for (int f = 0; f < 3; ++f) v16[3 * sl + f] = in ? s_r[(r * n + xs) * 3 + f] : __float2bfloat16_rn(0.f);
        }
        v16[15] = __float2bfloat16_rn(0.f);
        *reinterpret_cast<uint4 *>(hi_block(grid, r0 + r, x, 0, n, blocked)) = reinterpret_cast<const uint4 *>(v16)[0];
        *reinterpret_cast<uint4 *>(hi_block(grid, r0 + r, x, 1, n, blocked)) = reinterpret_cast<const uint4 *>(v16)[1];
    }
}

size_t vox_smem(int k, int max_atoms) {
    const int KW = 2 * k + 1;
    return (size_t)kStage * sizeof(int4) + (size_t)kStage * 3 * KW * 4 + (size_t)kStage * kFeatPad * 4 +
           (size_t)max_atoms * 4;
}

template <bool BF16, int CX>
void launch_vox_t(const VoxArgs &a, cudaStream_t s) {
    const int tiles = (a.grid_n + kTile - 1) / kTile;
    const size_t sm = vox_smem(a.k, a.max_atoms);
    cudaFuncSetAttribute(voxelize_kernel<BF16, CX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    // three 512-thread CTAs per SM (40 registers, 3 x 51 KB of shared memory at 1200 atoms): measured
    // 11% faster than two; four would need 32 registers and spill
    cudaFuncSetAttribute(voxelize_kernel<BF16, CX>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    dim3 grid(tiles * tiles * tiles, a.n_poses);
    voxelize_kernel<BF16, CX><<<grid, 512, sm, s>>>(a);
}

}  // namespace

void launch_prep(const PrepArgs &a, cudaStream_t s) {
    prep_kernel<<<a.n_poses, 256, 0, s>>>(a);
}

void launch_voxelize(const VoxArgs &a, cudaStream_t s) {
    if (a.out_bf16) {
        launch_vox_t<true, 32>(a, s);
        if (a.fold_pad >= 0) {
            const int rows = a.n_poses * a.grid_n * a.grid_n;
            fold_grid_kernel<<<(rows + 7) / 8, 256, (size_t)8 * a.grid_n * 3 * sizeof(__nv_bfloat16), s>>>(
                static_cast<__nv_bfloat16 *>(a.out), rows, a.grid_n, a.fold_pad, a.blocked);
        }
    } else if (a.cx == 24) {
        launch_vox_t<false, 24>(a, s);
    } else {
        launch_vox_t<false, 20>(a, s);
    }
}

}  // namespace fusion
