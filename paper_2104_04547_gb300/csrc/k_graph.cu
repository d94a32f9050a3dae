// Radius graph with two edge types (Section 1: edge types at distinct distance
// thresholds for covalent and non-covalent interactions; Table II cutoffs).
//
// Three launches: a count pass and a fill pass with kGraphSplit CTAs per pose,
// and between them one CTA per pose that scans the degrees into row offsets.
// Every CTA of the count and fill passes puts its pose's coordinates in shared
// memory and counting-sorts them into a cell list with cells no smaller than
// the non-covalent cutoff (so every neighbour lies in the 27 surrounding cells;
// the three x-adjacent cells of each of the 9 neighbour rows are contiguous in
// cell order).  A warp takes one query atom of the CTA's share at a time, its
// lanes testing the candidates in parallel; the fill pass packs the hits into
// the row by ballot and then sorts the row by neighbour index, so the output is
// canonical.  CTAs stay short (tens of microseconds), so on the low-priority
// stream they never hold an SM for long from the persistent convolutions.
//
// Edge test, exact IEEE float32 with no contraction:
//   s = ((dx*dx + dy*dy) + dz*dz), dx = x_i - x_j (and y, z);
//   covalent iff s < cut_cov^2; non-covalent iff not covalent and s < cut_nc^2; i != j.
// Pose p's edges of each type live at [atom_off[p] * max_degree, ...) of the
// column array; a pose whose edges exceed N * max_degree raises the capacity
// flag and gets no edges.
#include "fusion_internal.cuh"

namespace fusion {

namespace {

constexpr int kCells = kGridCellsMax * kGridCellsMax * kGridCellsMax;
constexpr int kThreads = 256;
constexpr int kGraphSplit = 8;      // CTAs per pose in the count and fill passes

// In-place exclusive scan of d[0..n) by the whole block; returns the total.
__device__ int block_exscan(int *d, int n, int *s_tmp /* [33] */) {
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
        int v = lane < nw ? s_tmp[lane] : 0;
        int wi = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < nw) s_tmp[lane] = wi - v;
        if (lane == 31) s_tmp[32] = wi;
    }
    __syncthreads();
    int run = s_tmp[warp] + incl - sum;
    for (int i = beg; i < end; ++i) {
        const int v = d[i];
        d[i] = run;
        run += v;
    }
    const int total = s_tmp[32];
    __syncthreads();
    return total;
}

__device__ __forceinline__ float dist2_rn(float xi, float yi, float zi, float xj, float yj, float zj) {
    const float dx = __fsub_rn(xi, xj), dy = __fsub_rn(yi, yj), dz = __fsub_rn(zi, zj);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// The pose's coordinates and cell list in shared memory, built by every CTA of the pose (linear in N).
struct CellList {
    float *sx, *sy, *sz;
    int *cell, *sorted, *start;
    int dim[3];
};

__device__ void build_cells(const GraphArgs &a, int a0, int N, unsigned char *smem, CellList &cl) {
    const int MA = a.max_atoms, tid = threadIdx.x, nt = blockDim.x;
    cl.sx = reinterpret_cast<float *>(smem);
    cl.sy = cl.sx + MA;
    cl.sz = cl.sy + MA;
    cl.cell = reinterpret_cast<int *>(cl.sz + MA);    // [MA]
    cl.sorted = cl.cell + MA;                         // [MA] atoms in cell order
    cl.start = cl.sorted + MA;                        // [kCells + 1]
    int *cur = cl.start + kCells + 1;                 // [kCells]
    __shared__ float s_red[6][kThreads / 32];
    __shared__ float s_lo[3], s_L[3];
    __shared__ int s_dim[3];
    __shared__ int s_tmp[33];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = tid; i < N; i += nt) {
        const float x = a.xyz[(size_t)(a0 + i) * 3], y = a.xyz[(size_t)(a0 + i) * 3 + 1], z = a.xyz[(size_t)(a0 + i) * 3 + 2];
        cl.sx[i] = x; cl.sy[i] = y; cl.sz[i] = z;
        lo[0] = fminf(lo[0], x); lo[1] = fminf(lo[1], y); lo[2] = fminf(lo[2], z);
        hi[0] = fmaxf(hi[0], x); hi[1] = fmaxf(hi[1], y); hi[2] = fmaxf(hi[2], z);
    }
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    if ((tid & 31) == 0)
        for (int d = 0; d < 3; ++d) { s_red[d][tid >> 5] = lo[d]; s_red[3 + d][tid >> 5] = hi[d]; }
    for (int c = tid; c <= kCells; c += nt) cl.start[c] = 0;
    __syncthreads();
    if (tid < 3) {
        float l = INFINITY, h = -INFINITY;
        for (int w = 0; w < nt / 32; ++w) { l = fminf(l, s_red[tid][w]); h = fmaxf(h, s_red[3 + tid][w]); }
        const float ext = h - l;
        float L = a.cut_nc * 1.001f + 1e-4f;
        if (ext / L > (float)(kGridCellsMax - 1)) L = ext / (float)(kGridCellsMax - 1) * 1.001f;
        int dim = (int)(ext / L) + 1;
        if (dim > kGridCellsMax) dim = kGridCellsMax;
        s_lo[tid] = l; s_L[tid] = L; s_dim[tid] = dim;
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt) {
        const int cx = max(0, min((int)((cl.sx[i] - s_lo[0]) / s_L[0]), s_dim[0] - 1));
        const int cy = max(0, min((int)((cl.sy[i] - s_lo[1]) / s_L[1]), s_dim[1] - 1));
        const int cz = max(0, min((int)((cl.sz[i] - s_lo[2]) / s_L[2]), s_dim[2] - 1));
        const int c = (cz * s_dim[1] + cy) * s_dim[0] + cx;
        cl.cell[i] = c;
        atomicAdd(&cl.start[c], 1);
    }
    __syncthreads();
    for (int d = 0; d < 3; ++d) cl.dim[d] = s_dim[d];
    const int ncell = cl.dim[0] * cl.dim[1] * cl.dim[2];
    block_exscan(cl.start, ncell + 1, s_tmp);
    for (int c = tid; c < ncell; c += nt) cur[c] = cl.start[c];
    __syncthreads();
    for (int i = tid; i < N; i += nt) {
        const int pos = atomicAdd(&cur[cl.cell[i]], 1);   // order within a cell is arbitrary: rows are sorted later
        cl.sorted[pos] = i;
    }
    __syncthreads();
}

// The query atoms of CTA `part` of a pose: a contiguous share of the pose's atoms.
__device__ __forceinline__ void part_range(int N, int part, int &i0, int &i1) {
    const int per = (N + kGraphSplit - 1) / kGraphSplit;
    i0 = min(part * per, N);
    i1 = min(i0 + per, N);
}

// Candidate run r (0..8) of atom i: the atoms of the three x-adjacent cells of neighbour row (oz, oy) = (r / 3 - 1,
// r % 3 - 1), which are contiguous in cell order.  Returns false if the row lies outside the cell grid.
__device__ __forceinline__ bool cand_run(const CellList &cl, int c, int r, int &q0, int &q1) {
    const int cx = c % cl.dim[0], cy = (c / cl.dim[0]) % cl.dim[1], cz = c / (cl.dim[0] * cl.dim[1]);
    const int zz = cz + r / 3 - 1, yy = cy + r % 3 - 1;
    if (zz < 0 || zz >= cl.dim[2] || yy < 0 || yy >= cl.dim[1]) return false;
    const int row = (zz * cl.dim[1] + yy) * cl.dim[0];
    q0 = cl.start[row + max(cx - 1, 0)];
    q1 = cl.start[row + min(cx + 1, cl.dim[0] - 1) + 1];
    return true;
}

// The query's candidates as one sequence: the 9 runs in order, each run's atoms in cell order.  Lane r < 9
// computes run r; on return every lane holds its run's first position (q0) and the run's offset in the
// sequence (pre, an exclusive prefix over the runs), and the sequence's length is returned.  Candidate idx
// of the sequence lies in the last run r with pre_r <= idx (empty runs share the next run's offset).
__device__ __forceinline__ int cand_seq(const CellList &cl, int c, int lane, int &q0, int &pre) {
    int len = 0;
    q0 = 0;
    if (lane < 9) {
        int a, b;
        if (cand_run(cl, c, lane, a, b)) {
            q0 = a;
            len = b - a;
        }
    }
    int incl = len;
    for (int o = 1; o < 16; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    pre = incl - len;
    return __shfl_sync(0xffffffffu, incl, 8);
}

// Position in cl.sorted of candidate idx of the sequence cand_seq described (q0, pre: this lane's values).
__device__ __forceinline__ int cand_at(int idx, int q0, int pre) {
    int r = 0;
#pragma unroll
    for (int t = 1; t < 9; ++t)
        if (__shfl_sync(0xffffffffu, pre, t) <= idx) r = t;
    return __shfl_sync(0xffffffffu, q0, r) + (idx - __shfl_sync(0xffffffffu, pre, r));
}

// Count pass: a warp per query atom, its lanes over the candidates of the 27 neighbouring cells.
__global__ void __launch_bounds__(kThreads) radius_count_kernel(GraphArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int p = blockIdx.x / kGraphSplit, part = blockIdx.x % kGraphSplit;
    const int a0 = a.atom_off[p];
    const int N = a.atom_off[p + 1] - a0;
    if (N < 1 || N > a.max_atoms || a0 < 0) return;   // flagged by the prep kernel
    CellList cl;
    build_cells(a, a0, N, smem, cl);
    const float c2 = __fmul_rn(a.cut_cov, a.cut_cov);
    const float n2 = __fmul_rn(a.cut_nc, a.cut_nc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int i0, i1;
    part_range(N, part, i0, i1);
    for (int i = i0 + warp; i < i1; i += kThreads / 32) {
        const float xi = cl.sx[i], yi = cl.sy[i], zi = cl.sz[i];
        int d0 = 0, d1 = 0;
        int q0r, prer;
        const int total = cand_seq(cl, cl.cell[i], lane, q0r, prer);
        for (int base = 0; base < total; base += 32) {
            const int q = cand_at(base + lane, q0r, prer);    // every lane takes part in the shuffles
            if (base + lane < total) {
                const int j = cl.sorted[q];
                if (j != i) {
                    const float s = dist2_rn(xi, yi, zi, cl.sx[j], cl.sy[j], cl.sz[j]);
                    if (s < c2) ++d0;
                    else if (s < n2) ++d1;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            d0 += __shfl_xor_sync(0xffffffffu, d0, o);
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        }
        if (lane == 0) { a.deg[0][a0 + i] = d0; a.deg[1][a0 + i] = d1; }
    }
}

// Row offsets: one CTA per pose scans the degrees; a pose whose edges of a type exceed N * max_degree raises the
// capacity flag and gets no edges.
__global__ void __launch_bounds__(kThreads) radius_scan_kernel(GraphArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int p = blockIdx.x;
    const int a0 = a.atom_off[p];
    const int N = a.atom_off[p + 1] - a0;
    if (N < 1 || N > a.max_atoms || a0 < 0) return;
    int *s_d = reinterpret_cast<int *>(smem);          // [max_atoms + 1]
    __shared__ int s_tmp[33];
    const long long cap = (long long)N * a.max_degree;
    const size_t base = (size_t)a0 * a.max_degree;
    for (int e = 0; e < 2; ++e) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) s_d[i] = a.deg[e][a0 + i];
        if (threadIdx.x == 0) s_d[N] = 0;
        __syncthreads();
        const int tot = block_exscan(s_d, N + 1, s_tmp);
        if (tot > cap) {
            if (threadIdx.x == 0) atomicOr(a.err, FUSION_ERR_EDGES);
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                for (int f = 0; f < 2; ++f) { a.beg[f][a0 + i] = (int)base; a.deg[f][a0 + i] = 0; }
            }
            return;
        }
        for (int i = threadIdx.x; i < N; i += blockDim.x) a.beg[e][a0 + i] = (int)(base + s_d[i]);
        __syncthreads();
    }
}

// Sort row[0..n) (distinct atom indices) ascending by the warp into dst[0..n) (dst == row: in place): each
// lane ranks up to kRankPerLane elements against the whole row, then all write after all have read; longer
// rows (only ever sorted in place) fall back to one lane's insertion sort.
constexpr int kRankPerLane = 4;
constexpr int kRowSmem = 32 * kRankPerLane;    // rows packed in shared memory (the fill pass)
__device__ void warp_sort_row(int32_t *row, int n, int lane, int32_t *dst) {
    if (n <= 0) return;
    if (n == 1) {
        if (lane == 0 && dst != row) dst[0] = row[0];
        __syncwarp();
        return;
    }
    if (n > 32 * kRankPerLane) {
        if (lane == 0)
            for (int u = 1; u < n; ++u) {
                const int v = row[u];
                int w = u - 1;
                while (w >= 0 && row[w] > v) { row[w + 1] = row[w]; --w; }
                row[w + 1] = v;
            }
        __syncwarp();
        return;
    }
    int val[kRankPerLane], rank[kRankPerLane];
#pragma unroll
    for (int t = 0; t < kRankPerLane; ++t) {
        const int e = lane + 32 * t;
        val[t] = e < n ? row[e] : 0;
        rank[t] = 0;
    }
    for (int f = 0; f < n; ++f) {
        const int u = row[f];
#pragma unroll
        for (int t = 0; t < kRankPerLane; ++t) rank[t] += (u < val[t]) ? 1 : 0;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < kRankPerLane; ++t)
        if (lane + 32 * t < n) dst[rank[t]] = val[t];
    __syncwarp();
}

// Fill pass: a warp per query atom packs its neighbours by ballot in candidate order (in shared memory while a
// row has at most kRowSmem entries, else in place in the row the scan placed), then sorts each row by
// neighbour index into its place, so the output is canonical.
__global__ void __launch_bounds__(kThreads) radius_fill_kernel(GraphArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t s_rows[kThreads / 32][2][kRowSmem];   // each warp's two rows while they are short
    const int p = blockIdx.x / kGraphSplit, part = blockIdx.x % kGraphSplit;
    const int a0 = a.atom_off[p];
    const int N = a.atom_off[p + 1] - a0;
    if (N < 1 || N > a.max_atoms || a0 < 0) return;
    CellList cl;
    build_cells(a, a0, N, smem, cl);
    const float c2 = __fmul_rn(a.cut_cov, a.cut_cov);
    const float n2 = __fmul_rn(a.cut_nc, a.cut_nc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int i0, i1;
    part_range(N, part, i0, i1);
    for (int i = i0 + warp; i < i1; i += kThreads / 32) {
        const int n0 = a.deg[0][a0 + i], n1 = a.deg[1][a0 + i];   // 0 for a pose over capacity
        int32_t *r0 = a.col[0] + a.beg[0][a0 + i];
        int32_t *r1 = a.col[1] + a.beg[1][a0 + i];
        const float xi = cl.sx[i], yi = cl.sy[i], zi = cl.sz[i];
        // rows of at most kRowSmem entries are packed and sorted in this warp's shared-memory rows, longer
        // ones in place in global memory
        int32_t *w0 = n0 <= kRowSmem ? s_rows[warp][0] : r0;
        int32_t *w1 = n1 <= kRowSmem ? s_rows[warp][1] : r1;
        int k0 = 0, k1 = 0;
        int q0r, prer;
        const int total = cand_seq(cl, cl.cell[i], lane, q0r, prer);
        for (int base = 0; base < total; base += 32) {
            const int q = cand_at(base + lane, q0r, prer);
            bool h0 = false, h1 = false;
            int j = 0;
            if (base + lane < total) {
                j = cl.sorted[q];
                if (j != i) {
                    const float s = dist2_rn(xi, yi, zi, cl.sx[j], cl.sy[j], cl.sz[j]);
                    h0 = s < c2;
                    h1 = !h0 && s < n2;
                }
            }
            const unsigned b0 = __ballot_sync(0xffffffffu, h0), b1 = __ballot_sync(0xffffffffu, h1);
            if (h0 && k0 + __popc(b0 & below) < n0) w0[k0 + __popc(b0 & below)] = a0 + j;
            if (h1 && k1 + __popc(b1 & below) < n1) w1[k1 + __popc(b1 & below)] = a0 + j;
            k0 += __popc(b0);
            k1 += __popc(b1);
        }
        __syncwarp();
        warp_sort_row(w0, n0, lane, r0);
        warp_sort_row(w1, n1, lane, r1);
    }
}

}  // namespace

size_t radius_graph_smem(int max_atoms) {
    return (size_t)max_atoms * 3 * 4 + (size_t)max_atoms * 2 * 4 + (size_t)(kCells + 1) * 4 + (size_t)kCells * 4;
}

void launch_radius_graph(const GraphArgs &a, cudaStream_t s) {
    const size_t sm = radius_graph_smem(a.max_atoms);
    cudaFuncSetAttribute(radius_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(radius_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    radius_count_kernel<<<a.n_poses * kGraphSplit, kThreads, sm, s>>>(a);
    radius_scan_kernel<<<a.n_poses, kThreads, (size_t)(a.max_atoms + 1) * 4, s>>>(a);
    radius_fill_kernel<<<a.n_poses * kGraphSplit, kThreads, sm, s>>>(a);
}

}  // namespace fusion
