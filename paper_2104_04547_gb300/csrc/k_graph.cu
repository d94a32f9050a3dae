// Radius graph with two edge types (Section 1: edge types at distinct distance
// thresholds for covalent and non-covalent interactions; Table II cutoffs).
//
// One CTA per pose.  The pose's coordinates go to shared memory, atoms are
// counting-sorted into a cell list with cells no smaller than the
// non-covalent cutoff (so every neighbour lies in the 27 surrounding cells),
// then a count pass, a block-wide exclusive scan and a fill pass write CSR
// rows, and each row is sorted by neighbour index so the output is canonical.
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
constexpr int kThreads = 512;

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

__global__ void __launch_bounds__(kThreads) radius_graph_kernel(GraphArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int p = blockIdx.x;
    const int a0 = a.atom_off[p];
    const int N = a.atom_off[p + 1] - a0;
    const int MA = a.max_atoms;
    const int tid = threadIdx.x;
    if (N < 1 || N > MA || a0 < 0) return;   // flagged by the prep kernel

    float *sx = reinterpret_cast<float *>(smem);
    float *sy = sx + MA;
    float *sz = sy + MA;
    int *s_cell = reinterpret_cast<int *>(sz + MA);   // [MA]
    int *s_sorted = s_cell + MA;                      // [MA] atoms in cell order
    int *s_d0 = s_sorted + MA;                        // [MA + 1] covalent degree -> offset
    int *s_d1 = s_d0 + MA + 1;                        // [MA + 1] non-covalent degree -> offset
    int *s_start = s_d1 + MA + 1;                     // [kCells + 1]
    int *s_cur = s_start + kCells + 1;                // [kCells]
    __shared__ float s_red[6][kThreads / 32];
    __shared__ float s_lo[3], s_L[3];
    __shared__ int s_dim[3];
    __shared__ int s_tmp[33];

    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = tid; i < N; i += kThreads) {
        const float x = a.xyz[(size_t)(a0 + i) * 3], y = a.xyz[(size_t)(a0 + i) * 3 + 1], z = a.xyz[(size_t)(a0 + i) * 3 + 2];
        sx[i] = x; sy[i] = y; sz[i] = z;
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
    for (int c = tid; c <= kCells; c += kThreads) s_start[c] = 0;
    __syncthreads();
    if (tid < 3) {
        float l = INFINITY, h = -INFINITY;
        for (int w = 0; w < kThreads / 32; ++w) { l = fminf(l, s_red[tid][w]); h = fmaxf(h, s_red[3 + tid][w]); }
        const float ext = h - l;
        float L = a.cut_nc * 1.001f + 1e-4f;
        if (ext / L > (float)(kGridCellsMax - 1)) L = ext / (float)(kGridCellsMax - 1) * 1.001f;
        int dim = (int)(ext / L) + 1;
        if (dim > kGridCellsMax) dim = kGridCellsMax;
        s_lo[tid] = l; s_L[tid] = L; s_dim[tid] = dim;
    }
    __syncthreads();
    for (int i = tid; i < N; i += kThreads) {
        const int cx = max(0, min((int)((sx[i] - s_lo[0]) / s_L[0]), s_dim[0] - 1));
        const int cy = max(0, min((int)((sy[i] - s_lo[1]) / s_L[1]), s_dim[1] - 1));
        const int cz = max(0, min((int)((sz[i] - s_lo[2]) / s_L[2]), s_dim[2] - 1));
        const int c = (cz * s_dim[1] + cy) * s_dim[0] + cx;
        s_cell[i] = c;
        atomicAdd(&s_start[c], 1);
    }
    __syncthreads();
    const int ncell = s_dim[0] * s_dim[1] * s_dim[2];
    block_exscan(s_start, ncell + 1, s_tmp);
    for (int c = tid; c < ncell; c += kThreads) s_cur[c] = s_start[c];
    __syncthreads();
    for (int i = tid; i < N; i += kThreads) {
        const int pos = atomicAdd(&s_cur[s_cell[i]], 1);
        s_sorted[pos] = i;
    }
    __syncthreads();

    const float c2 = __fmul_rn(a.cut_cov, a.cut_cov);
    const float n2 = __fmul_rn(a.cut_nc, a.cut_nc);

    // count pass
    for (int i = tid; i < N; i += kThreads) {
        const int c = s_cell[i];
        const int cx = c % s_dim[0], cy = (c / s_dim[0]) % s_dim[1], cz = c / (s_dim[0] * s_dim[1]);
        int d0 = 0, d1 = 0;
        for (int oz = -1; oz <= 1; ++oz) {
            const int zz = cz + oz;
            if (zz < 0 || zz >= s_dim[2]) continue;
            for (int oy = -1; oy <= 1; ++oy) {
                const int yy = cy + oy;
                if (yy < 0 || yy >= s_dim[1]) continue;
                for (int ox = -1; ox <= 1; ++ox) {
                    const int xx = cx + ox;
                    if (xx < 0 || xx >= s_dim[0]) continue;
                    const int cc = (zz * s_dim[1] + yy) * s_dim[0] + xx;
                    for (int q = s_start[cc]; q < s_start[cc + 1]; ++q) {
                        const int j = s_sorted[q];
                        if (j == i) continue;
                        const float s = dist2_rn(sx[i], sy[i], sz[i], sx[j], sy[j], sz[j]);
                        if (s < c2) ++d0;
                        else if (s < n2) ++d1;
                    }
                }
            }
        }
        s_d0[i] = d0;
        s_d1[i] = d1;
    }
    if (tid == 0) { s_d0[N] = 0; s_d1[N] = 0; }
    __syncthreads();
    const int tot0 = block_exscan(s_d0, N + 1, s_tmp);
    const int tot1 = block_exscan(s_d1, N + 1, s_tmp);
    const long long cap = (long long)N * a.max_degree;
    const size_t base = (size_t)a0 * a.max_degree;
    if (tot0 > cap || tot1 > cap) {
        if (tid == 0) atomicOr(a.err, FUSION_ERR_EDGES);
        for (int i = tid; i < N; i += kThreads) {
            a.beg[0][a0 + i] = (int)base; a.deg[0][a0 + i] = 0;
            a.beg[1][a0 + i] = (int)base; a.deg[1][a0 + i] = 0;
        }
        return;
    }

    // fill pass, then sort each row by neighbour index
    for (int i = tid; i < N; i += kThreads) {
        const int c = s_cell[i];
        const int cx = c % s_dim[0], cy = (c / s_dim[0]) % s_dim[1], cz = c / (s_dim[0] * s_dim[1]);
        int32_t *r0 = a.col[0] + base + s_d0[i];
        int32_t *r1 = a.col[1] + base + s_d1[i];
        const int n0 = s_d0[i + 1] - s_d0[i], n1 = s_d1[i + 1] - s_d1[i];
        int k0 = 0, k1 = 0;
        for (int oz = -1; oz <= 1; ++oz) {
            const int zz = cz + oz;
            if (zz < 0 || zz >= s_dim[2]) continue;
            for (int oy = -1; oy <= 1; ++oy) {
                const int yy = cy + oy;
                if (yy < 0 || yy >= s_dim[1]) continue;
                for (int ox = -1; ox <= 1; ++ox) {
                    const int xx = cx + ox;
                    if (xx < 0 || xx >= s_dim[0]) continue;
                    const int cc = (zz * s_dim[1] + yy) * s_dim[0] + xx;
                    for (int q = s_start[cc]; q < s_start[cc + 1]; ++q) {
                        const int j = s_sorted[q];
                        if (j == i) continue;
                        const float s = dist2_rn(sx[i], sy[i], sz[i], sx[j], sy[j], sz[j]);
                        if (s < c2) { if (k0 < n0) r0[k0++] = a0 + j; }
                        else if (s < n2) { if (k1 < n1) r1[k1++] = a0 + j; }
                    }
                }
            }
        }
        for (int u = 1; u < n0; ++u) {
            const int v = r0[u];
            int w = u - 1;
            while (w >= 0 && r0[w] > v) { r0[w + 1] = r0[w]; --w; }
            r0[w + 1] = v;
        }
        for (int u = 1; u < n1; ++u) {
            const int v = r1[u];
            int w = u - 1;
            while (w >= 0 && r1[w] > v) { r1[w + 1] = r1[w]; --w; }
            r1[w + 1] = v;
        }
        a.beg[0][a0 + i] = (int)(base + s_d0[i]);
        a.deg[0][a0 + i] = n0;
        a.beg[1][a0 + i] = (int)(base + s_d1[i]);
        a.deg[1][a0 + i] = n1;
    }
}

}  // namespace

size_t radius_graph_smem(int max_atoms) {
    return (size_t)max_atoms * 3 * 4 + (size_t)max_atoms * 2 * 4 + (size_t)(max_atoms + 1) * 2 * 4 +
           (size_t)(kCells + 1) * 4 + (size_t)kCells * 4;
}

void launch_radius_graph(const GraphArgs &a, cudaStream_t s) {
    const size_t sm = radius_graph_smem(a.max_atoms);
    cudaFuncSetAttribute(radius_graph_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    radius_graph_kernel<<<a.n_poses, kThreads, sm, s>>>(a);
}

}  // namespace fusion
