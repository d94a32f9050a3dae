// Spatial-graph CNN: PotentialNet-style gated graph convolution (Section
// 3.3.1, Table II; Gated Graph Sequence Neural Networks and PotentialNet are
// the architectures it cites).
//
//   h0 = atom features zero-padded to H
//   per step of a stage: m_i = sum over the stage's edge types e, neighbours j of (W_e h_j + b_e)
//                        h_i <- GRU(m_i, h_i)        (gate rows reset, update, new)
//   between stages:      h_i <- sigmoid(W_i [h_i, h0_i] + b_i) * (W_j h_i + b_j)
//   ligand gather:       sum over ligand atoms of sigmoid(W_g [h_i, x_i] + b_g) * (W_o h_i + b_o)
//                        (x_i = input of the last stage), or sum of (W h_i + b)
//
// A warp takes a few consecutive nodes (sharing each weight load); lane l owns
// features l and l + 32 of each.  The per-edge-type transforms W_e h_j + b_e
// are computed once per node and step (sg_transform_kernel at a stage start,
// then by the previous step), so a step is a segment sum over the sorted CSR
// row in a fixed order followed by the GRU matrix-vector products, all
// deterministic.  The gather is one CTA per
// pose and 32 outputs: warps take ligand atoms round robin and the warp
// partials are added in warp order.
#include "fusion_internal.cuh"

namespace fusion {

namespace {

constexpr int kWarps = 8;

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ __forceinline__ float f4(const float4 &x, int i) { return i == 0 ? x.x : i == 1 ? x.y : i == 2 ? x.z : x.w; }

// T = W_e x + b_e for the warp's NP nodes, x = v[n][0..H).  Lane l computes outputs o = l + 32 j; its weights
// for input k are the H/32 floats at we_p[(k * 32 + l) * H/32] (one 8- or 4-byte load), and the node vectors
// are read four inputs at a time from shared memory.  Every sum runs from the bias over k ascending.
template <int H, int NP>
__device__ __forceinline__ void edge_transform(const float (*v)[2 * H], const float *we_p, const float *be, int lane,
                                               int np, int i0, float *T) {
    constexpr int HJ = H / 32;
    float t[NP][HJ];
#pragma unroll
    for (int j = 0; j < HJ; ++j) {
        const float b = be[lane + 32 * j];
#pragma unroll
        for (int n = 0; n < NP; ++n) t[n][j] = b;
    }
    const float *wl = we_p + lane * HJ;
    for (int k0 = 0; k0 < H; k0 += 4) {
        float4 x[NP];
#pragma unroll
        for (int n = 0; n < NP; ++n) x[n] = *reinterpret_cast<const float4 *>(&v[n][k0]);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            float w[HJ];
            if constexpr (HJ == 2) {
                const float2 q = __ldg(reinterpret_cast<const float2 *>(wl + (size_t)(k0 + kk) * 32 * HJ));
                w[0] = q.x;
                w[1] = q.y;
            } else {
                w[0] = __ldg(wl + (size_t)(k0 + kk) * 32 * HJ);
            }
#pragma unroll
            for (int n = 0; n < NP; ++n) {
                const float xk = f4(x[n], kk);
#pragma unroll
                for (int j = 0; j < HJ; ++j) t[n][j] = fmaf(w[j], xk, t[n][j]);
            }
        }
    }
#pragma unroll
    for (int n = 0; n < NP; ++n)
#pragma unroll
        for (int j = 0; j < HJ; ++j)
            if (n < np) T[(size_t)(i0 + n) * H + lane + 32 * j] = t[n][j];
}

// A warp takes NP consecutive nodes (1, 2, 4 or 8; SgStepArgs::nodes_per_warp): the matrix-vector products
// load each weight once for all of them, while every node's sums keep the order of a warp per node, so the
// results do not depend on NP.  The weights are packed in the order a lane reads them (its GRU weights for
// one input in 16-byte loads, its edge-transform weights in one 8-byte load), so the L1 weight reads that
// bounded these kernels take a quarter of the load instructions.

template <int H, int NP>
__global__ void __launch_bounds__(kWarps * 32) sg_transform_kernel(SgTransformArgs a) {
    constexpr int HJ = H / 32;
    __shared__ __align__(16) float sv[kWarps][NP][2 * H];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int A = a.A_dev ? *a.A_dev : a.A;
    const int i0 = (blockIdx.x * kWarps + warp) * NP;
    if (i0 >= A) return;
    const int np = min(NP, A - i0);          // nodes of this warp (the rest of the NP slots are zero)
    float (*v)[2 * H] = sv[warp];
#pragma unroll
    for (int n = 0; n < NP; ++n)
#pragma unroll
        for (int j = 0; j < HJ; ++j) {
            const int o = lane + 32 * j;
            const size_t i = (size_t)(i0 + n);
            v[n][H + o] = (n < np && o < kFeat) ? a.feat[i * kFeat + o] : 0.f;
            v[n][o] = (n < np && !a.init) ? a.h_in[i * H + o] : 0.f;
        }
    __syncwarp();
    float x[NP][HJ];
#pragma unroll
    for (int j = 0; j < HJ; ++j) {
        const int o = lane + 32 * j;
        if (a.init) {
#pragma unroll
            for (int n = 0; n < NP; ++n) x[n][j] = v[n][H + o];
        } else if (a.gi_t) {
            float u[NP], w[NP];
#pragma unroll
            for (int n = 0; n < NP; ++n) { u[n] = a.gbi[o]; w[n] = a.gbj[o]; }
            for (int k = 0; k < 2 * H; ++k) {
                const float g = a.gi_t[k * H + o];
#pragma unroll
                for (int n = 0; n < NP; ++n) u[n] = fmaf(g, v[n][k], u[n]);
            }
            for (int k = 0; k < H; ++k) {
                const float g = a.gj_t[k * H + o];
#pragma unroll
                for (int n = 0; n < NP; ++n) w[n] = fmaf(g, v[n][k], w[n]);
            }
#pragma unroll
            for (int n = 0; n < NP; ++n) x[n][j] = sigm(u[n]) * w[n];
        } else {
#pragma unroll
            for (int n = 0; n < NP; ++n) x[n][j] = v[n][o];
        }
    }
    __syncwarp();
#pragma unroll
    for (int n = 0; n < NP; ++n)
#pragma unroll
        for (int j = 0; j < HJ; ++j) {
            const int o = lane + 32 * j;
            v[n][o] = x[n][j];
            if (n < np) a.h_out[(size_t)(i0 + n) * H + o] = x[n][j];
        }
    __syncwarp();
    for (int e = 0; e < 2; ++e)
        if (a.we_p[e]) edge_transform<H, NP>(v, a.we_p[e], a.be[e], lane, np, i0, a.T[e]);
}

// Blocks per SM the step kernel is compiled for: four at H = 64 and up to four nodes per warp (64 registers),
// since the message sums are latency-bound and need the warps (at 80 registers, three blocks, the
// paper-final model's calls took 3% longer); the other shapes state no minimum (0) and keep the registers
// the compiler gives them.
template <int H, int NP>
constexpr int step_min_blocks() { return (H == 64 && NP <= 4) ? 4 : 0; }

// Messages of the warp's NP nodes i0 .. i0 + np: the segment sum of the neighbours' transforms, edge type by
// edge type, each node's row in order.  The nodes walk their rows side by side (the q-th neighbour of every
// node per iteration), so NP neighbour rows are in flight at once; every node still adds its own neighbours in
// row order, so the sums do not depend on NP.  Lane l holds features l + 32 j of each node's message.
template <int H, int NP>
__device__ __forceinline__ void message_sums(const SgStepArgs &a, int lane, int i0, int np, float (&m)[NP][H / 32]) {
    constexpr int HJ = H / 32;
#pragma unroll
    for (int n = 0; n < NP; ++n)
#pragma unroll
        for (int j = 0; j < HJ; ++j) m[n][j] = 0.f;
    for (int e = 0; e < 2; ++e) {
        if (!a.T_in[e]) continue;
        const float *T = a.T_in[e];
        // lane n < NP holds node n's row start and degree
        const int rb = lane < np ? a.beg[e][i0 + lane] : 0;
        const int rd = lane < np ? a.deg[e][i0 + lane] : 0;
        int dmax = rd;
        for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        for (int q0 = 0; q0 < dmax; q0 += 32) {
            int jl[NP];
#pragma unroll
            for (int n = 0; n < NP; ++n) {
                const int bn = __shfl_sync(0xffffffffu, rb, n), dn = __shfl_sync(0xffffffffu, rd, n);
                jl[n] = (q0 + lane < dn) ? a.col[e][bn + q0 + lane] : -1;
            }
            const int nq = min(32, dmax - q0);
#pragma unroll 2
            for (int q = 0; q < nq; ++q) {
#pragma unroll
                for (int n = 0; n < NP; ++n) {
                    const int jn = __shfl_sync(0xffffffffu, jl[n], q);
                    if (jn >= 0) {                         // warp-uniform: q0 + q < the node's degree
#pragma unroll
                        for (int j = 0; j < HJ; ++j) m[n][j] += __ldg(T + (size_t)jn * H + lane + 32 * j);
                    }
                }
            }
        }
    }
}

// The messages alone, written to m_out [A][H] (the tensor-core GRU reads them).
template <int H, int NP>
__global__ void __launch_bounds__(kWarps * 32) sg_message_kernel(SgStepArgs a, float *m_out) {
    constexpr int HJ = H / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int A = a.A_dev ? *a.A_dev : a.A;
    const int i0 = (blockIdx.x * kWarps + warp) * NP;
    if (i0 >= A) return;
    const int np = min(NP, A - i0);
    float m[NP][HJ];
    message_sums<H, NP>(a, lane, i0, np, m);
#pragma unroll
    for (int n = 0; n < NP; ++n)
#pragma unroll
        for (int j = 0; j < HJ; ++j)
            if (n < np) m_out[(size_t)(i0 + n) * H + lane + 32 * j] = m[n][j];
}

template <int H, int NP>
__global__ void __launch_bounds__(kWarps * 32, step_min_blocks<H, NP>()) sg_step_kernel(SgStepArgs a) {
    constexpr int HJ = H / 32;
    __shared__ __align__(16) float sv[kWarps][NP][2 * H];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int A = a.A_dev ? *a.A_dev : a.A;
    const int i0 = (blockIdx.x * kWarps + warp) * NP;
    if (i0 >= A) return;
    const int np = min(NP, A - i0);          // nodes of this warp (the rest of the NP slots are zero)
    float (*v)[2 * H] = sv[warp];

    float m[NP][HJ];
    message_sums<H, NP>(a, lane, i0, np, m);
#pragma unroll
    for (int n = 0; n < NP; ++n)
#pragma unroll
        for (int j = 0; j < HJ; ++j) {
            const int o = lane + 32 * j;
            v[n][o] = m[n][j];
            v[n][H + o] = n < np ? a.h_in[(size_t)(i0 + n) * H + o] : 0.f;
        }
    __syncwarp();
    // GRU.  Lane l owns outputs o = l + 32 j of each gate, one j at a time (24 accumulators at NP = 4, so
    // four blocks fit an SM and the latency-bound message sums keep their warps).  Its weights for input k
    // and output o are six consecutive floats of its P (W_ih rows r, z, n, then W_hh rows r, z, n, at row
    // o), read as one 16-byte and one 8-byte load; the node vectors [m, h] are read four inputs at a time.
    // Every sum runs from the bias over k ascending.
    constexpr int P = (6 * HJ + 3) / 4 * 4;
    const float *wl = a.gru_p + lane * P;
    float hn[NP][HJ];
#pragma unroll
    for (int j = 0; j < HJ; ++j) {
        const int o = lane + 32 * j;
        float acc[NP][6];
        {
            float b[6];
#pragma unroll
            for (int g = 0; g < 3; ++g) { b[g] = a.bih[g * H + o]; b[3 + g] = a.bhh[g * H + o]; }
#pragma unroll
            for (int n = 0; n < NP; ++n)
#pragma unroll
                for (int q = 0; q < 6; ++q) acc[n][q] = b[q];
        }
        for (int k0 = 0; k0 < H; k0 += 4) {
            float4 xm[NP], xh[NP];
#pragma unroll
            for (int n = 0; n < NP; ++n) {
                xm[n] = *reinterpret_cast<const float4 *>(&v[n][k0]);
                xh[n] = *reinterpret_cast<const float4 *>(&v[n][H + k0]);
            }
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float *wk = wl + (size_t)(k0 + kk) * 32 * P + 6 * j;   // 16-byte aligned at even j
                float w[6];
                if (j % 2 == 0) {
                    const float4 t = __ldg(reinterpret_cast<const float4 *>(wk));
                    const float2 u = __ldg(reinterpret_cast<const float2 *>(wk + 4));
                    w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w; w[4] = u.x; w[5] = u.y;
                } else {
                    const float2 t = __ldg(reinterpret_cast<const float2 *>(wk));
                    const float4 u = __ldg(reinterpret_cast<const float4 *>(wk + 2));
                    w[0] = t.x; w[1] = t.y; w[2] = u.x; w[3] = u.y; w[4] = u.z; w[5] = u.w;
                }
#pragma unroll
                for (int n = 0; n < NP; ++n) {
                    const float mk = f4(xm[n], kk), hk = f4(xh[n], kk);
#pragma unroll
                    for (int g = 0; g < 3; ++g) {
                        acc[n][g] = fmaf(w[g], mk, acc[n][g]);
                        acc[n][3 + g] = fmaf(w[3 + g], hk, acc[n][3 + g]);
                    }
                }
            }
        }
#pragma unroll
        for (int n = 0; n < NP; ++n) {
            const float r = sigm(acc[n][0] + acc[n][3]);
            const float z = sigm(acc[n][1] + acc[n][4]);
            const float nn = tanhf(acc[n][2] + r * acc[n][5]);
            hn[n][j] = (1.f - z) * nn + z * v[n][H + o];
            if (n < np) a.h_out[(size_t)(i0 + n) * H + o] = hn[n][j];
        }
    }
    if (!a.T_out[0] && !a.T_out[1]) return;
    __syncwarp();
#pragma unroll
    for (int n = 0; n < NP; ++n)
#pragma unroll
        for (int j = 0; j < HJ; ++j) v[n][lane + 32 * j] = hn[n][j];
    __syncwarp();
    for (int e = 0; e < 2; ++e)
        if (a.T_out[e]) edge_transform<H, NP>(v, a.we_p[e], a.be[e], lane, np, i0, a.T_out[e]);
}

// One CTA per (pose, 32 gather outputs): lane l computes output g = 32 blockIdx.y + l; the warps take the
// pose's ligand atoms round robin and their partials are added in warp order, so every output's sum has the
// same order whatever the gather width.  A warp evaluates its next four atoms together (four independent
// multiply-add chains per lane) and adds them to its partial in atom order.
constexpr int kGatherAtoms = 4;

template <int H>
__global__ void __launch_bounds__(kWarps * 32) sg_gather_kernel(SgGatherArgs a) {
    __shared__ float sv[kWarps][kGatherAtoms][2 * H];
    __shared__ float part[kWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x;
    const int g = blockIdx.y * 32 + lane;
    const int a0 = a.atom_off[p];
    const int N = a.atom_off[p + 1] - a0;
    int nl = a.n_lig[p];
    if (nl > N || nl < 0) nl = 0;      // invalid pose: flagged by the prep kernel
    const int G = a.G;
    const bool on = g < G;
    const int gc = on ? g : 0;         // a valid column for the loads of idle lanes
    float acc = 0.f;
    float (*v)[2 * H] = sv[warp];
    for (int i0 = warp; i0 < nl; i0 += kWarps * kGatherAtoms) {
        int na = 0;                    // atoms of this group: i0, i0 + 8, ... below nl
#pragma unroll
        for (int t = 0; t < kGatherAtoms; ++t) {
            const int i = i0 + t * kWarps;
            if (i < nl) {
                const size_t ai = (size_t)a0 + i;
                for (int o = lane; o < H; o += 32) {
                    v[t][o] = a.h[ai * H + o];
                    v[t][H + o] = a.x[ai * H + o];
                }
                na = t + 1;
            }
        }
        __syncwarp();
        float w[kGatherAtoms], u[kGatherAtoms];
#pragma unroll
        for (int t = 0; t < kGatherAtoms; ++t) {
            w[t] = a.bo[gc];
            u[t] = a.gated ? a.bg[gc] : 0.f;   // the linear gather has no gate (bg, wg_t are null)
        }
#pragma unroll 4
        for (int k = 0; k < H; ++k) {
            const float wk = __ldg(a.wo_t + k * G + gc);
#pragma unroll
            for (int t = 0; t < kGatherAtoms; ++t) w[t] = fmaf(wk, v[t][k], w[t]);
        }
        if (a.gated) {
#pragma unroll 4
            for (int k = 0; k < 2 * H; ++k) {
                const float wk = __ldg(a.wg_t + k * G + gc);
#pragma unroll
                for (int t = 0; t < kGatherAtoms; ++t) u[t] = fmaf(wk, v[t][k], u[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < kGatherAtoms; ++t)
            if (t < na) acc += a.gated ? sigm(u[t]) * w[t] : w[t];
        __syncwarp();
    }
    part[warp][lane] = acc;
    __syncthreads();
    if (threadIdx.x < 32 && on) {
        float s = 0.f;
        for (int w = 0; w < kWarps; ++w) s += part[w][lane];
        a.out[(size_t)p * G + g] = s;
    }
}

}  // namespace

template <int H, int NP>
void launch_transform_np(const SgTransformArgs &a, cudaStream_t s) {
    const int blocks = (a.A + kWarps * NP - 1) / (kWarps * NP);
    sg_transform_kernel<H, NP><<<blocks, kWarps * 32, 0, s>>>(a);
}

template <int H, int NP>
void launch_step_np(const SgStepArgs &a, cudaStream_t s) {
    const int blocks = (a.A + kWarps * NP - 1) / (kWarps * NP);
    sg_step_kernel<H, NP><<<blocks, kWarps * 32, 0, s>>>(a);
}

template <int H, int NP>
void launch_message_np(const SgStepArgs &a, float *m, cudaStream_t s) {
    const int blocks = (a.A + kWarps * NP - 1) / (kWarps * NP);
    sg_message_kernel<H, NP><<<blocks, kWarps * 32, 0, s>>>(a, m);
}

template <int H>
void launch_message_h(const SgStepArgs &a, float *m, cudaStream_t s) {
    switch (a.nodes_per_warp) {
    case 1: launch_message_np<H, 1>(a, m, s); break;
    case 2: launch_message_np<H, 2>(a, m, s); break;
    case 8: launch_message_np<H, 8>(a, m, s); break;
    default: launch_message_np<H, 4>(a, m, s); break;
    }
}

template <int H>
void launch_transform_h(const SgTransformArgs &a, cudaStream_t s) {
    switch (a.nodes_per_warp) {
    case 1: launch_transform_np<H, 1>(a, s); break;
    case 2: launch_transform_np<H, 2>(a, s); break;
    case 8: launch_transform_np<H, 8>(a, s); break;
    default: launch_transform_np<H, 4>(a, s); break;
    }
}

template <int H>
void launch_step_h(const SgStepArgs &a, cudaStream_t s) {
    switch (a.nodes_per_warp) {
    case 1: launch_step_np<H, 1>(a, s); break;
    case 2: launch_step_np<H, 2>(a, s); break;
    case 8: launch_step_np<H, 8>(a, s); break;
    default: launch_step_np<H, 4>(a, s); break;
    }
}

void launch_sg_transform(const SgTransformArgs &a, cudaStream_t s) {
    if (a.H == 64) launch_transform_h<64>(a, s);
    else launch_transform_h<32>(a, s);
}

void launch_sg_step(const SgStepArgs &a, cudaStream_t s) {
    if (a.H == 64) launch_step_h<64>(a, s);
    else launch_step_h<32>(a, s);
}

void launch_sg_message(const SgStepArgs &a, float *m, cudaStream_t s) {
    if (a.H == 64) launch_message_h<64>(a, m, s);
    else launch_message_h<32>(a, m, s);
}

void launch_sg_gather(const SgGatherArgs &a, cudaStream_t s) {
    const dim3 grid(a.B, (a.G + 31) / 32);
    if (a.H == 64) sg_gather_kernel<64><<<grid, kWarps * 32, 0, s>>>(a);
    else sg_gather_kernel<32><<<grid, kWarps * 32, 0, s>>>(a);
}

}  // namespace fusion
