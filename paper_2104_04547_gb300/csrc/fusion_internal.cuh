// Internal declarations shared by the CUDA translation units of the library.
// Layouts in device memory (all row-major, batch outermost):
//   grid / activations: NDHWC, [pose][z][y][x][channel], channels padded to `cx`
//   conv weights (FP32 path): [k^3 offset][c_in padded][c_out]
//   graph: per edge type, per atom i: beg[i], deg[i]; col[beg .. beg+deg) global atom indices, sorted
//   node states: [atom][H]
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/fusion.h"

#define FUSION_ERR_INPUT     1u   // invalid pose data seen on the device
#define FUSION_ERR_EDGES     2u   // edge capacity of a pose exceeded
#define FUSION_ERR_TIMEOUT   4u   // a bounded wait ran out

namespace fusion {

constexpr int kFeat = 19;
constexpr int kMaxSupportW = 11;     // 2k+1 for k <= 5
constexpr int kGridCellsMax = 16;    // graph cell list: at most 16 cells per axis

// ---- pose prep + voxelize -------------------------------------------------

struct PrepArgs {
    const int32_t *atom_off;
    const int32_t *n_lig;
    const float *xyz;
    const float *feat;    // [A][19]
    int n_poses;
    int max_atoms;
    int grid_n;
    float h, sigma;
    int k;
    float *origin;        // [B][3]
    unsigned *err;
    // 1 A voxel-cell list of each pose: the atoms whose support cube meets the grid, sorted by containing
    // voxel (z, y, x) over the extended range [-k, n-1+k]^3 and then by atom index.  Record j of pose p
    // (atom_rec + (atom_off[p] + j) * atom_rec_floats(k)) is the j-th atom in that order: its containing
    // voxel and pose as int (cz, cy, cx, p), its 3 x (2k+1) axis weights (z, y, x; zero-padded to a multiple
    // of 4) and its 19 features + one zero.  cell_row[p][(cz + k) R + (cy + k)] (R = n + 2k) is where the
    // (cz, cy) row of cells starts, cell_row[p][R^2] the number of listed atoms.
    int32_t *cell_row;    // [B][cell_row_stride(n, k)]
    float *atom_rec;      // [A][atom_rec_floats(k)]
};
// Entries of one pose's cell-row index: (n + 2k)^2 + 1.
inline int cell_row_stride(int n, int k) { return (n + 2 * k) * (n + 2 * k) + 1; }
// Floats of an atom record: 4 (voxel, pose) + 3 (2k+1) weights rounded up to a multiple of 4 + 20 features.
__host__ __device__ inline int atom_rec_wpad(int k) { return (3 * (2 * k + 1) + 3) & ~3; }
__host__ __device__ inline int atom_rec_floats(int k) { return 4 + atom_rec_wpad(k) + 20; }
void launch_prep(const PrepArgs &a, cudaStream_t s);

struct VoxArgs {
    const int32_t *atom_off;
    int n_poses;
    int grid_n;
    int k;
    int max_atoms;
    void *out;            // [B][n][n][n][cx]
    int cx;               // padded channel count of the output layout
    int out_bf16;         // 0: float32, 1: bfloat16
    int fold_pad;         // bf16 only: -1 = plain channels; p >= 0 = channels 16..18 folded along x:
                          // channel 16 + 3 s + f of voxel x holds feature 16 + f of voxel x - p + s
                          // (s = 0..4, zero outside the grid), channel 31 zero
    int blocked;          // bf16 only: store channel-blocked, [B][n][n][cx / 8][n][8]
    const int32_t *cell_row;     // PrepArgs::cell_row
    const float *atom_rec;       // PrepArgs::atom_rec (records in cell order)
    float *amax;          // bf16 only, may be null: per-pose max |stored value| (atomic max; zeroed by the caller)
};
void launch_voxelize(const VoxArgs &a, cudaStream_t s);

// ---- 3D-CNN ----------------------------------------------------------------

struct ConvArgs {
    const float *x;       // [B][n_in]^3[cx_in]
    const float *w;       // [k^3][cx_in][c_out]
    const float *bias;    // [c_out]
    float *y;             // [B][n_out]^3[c_out]
    int B, n_in, n_out, cx_in, c_out, k, stride, pad, residual;
};
void launch_conv3d_f32(const ConvArgs &a, cudaStream_t s);

struct PoolArgs {
    const void *x; void *y;
    int B, n_in, n_out, c;
    int bf16;
};
void launch_maxpool(const PoolArgs &a, cudaStream_t s);

struct DenseArgs {
    const void *x;        // [B][K] (float or bf16)
    const void *w;        // [N][K] (float or bf16)
    const float *bias;    // [N]
    float *part;          // [splits][B][N]
    float *y;             // [B][N]
    int B, N, K, splits;
    int bf16;
    int relu;
};
void launch_dense(const DenseArgs &a, cudaStream_t s);
int dense_splits(int K);
// The fixed-order split reduction + bias + activation of launch_dense, on partials [splits][B][N].
void launch_dense_reduce(const DenseArgs &a, cudaStream_t s);

// Tensor-core (tcgen05) bf16 CNN dense: a plan holds the TMA tensor maps of the model's pooled-input
// buffer x [max_poses][K] and weights w [N][K]; launch writes the FP32 split partials [splits][B][N].
struct DenseTcPlan {
    struct Impl;
    Impl *impl;
    DenseTcPlan();
    ~DenseTcPlan();
    DenseTcPlan(const DenseTcPlan &) = delete;
    DenseTcPlan &operator=(const DenseTcPlan &) = delete;
};
int dense_tc_splits(int K, int N);
int dense_tc_plan(DenseTcPlan &plan, const void *x, const void *w, int max_poses, int N, int K, unsigned *err,
                  char *why, size_t why_len);
void dense_tc_launch(DenseTcPlan &plan, int B, float *part, cudaStream_t s);

// Tensor-core (tcgen05) BF16 conv: a plan per layer holds the TMA tensor map of
// the layer's input buffer and the launch geometry.
struct ConvTcPlan {
    struct Impl;
    Impl *impl;
    ConvTcPlan();
    ~ConvTcPlan();
    ConvTcPlan(const ConvTcPlan &) = delete;
    ConvTcPlan &operator=(const ConvTcPlan &) = delete;
};
// Output slices per CTA for a layer with c_out output channels.
int conv_tc_tile_slices(int c_out);
// Bytes of the arranged weights of one layer (elem = 2 for bf16, 1 for FP8 E4M3; fold: 0 plain input,
// 1 the bf16 grid with channels 16..18 folded along x (VoxArgs::fold_pad), 2 the FP8 folded grid of
// launch_quantize_fold_fp8).
size_t conv_tc_weight_bytes(int cin_pad, int c_out, int k, int stride, int elem, int fold);
// Whether a first layer can read an x-folded grid (19 channels in 32, stride 1, k in {3, 5, 7}).
bool conv_tc_fold_ok(int c_in, int cin_pad, int k, int stride, int elem);
// Blob conv weights [co][ci][k][k][k] -> [channel chunk][phase][ty][tx][16-byte half][tz = nz-1..0][co][16 bytes];
// FP8 also returns the per-output-channel scales s_w[c_out] (weights = stored code * s_w).
void conv_tc_arrange_weights(const float *w, int c_out, int c_in, int cin_pad, int k, int stride, int elem,
                             int fold, uint8_t *out, float *s_w);
struct ConvTcSpec {
    const void *x;          // input (bf16 or FP8) [max_poses][n_in]^3[cin_pad], read by TMA
    int elem;               // 2 = bf16, 1 = FP8 E4M3
    int max_poses, n_in, cin_pad;
    const void *w;          // arranged weights
    const float *bias;      // [c_out]
    const float *s_w;       // FP8: weight scales [c_out]
    const float *s_in;      // FP8: per-pose input scales [max_poses]
    float *amax;            // FP8: per-pose max |output| (atomic max), or null
    const void *xres;       // bf16 residual source [max_poses][n_in]^3[cres]
    int cres;
    void *y;                // bf16 output [max_poses][n_out]^3[c_out]
    int n_out, c_out, k, stride, residual;
    unsigned *err;
    int T;                  // output slices per CTA (0: default for c_out)
    int groups_per_stage;   // (ty, tx) kernel-offset groups per weight stage (0: about 48 KB per stage)
    int nbs;                // weight stages in the ring (0: 2)
    int group;              // output slices per MMA (1, 2, 4; N = group x c_out); <= 0: default for the layer
    int fold;               // x-folded first-layer input: 0 no, 1 bf16 grid (VoxArgs::fold_pad = k / 2),
                            // 2 FP8 grid of launch_quantize_fold_fp8 (cin_pad 64, stored from x = -1)
    int blocked;            // 1: input stored channel-blocked, [pose][z][y][16-byte channel block][x][16 bytes],
                            // so a halo row is hw x 16 contiguous bytes (one TMA box row per 16-byte block and
                            // W-line instead of one per voxel); stride 1 only.  2: parity-split (stride 2, n_in
                            // even, no fold): the blocked layout of each of the 8 sub-grids of one coordinate
                            // parity, [pose][(z&1) 4 + (y&1) 2 + (x&1)][z/2][y/2][block][x/2][16 bytes], so that
                            // each parity phase's halo is one plain box of whole W-lines
    int out_blocked;        // write the bf16 output 1: channel-blocked, [pose][z][y][c_out / 8][x][8];
                            // 2: parity-split, [pose][8][n_out/2][n_out/2][c_out / 8][n_out/2][8] (n_out even)
    int res_blocked;        // the bf16 residual source is channel-blocked, [pose][z][y][cres / 8][x][8]
};
// Build the plan; returns 0, or nonzero with a reason in `why`.
int conv_tc_plan(ConvTcPlan &plan, const ConvTcSpec &spec, char *why, size_t why_len);
void conv_tc_launch(ConvTcPlan &plan, int B, cudaStream_t s);
// Test of the bounded waits: the plan's next launch issues no loads, so its waits run out (about 1 s)
// and it sets FUSION_ERR_TIMEOUT; later launches are normal.
void conv_tc_stall_next(ConvTcPlan &plan);
void conv_tc_describe(const ConvTcPlan &plan, int *T, int *groups_per_stage, int *nbs, size_t *smem, int *group);

// Per-pose FP8 quantization of the plain bf16 grid [B][n]^3[32] (channels 0..18) into the folded layout
// the first FP8 conv reads, [B][n][n][n + 1][64]: stored voxel j holds channels 0..15 of grid voxels
// j - 1 and j (slots 0..31), and channels 16..18 of voxels j - 1 - p + s, s = 0 .. 2p (slots 32 + 3 s + f),
// zero outside the grid and in the unused slots; codes use the per-pose scale of launch_quantize_per_pose.
// blocked != 0: the same codes stored channel-blocked, [B][n][n][4][n + 1][16] (see ConvTcSpec::blocked).
void launch_quantize_fold_fp8(const void *grid_bf16, void *q_fp8, int B, int n, int p, const float *amax,
                              float *scale, int blocked, cudaStream_t s);
// Per-pose FP8 quantization of bf16 NDHWC activations (per_pose elements per pose, a multiple of 8).
void launch_amax_per_pose(const void *x_bf16, int B, size_t per_pose, float *amax, cudaStream_t s);
void launch_quantize_per_pose(const void *x_bf16, void *q_fp8, int B, size_t per_pose, const float *amax, float *scale,
                              cudaStream_t s);
// The same codes for bf16 NDHWC activations [B][n]^3[C] (C a multiple of 16), stored channel-blocked:
// [B][n][n][C / 16][n][16] (z, y, 16-channel block, x, channel in block).  split != 0 and n even: stored
// parity-split (ConvTcSpec::blocked 2), [B][8][h][h][C / 16][h][16] with h = n / 2 and sub-grid
// (z&1) 4 + (y&1) 2 + (x&1); an odd n is stored channel-blocked.
void launch_quantize_blocked(const void *x_bf16, void *q_fp8, int B, int n, int C, const float *amax, float *scale,
                             int split, cudaStream_t s);

// ---- radius graph ----------------------------------------------------------

struct GraphArgs {
    const int32_t *atom_off;
    const float *xyz;
    int n_poses;
    int max_atoms;
    int max_degree;
    float cut_cov, cut_nc;
    int32_t *beg[2], *deg[2], *col[2];   // 0 covalent, 1 non-covalent
    unsigned *err;
};
void launch_radius_graph(const GraphArgs &a, cudaStream_t s);
size_t radius_graph_smem(int max_atoms);

// ---- SG-CNN ----------------------------------------------------------------

struct SgTransformArgs {
    const float *feat;     // [A][19]
    const float *h_in;     // [A][H] (unused in init mode)
    float *h_out;          // [A][H]: the stage input written here
    float *T[2];           // [A][H] per edge type slot
    const float *we_p[2];  // edge transforms, [k][lane][H/32]: W_e[lane + 32 j][k] (nullptr: slot unused)
    const float *be[2];
    const float *gi_t, *gbi, *gj_t, *gbj;   // gate ([2H][H], [H], [H][H], [H]); nullptr: no gate
    int A, H;
    int init;              // 1: stage input = h0 (features zero-padded to H)
    const int32_t *A_dev;  // non-null: the atom count is *A_dev (A is then the launch capacity)
    int nodes_per_warp;    // 1, 2, 4 or 8 (anything else: 4); the results do not depend on it
};
void launch_sg_transform(const SgTransformArgs &a, cudaStream_t s);

struct SgStepArgs {
    const float *h_in;     // [A][H]
    float *h_out;          // [A][H]
    const float *T_in[2];  // neighbour transforms of this step (nullptr: slot unused)
    float *T_out[2];       // transforms of h_out for the next step (nullptr: not needed)
    const int32_t *beg[2], *deg[2], *col[2];   // edges of each slot
    const float *gru_p;    // GRU weights, [k][lane][P]: per j, W_ih[gH + o][k] then W_hh[gH + o][k] (g = 0..2,
                           // o = lane + 32 j), zero-padded to P = 6H/32 rounded up to a multiple of 4
    const float *bih, *bhh;                     // GRU biases [3H], [3H]
    const float *we_p[2], *be[2];               // for T_out (layout as SgTransformArgs::we_p)
    int A, H;
    const int32_t *A_dev;  // non-null: the atom count is *A_dev (A is then the launch capacity)
    int nodes_per_warp;    // 1, 2, 4 or 8 (anything else: 4); the results do not depend on it
};
void launch_sg_step(const SgStepArgs &a, cudaStream_t s);
// The step's messages alone (the sums of sg_step_kernel, same order) into m [A][H].
void launch_sg_message(const SgStepArgs &a, float *m, cudaStream_t s);

// The step's GRU update and the next step's transforms on the tensor cores (k_sgcnn_tc.cu), from the
// messages of launch_sg_message.
struct SgGruTcArgs {
    const float *m;        // [A][H] messages
    const float *h_in;     // [A][H]
    float *h_out;          // [A][H]
    float *T_out[2];       // [A][H] transforms of h_out for the next step (nullptr: not needed)
    const uint16_t *w;     // the stage's weight image (sg_gru_tc_pack), 16-byte aligned
    const float *bih, *bhh;   // GRU biases [3H], [3H]
    const float *be[2];       // transform biases [H] of the T_out slots
    int A, H;              // H = 32 or 64
    const int32_t *A_dev;  // non-null: the atom count is *A_dev (A is then the launch capacity)
    unsigned *err;
    int stall;             // test of the bounded waits: no weight copy is issued, so the first wait runs out
};
void launch_sg_gru_tc(const SgGruTcArgs &a, cudaStream_t s);
// Sets the tensor-core graph kernels' shared-memory limits and sizes their persistent grids (call before
// any capture).
void sg_gru_tc_prepare(int H);

// A stage's input and first transforms on the tensor cores (k_sgcnn_tc.cu): x = the gate of the previous
// stage's states and h0 (wg set), or h0 (h_in null), or h_in; T_e = W_e x + b_e.
struct SgStageTcArgs {
    const float *feat;     // [A][19]
    const float *h_in;     // [A][H] previous stage's final states (nullptr: the first stage, x = h0)
    float *x_out;          // [A][H] the stage input (may be h_in: each row is read before it is written)
    float *T_out[2];       // [A][H] transforms of x (nullptr: not needed)
    const uint16_t *wg;    // gate image (sg_stage_tc_pack), nullptr: no gate
    const uint16_t *we;    // the stage's two W_e slots, laid out as in the GRU image (its last 4 H^2 values)
    const float *gbi, *gbj;   // gate biases [H]
    const float *be[2];       // transform biases [H] of the T_out slots
    int A, H;
    const int32_t *A_dev;
    unsigned *err;
    int stall;             // as SgGruTcArgs::stall
};
void launch_sg_stage_tc(const SgStageTcArgs &a, cudaStream_t s);
// The gate image: BF16 hi / lo parts of [W_i columns of h ; W_j] ([2H][H]) then of W_i's columns of h0
// ([H][H]), K-major; wi is the padded [H][2H] gate matrix, wj [H][H]; sg_stage_tc_image_elems(H) values.
size_t sg_stage_tc_image_elems(int H);
void sg_stage_tc_pack(const float *wi, const float *wj, int H, uint16_t *img);
// The weight image of a stage: BF16 hi / lo parts of W_ih and W_hh ([3H][H]) and of the two transform
// slots' W_e ([H][H]; nullptr: zeros), each part K-major [H/8][rows][8]; sg_gru_tc_image_elems(H) values.
size_t sg_gru_tc_image_elems(int H);
void sg_gru_tc_pack(const float *wih, const float *whh, const float *we0, const float *we1, int H, uint16_t *img);

struct SgGatherArgs {
    const int32_t *atom_off;
    const int32_t *n_lig;
    const float *h;        // [A][H] final node states
    const float *x;        // [A][H] input of the last stage
    const float *wg_t, *bg;   // gated: [2H][G], [G]
    const float *wo_t, *bo;   // [H][G], [G] (linear gather: the only matrix)
    float *out;            // [B][G]
    int B, H, G, gated;
};
void launch_sg_gather(const SgGatherArgs &a, cudaStream_t s);

// ---- head ------------------------------------------------------------------

constexpr int kHeadMaxWidth = 1024;
struct HeadArgs {
    const float *cnn;      // [B][Dc]
    const float *sg;       // [B][G]
    const float *wt[FUSION_MAX_HEAD];   // fusion layers, [in][out] transposed
    const float *b[FUSION_MAX_HEAD];
    int width[FUSION_MAX_HEAD];
    int n_layers;
    const float *bwt[2][FUSION_MAX_HEAD];   // branch layers (0: CNN latent, 1: SG latent), [in][out]
    const float *bb[2][FUSION_MAX_HEAD];
    int bwidth[2][FUSION_MAX_HEAD];
    int n_branch[2];
    int mode;              // FUSION_COHERENT / FUSION_MID / FUSION_LATE
    int residual;          // hidden fusion layers with equal widths add their input
    int B, Dc, G;
    float *out;            // [B]
};
void launch_head(const HeadArgs &a, cudaStream_t s);

// Record `msg` as the calling thread's fusion_last_error() message; returns `code`.
int set_last_error(int code, const char *msg);

}  // namespace fusion
