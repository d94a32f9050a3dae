/*
 * fusion.h - C ABI of the GB300 Coherent Fusion pose-scoring library.
 *
 * The library scores docked protein-ligand poses with a Coherent Fusion model
 * (a 3D-CNN over a voxel grid and a spatial-graph CNN, fused by dense layers;
 * Section 2.2, Fig. 1 and Section 3.3 of "High-Throughput Virtual Screening of
 * Small Molecule Inhibitors for SARS-CoV-2 Protein Targets with Deep Fusion
 * Models").  The output of each pose is a predicted binding affinity in pK
 * units (Eq. 1).  Every step of the scoring path runs in CUDA kernels compiled
 * for sm_103a; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *  - Return value: FUSION_OK (0) or a negative FUSION_E* code; the message of
 *    the last failure on the calling thread is in fusion_last_error().
 *  - The library never keeps a caller pointer after a call returns.
 *  - On error, outputs are left untouched and the model stays usable.
 */
#ifndef FUSION_H
#define FUSION_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define FUSION_OK            0
#define FUSION_EINVAL       -1  /* bad argument, descriptor or pose (NaN/Inf coordinate, n_lig outside [1, N], N above capacity) */
#define FUSION_EWEIGHTS     -2  /* weights blob length differs from fusion_weights_bytes(desc) */
#define FUSION_ENOMEM       -3  /* device or pinned-host allocation failed */
#define FUSION_ECAPACITY    -4  /* a device capacity flag was raised (edge capacity of a pose exceeded) */
#define FUSION_ECUDA        -5  /* a CUDA runtime call failed */
#define FUSION_ETIMEOUT     -6  /* a bounded device wait ran out */
#define FUSION_EUNSUPPORTED -7  /* descriptor valid but not supported by this library (dtype or shape) */
#define FUSION_EAGAIN       -8  /* server: queue full, or the result is not ready yet */

/* Compute dtypes of the CNN contractions (density, distances, pooling and head stay FP32). */
#define FUSION_F32  0
#define FUSION_BF16 1
#define FUSION_FP8  2

/* Edge-type bits of a graph-convolution stage (Section 1, Table II: covalent and non-covalent edges). */
#define FUSION_EDGE_COV 1
#define FUSION_EDGE_NC  2

/* Ligand gather kinds (Section 3.3.1, PotentialNet gather). */
#define FUSION_GATHER_LINEAR 0   /* sum_i (W h_i + b) over ligand atoms i */
#define FUSION_GATHER_GATED  1   /* sum_i sigmoid(W_g [h_i, x_i] + b_g) * (W_o h_i + b_o) */

/* Fusion forms (Section 2.2 and Section 3.3.3): how the two branch latents become an affinity. */
#define FUSION_COHERENT 0   /* fusion layers on [cnn latent, sg latent] (Table V) */
#define FUSION_MID      1   /* model-specific dense layers on each latent first, their outputs appended
                               to the latents, then the fusion layers (Mid-level Fusion, Table IV) */
#define FUSION_LATE     2   /* mean of the two branches' own affinities (Late Fusion); no fusion layers */

#define FUSION_MAX_CONV   8
#define FUSION_MAX_STAGES 2
#define FUSION_MAX_HEAD   6

/* One 3D convolution (Section 3.3.1, Table III): same padding k/2, bias, ReLU.
 * residual != 0: y = x + ReLU(conv(x)) (needs c_in == c_out and stride 1). */
typedef struct {
    int32_t c_in, c_out, k, stride, residual;
} fusion_conv_desc;

/* Model description.  Layer widths and kernel sizes follow the paper's
 * hyper-parameter tables (Tables I-III, V); all fields are plain values. */
typedef struct {
    int32_t n_feat;            /* atom features per atom = grid channels; must be 19 */
    int32_t grid_n;            /* voxels per grid side (4..96) */
    float   grid_h;            /* voxel edge, Angstrom (> 0) */
    float   sigma;             /* Gaussian width of an atom's density, Angstrom (> 0) */
    int32_t support;           /* k: an atom reaches voxels within +-k of its own voxel (1..5) */
    int32_t n_conv;            /* number of conv layers (1..FUSION_MAX_CONV) */
    fusion_conv_desc conv[FUSION_MAX_CONV];
    int32_t pool;              /* 2: 2^3 max-pool stride 2 after the convs; 0 or 1: none */
    int32_t cnn_dense;         /* width of the CNN dense layer (ReLU) */
    int32_t sg_hidden;         /* H: node-state width (32 or 64) */
    int32_t sg_n_stages;       /* graph-convolution stages (1 or 2) */
    int32_t sg_steps[FUSION_MAX_STAGES];  /* GRU steps per stage (0..16) */
    int32_t sg_edges[FUSION_MAX_STAGES];  /* FUSION_EDGE_* bits used by each stage */
    int32_t sg_gate;           /* 1: per-node gate between stage 0 and stage 1 */
    int32_t sg_gather;         /* FUSION_GATHER_* */
    int32_t sg_gather_width;   /* G: width of the SG latent (<= 256) */
    float   cut_cov;           /* covalent cutoff, Angstrom */
    float   cut_nc;            /* non-covalent cutoff, Angstrom (> cut_cov) */
    int32_t n_head;            /* fusion (head) layers (1..FUSION_MAX_HEAD; 0 for FUSION_LATE) */
    int32_t head[FUSION_MAX_HEAD];  /* output widths (<= 1024); the last must be 1 */
    int32_t dtype;             /* FUSION_F32 / FUSION_BF16 / FUSION_FP8 */
    int32_t max_poses;         /* batch capacity of one fusion_score call */
    int32_t max_atoms;         /* atom capacity of one pose (<= 4096) */
    int32_t max_degree;        /* edge capacity per atom and edge type (mean over a pose) */
    int32_t keep_stages;       /* 1: keep every intermediate for fusion_fetch_stage (more memory) */
    int32_t fusion;            /* FUSION_COHERENT / FUSION_MID / FUSION_LATE */
    int32_t n_cnn_out;         /* branch layers on the CNN latent (0 for coherent; >= 1 otherwise) */
    int32_t cnn_out[FUSION_MAX_HEAD];  /* their widths (late: the last must be 1) */
    int32_t n_sg_out;          /* branch layers on the SG latent, as n_cnn_out */
    int32_t sg_out[FUSION_MAX_HEAD];
    int32_t head_residual;     /* 1: a hidden fusion layer whose input and output widths match returns
                                  x + SELU(W x + b) */
    int32_t cnn_dense2;        /* 0, or the width of a second CNN dense layer (ReLU) after the first
                                  (Section 3.3.1: the first reduced by a factor of 2); the CNN latent the
                                  fusion layers and branches read is then its output, the 3D-CNN's last
                                  hidden layer Layer^{M-1} (Section 2.2).  cnn_dense must then be a multiple
                                  of 8 */
    int32_t sg_width[FUSION_MAX_STAGES];  /* node-state width of each stage (0 = sg_hidden; at most
                                  sg_hidden; stage 0 at least n_feat).  The gate maps stage 0's states to
                                  stage 1's width (Table II: the covalent gather width), so unequal widths
                                  need sg_gate; the GPU carries every stage at sg_hidden with the extra
                                  channels held at exactly zero */
} fusion_model_desc;

/* A batch of poses in packed structure-of-arrays form.  Ligand atoms come
 * first in each pose.  Caller-owned, read-only during the call. */
typedef struct {
    int32_t        n_poses;
    const int32_t *atom_off;   /* [n_poses + 1]: atoms of pose p are [atom_off[p], atom_off[p+1]); atom_off[0] == 0 */
    const int32_t *n_lig;      /* [n_poses]: ligand atoms of pose p are its first n_lig[p] atoms */
    const float   *xyz;        /* [atom_off[n_poses]][3] float32 coordinates, Angstrom */
    const float   *feat;       /* [atom_off[n_poses]][19] float32 atom features */
    int32_t        on_device;  /* 0: host pointers (copied in); 1: device pointers valid on the model's stream */
} fusion_poses;

typedef struct fusion_model fusion_model;

/* Bytes of the weights blob for `desc`: every tensor row-major float32
 * little-endian, no header, in this order (PyTorch shape conventions):
 *   per conv i: W [c_out][c_in][k][k][k], b [c_out]
 *   CNN dense: W [cnn_dense][C*S*S*S] (input in (C, D, H, W) flatten order of the pooled map), b
 *   if cnn_dense2: W [cnn_dense2][cnn_dense], b [cnn_dense2]
 *   per stage s (H = the stage's width w_s): per edge type present (covalent first): W_e [H][H], b_e [H];
 *                GRU W_ih [3H][H], W_hh [3H][H], b_ih [3H], b_hh [3H] (gate rows reset, update, new);
 *                if sg_gate and s is not the last stage: W_i [w_{s+1}][H + w_0], b_i [w_{s+1}],
 *                W_j [w_{s+1}][H], b_j [w_{s+1}]
 *   gather (H = the last stage's width): gated: W_g [G][2H], b_g [G], W_o [G][H], b_o [G];
 *                                        linear: W [G][H], b [G]
 *   per CNN branch layer l: W [out][in], b [out]  (in = the CNN latent width for l = 0)
 *   per SG branch layer l: W [out][in], b [out]   (in = G for l = 0)
 *   per head layer l: W [out][in], b [out]  (in = CNN latent width + G for l = 0, plus the last CNN and
 *                                            SG branch widths for FUSION_MID)
 * The CNN latent width is cnn_dense2 when nonzero, else cnn_dense.
 * Branch layers: FUSION_MID applies SELU after each; FUSION_LATE applies ReLU between them, the last
 * linear, and averages the two branch outputs.  Fusion layers: SELU between, the last linear.
 * Returns 0 if the descriptor is invalid. */
size_t fusion_weights_bytes(const fusion_model_desc *desc);

/* Create a model on the current CUDA device.  Copies and reformats the
 * weights to device memory and allocates the workspace for max_poses poses of
 * max_atoms atoms.  `cuda_stream` is a cudaStream_t the model launches on
 * (NULL: the model creates and owns a non-blocking stream).  `*out` receives
 * the model (owned by the library until fusion_destroy). */
int fusion_create(const fusion_model_desc *desc, const void *weights, size_t weights_bytes,
                  void *cuda_stream, fusion_model **out);

/* Score `n_poses` poses (Section 4.2: each pose gets a predicted affinity):
 * voxelize, 3D-CNN, radius graph, gated graph convolution, ligand gather and
 * fusion head.  `out_affinity` is [n_poses] float32: a host pointer when
 * poses->on_device == 0, a device pointer when 1.  Returns after the results
 * are written (synchronous on the model's stream).  n_poses == 0 is a no-op. */
int fusion_score(fusion_model *m, const fusion_poses *poses, int32_t n_poses, float *out_affinity);

/* Free the model and everything it allocated.  NULL-safe. */
void fusion_destroy(fusion_model *m);

/* Message of the last failure on the calling thread ("" if none). */
const char *fusion_last_error(void);

/* ---- diagnostics: intermediate results of the last fusion_score call ---- */

#define FUSION_STAGE_ORIGIN      1   /* float[3] grid origin of pose `index` */
#define FUSION_STAGE_GRID        2   /* float[n][n][n][19] voxel grid of pose `index` (z, y, x, c) */
#define FUSION_STAGE_CONV        3   /* float[S][S][S][C] output of conv layer (index >> 16) for pose (index & 0xffff); needs keep_stages */
#define FUSION_STAGE_POOL        4   /* float[S][S][S][C] pooled map of pose `index` */
#define FUSION_STAGE_CNN_LATENT  5   /* float[cnn_dense] of pose `index` */
#define FUSION_STAGE_EDGES_COV   6   /* int32 row_ptr[N+1] then col[E], local atom indices, of pose `index` */
#define FUSION_STAGE_EDGES_NC    7   /* same for non-covalent edges */
#define FUSION_STAGE_SG_STATE    8   /* float[N][H] final node states of pose `index` */
#define FUSION_STAGE_SG_LATENT   9   /* float[G] of pose `index` */
#define FUSION_STAGE_AFFINITY   10   /* float[n_poses] */

/* Bytes that fusion_fetch_stage would write (negative status on error). */
int64_t fusion_stage_bytes(fusion_model *m, int32_t stage, int32_t index);

/* Copy an intermediate of the last fusion_score call into the host buffer
 * `dst` of `bytes` bytes (must be >= fusion_stage_bytes). */
int fusion_fetch_stage(fusion_model *m, int32_t stage, int32_t index, void *dst, size_t bytes);

/* Device time in milliseconds of each kernel group of the last fusion_score
 * call, measured with CUDA events on the model's stream.  Index:
 *   0 pose prep (validation, grid origin, per-atom weights)   1 voxelize
 *   2..9 conv layer 0..7 (FP8: with the layer's input quantization)   10 max-pool
 *   11 CNN dense                                              12 radius graph
 *   13 graph-convolution steps                                14 ligand gather
 *   15 fusion head                                            16 whole forward pass
 * Entries 12-14 are elapsed times on the model's second stream, where the
 * graph branch runs concurrently with the grid branch (so they overlap the
 * conv entries).  Entries of absent layers are 0; with CUDA graphs only
 * entry 16 is measured.
 * `n` entries are written (n <= 17). */
int fusion_last_timings(fusion_model *m, float *out, int32_t n);

/* ---- batching: options and tile autotuning ---- */

#define FUSION_OPT_CUDA_GRAPH 1   /* value 1: fusion_score replays a CUDA graph of the whole device-side
                                     forward pass, captured on first use for each batch size (inputs are
                                     copied into the model's own buffers first); 0: plain launches */
#define FUSION_OPT_CONV_SLICES_PER_MMA 2   /* tensor-core convs: value 1, 2, 4 or 8 = every layer has each MMA
                                              serve that many adjacent output slices (N = value x output
                                              channels; 8 only for 32-channel layers at 16 slices per CTA;
                                              FUSION_EUNSUPPORTED where a layer cannot), -1 = the default per
                                              layer (for stride-1 layers 8 at 16 slices per CTA, else 4 where
                                              it fits, else 2, else 1; 1 for stride 2).  Re-plans the layers
                                              and drops captured graphs; scores are the same in every mode */

#define FUSION_OPT_TEST_WAIT_TIMEOUT 3   /* value 1: test of failure detection.  In the next fusion_score
                                            call the first tensor-core conv launch loads nothing, so its
                                            bounded waits run out (about 1 s): the call returns
                                            FUSION_ETIMEOUT with the output untouched, and later calls are
                                            normal.  Nothing faults or hangs.  FUSION_EUNSUPPORTED on the
                                            FP32 path or with CUDA graphs on.  Value 2: the same for the
                                            first tensor-core graph launch (its weight copy is not issued);
                                            FUSION_EUNSUPPORTED unless the graph runs on the tensor cores */

#define FUSION_OPT_GRAPH_NODES_PER_WARP 4   /* graph convolution (gated graph steps and stage transforms on
                                               the CUDA cores; the message sums alone with the graph on the
                                               tensor cores): value 1, 2, 4 or 8 nodes per warp, each weight
                                               load serving them all; -1 = the default, 2 with the graph on the
                                               tensor cores, else 4.  Every node's sums keep their
                                               order, so scores are the same for every value.  Drops
                                               captured graphs.  Any dtype */
#define FUSION_OPT_SERIAL_BRANCHES 5   /* measurement mode: value 1 runs the graph branch after the grid
                                          branch on one stream, so fusion_last_timings gives each stage's
                                          kernel time alone (normally the branches overlap on two streams);
                                          0 restores the default.  Scores are the same.  Drops captured
                                          graphs.  Any dtype */

#define FUSION_OPT_GRAPH_TENSOR_CORES 6   /* graph convolution: value 1 runs the stage gate, each gated step's
                                            GRU update and the edge transforms (Section 3.3.1) on the tcgen05
                                            tensor cores, 128 nodes per tile, each product as three BF16 MMAs
                                            of the operands' BF16 high and low parts with FP32 accumulation
                                            (each product within 3 x 2^-16 of FP32's; node states within
                                            about 1e-3 of the FP32 path's after 9 steps); 0 runs them on the CUDA
                                            cores in FP32; -1 = the default, 1 for BF16 / FP8 models and 0
                                            for FP32 ones.  The message sums stay in their order either way.
                                            Drops captured graphs.  Any dtype */

#define FUSION_OPT_CONV_STRIDE2_SPLIT 7   /* tensor-core convs: value 1 (the default, also -1) = a stride-2
                                             layer after the first with an even input size reads its input
                                             parity-split (the previous layer's epilogue, or the FP8
                                             quantizer, stores the 8 sub-grids of one coordinate parity
                                             apart, each channel-blocked), so each parity phase's halo is one
                                             TMA box of whole W-lines; 0 = it reads NDHWC through the TMA
                                             element stride of 2.  The MMAs and their order are the same, so
                                             scores and conv maps are the same in both modes.  Re-plans the
                                             layers and drops captured graphs; FUSION_EUNSUPPORTED on the
                                             FP32 path */

/* Set a runtime option of a model (FUSION_OPT_*). */
int fusion_set_option(fusion_model *m, int32_t option, int64_t value);

/* Pick, for every conv layer of a tensor-core model (bf16 / fp8), the
 * fastest tile configuration (output slices per CTA, output slices per MMA,
 * kernel-offset groups per weight stage, weight stages) by timing
 * every configuration that fits shared memory on the given batch (scored once
 * first); the sweep's winner replaces the layer's default only if, timed
 * against it three more times in alternation, its best time is at least 2%
 * under the default's.  Then the graph convolution's nodes per warp (1, 2, 4, 8) by timing
 * whole scoring calls of the batch, since that branch runs beside the
 * convolutions.  Every configuration sums each output in the same order, so
 * the scores do not change.  Replaces the layer plans and the graph schedule;
 * captured graphs are dropped.  FUSION_EUNSUPPORTED on the FP32 path. */
int fusion_autotune(fusion_model *m, const fusion_poses *poses, int32_t n_poses);

/* The graph convolution's current nodes per warp (FUSION_OPT_GRAPH_NODES_PER_WARP, or the autotuner's
 * choice) into *nodes_per_warp.  FUSION_EINVAL on NULL arguments. */
int fusion_graph_schedule(fusion_model *m, int32_t *nodes_per_warp);

/* Tile configuration of conv `layer`: out5 = {output slices per CTA, (ty, tx)
 * kernel-offset groups per weight stage, weight stages, shared-memory bytes,
 * adjacent output slices each MMA serves (1, 2 or 4; N = that x output
 * channels)}.  FUSION_EUNSUPPORTED on the FP32 path. */
int fusion_describe_conv(fusion_model *m, int32_t layer, int32_t *out5);

/* ---- aggregation ----
 * The paper ranks compounds by their strongest predicted affinity over all of
 * their docked poses at a binding site (Section 4.4: the maximum for
 * Coherent Fusion).  Given the affinities of n poses and the compound (or
 * compound and site) index of each pose, best[c] = max over poses i of
 * compound c of affinity[i] and best_pose[c] = the smallest such i attaining
 * it; a compound with no poses gets best = -INFINITY and best_pose = -1.
 * Host arrays: affinity [n], compound [n] with values in [0, n_compounds),
 * best [n_compounds], best_pose [n_compounds] (may be NULL).  FUSION_EINVAL
 * on a NULL array, a compound index out of range or a NaN affinity (nothing
 * is written then).  Runs on the host; needs no device. */
int fusion_best_per_compound(const float *affinity, const int32_t *compound, int32_t n, int32_t n_compounds,
                             float *best, int32_t *best_pose);

/* ---- serving: continuous batching request loop ----
 * The paper scores a job's poses in fixed batches and writes every result at
 * job end, noting that results should be written as they are computed
 * (Section 4.3).  A server scores poses one by one as they arrive: requests are
 * queued, and each of its slots (a model replica with its own workspace and
 * stream) repeatedly takes the queued poses (waiting at most batch_window_us
 * for max_batch of them) and scores them as one batch.  While one slot's batch
 * runs on the GPU, the other slots take the requests that arrived meanwhile,
 * so batches overlap on the device.  A pose's result does not depend on the
 * poses it was batched with. */
typedef struct {
    int32_t slots;             /* slots (batches in flight); 0 = up to 4, as the HBM budget admits */
    int32_t max_batch;         /* poses per batch, 1 .. desc->max_poses */
    double  batch_window_us;   /* longest wait for a batch to fill once a request is queued */
    size_t  hbm_budget_bytes;  /* device memory the slots may use; 0 = no limit */
    int32_t queue_capacity;    /* poses that may wait in the queues; beyond it submit returns FUSION_EAGAIN */
    int32_t dtypes;            /* mask of (1 << FUSION_F32 / FUSION_BF16 / FUSION_FP8): the dtypes the server
                                  runs slots of, besides desc->dtype (0 = desc->dtype only); slots cycle
                                  through them, at least one slot per dtype */
} fusion_server_config;

typedef struct {
    int32_t slots;             /* slots admitted */
    size_t  slot_bytes;        /* measured device footprint of one slot */
    int64_t submitted, completed, rejected, failed, batches, queued, inflight;
    double  gpu_busy_s;        /* summed wall time of the slots' scoring calls */
    int32_t slots_by_dtype[3]; /* slots admitted per dtype (FUSION_F32, FUSION_BF16, FUSION_FP8) */
} fusion_server_stats;

typedef struct fusion_server fusion_server;

/* Start a server on the current device: creates the slots (model replicas from
 * desc and the weights blob, desc->max_poses >= cfg->max_batch) and one worker
 * thread per slot. */
int fusion_server_create(const fusion_model_desc *desc, const void *weights, size_t weights_bytes,
                         const fusion_server_config *cfg, fusion_server **out);

/* Queue one pose (host arrays xyz[n_atoms][3], feat[n_atoms][19], ligand atoms
 * first; copied before return) for scoring in desc->dtype.  *ticket identifies
 * its result.  Invalid poses return FUSION_EINVAL; a full queue returns
 * FUSION_EAGAIN. */
int fusion_server_submit(fusion_server *s, const float *xyz, const float *feat, int32_t n_atoms, int32_t n_lig,
                         uint64_t *ticket);

/* As fusion_server_submit, scored by a slot of `dtype` (FUSION_F32 / FUSION_BF16
 * / FUSION_FP8), which must be one the server runs (FUSION_EINVAL otherwise).
 * A pose's result depends only on the pose and its dtype, not on the poses it
 * is batched with. */
int fusion_server_submit_dtype(fusion_server *s, const float *xyz, const float *feat, int32_t n_atoms,
                               int32_t n_lig, int32_t dtype, uint64_t *ticket);

/* Non-blocking: FUSION_OK with the affinity and the latency from submission
 * to completion (seconds) once the pose is scored (each result is returned
 * once), FUSION_EAGAIN while it is pending; FUSION_EINVAL for a ticket this
 * server never issued or whose result was already collected. */
int fusion_server_poll(fusion_server *s, uint64_t ticket, float *affinity, double *latency_s);

/* Wait until every submitted pose is scored (FUSION_ETIMEOUT after timeout_s). */
int fusion_server_drain(fusion_server *s, double timeout_s);

int fusion_server_get_stats(fusion_server *s, fusion_server_stats *out);

/* Stop: finishes queued work, joins the workers, frees the slots.  NULL-safe. */
void fusion_server_destroy(fusion_server *s);

/* ---- dense layer without any allocation ----
 * The paper has no counterpart to this entry point; it serves deployment.
 *
 * y[b][n] = act(bias[n] + sum_k x[b][k] * w[n][k]) for b < B, n < N (act =
 * ReLU when relu != 0, identity otherwise): the CNN dense layer of
 * fusion_score, run as the same split-K kernels, for callers that cannot
 * allocate device memory.  Such callers include a serving process that admits
 * requests against a device-memory budget it does not own, a host application
 * whose own allocator owns every byte of the device, and a latency-bound
 * request loop that cannot take the implicit synchronisation and unbounded
 * latency of cudaMalloc / cudaFree.  The call allocates nothing: the split-K
 * partials go to a fixed 8 MiB array that the library keeps in every GPU
 * that loads it until the process exits.
 *
 * x: device float32 [B][K]; w: device float32 [N][K]; bias: device float32 [N];
 * y: device float32 [B][N]; all caller-owned.  x and w must be 16-byte
 * aligned (they are read 16 bytes at a time), bias and y 4-byte aligned;
 * other pointers return FUSION_EINVAL before anything is launched.  K must be a positive multiple
 * of 8, and splits(K) x B x N must fit FUSION_NOALLOC_MAX_PARTIALS floats,
 * where splits(K) = clamp(K / 2048, 1, 128); larger sizes return FUSION_EINVAL
 * with a message naming the limit.  The kernels are enqueued on `cuda_stream`
 * (a cudaStream_t; NULL is the legacy default stream) and the call returns
 * without waiting for them.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  The address is kept until the
 * process exits and does not survive cudaDeviceReset: do not call this entry
 * point again after resetting the device.  A CUDA error already pending when
 * the call starts is returned as FUSION_ECUDA and nothing is launched.  Every call shares the one array:
 * calls whose kernels overlap on the GPU race and must be serialised by the
 * caller (for example by issuing them on one stream).  Nothing in the array
 * needs clearing between calls. */
#define FUSION_NOALLOC_MAX_PARTIALS (1 << 21)
int fusion_cnn_dense_noalloc(const float *x, const float *w, const float *bias, int32_t B, int32_t N, int32_t K,
                             int32_t relu, float *y, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FUSION_H */
