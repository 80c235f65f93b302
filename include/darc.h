/*
 * darc.h -- C ABI of libdarc.so, a GB300 (sm_103a) implementation of the hot
 * path of DARC, "Diffeomorphic Atlas Registration via Coordinate descent"
 * (Zou et al., arXiv 2508.10743): the per-subject update of Eq. 3 (scaling
 * and squaring, warp, MSE or local NCC plus the diffusion regulariser of
 * Eq. 2, the adjoint of all of these, Adam), the centrality activation, the
 * atlas re-estimate, and one-shot label propagation (Eq. oneshot).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - A volume has D x H x W voxels (z, y, x), x fastest, V = D*H*W.
 *  - An image is float32 [V].  A field (velocity v, displacement u,
 *    gradient) is planar float32 [3][V]; channel a is the component along
 *    axis a (0 = z, 1 = y, 2 = x), in voxel units.  A batch of B images or
 *    fields is stored subject after subject: [B][V] or [B][3][V].
 *  - Every pointer named *_dev is CUDA device memory of the current device;
 *    *_host is host memory.  The caller owns every buffer it passes; the
 *    library keeps no pointer past the call, except the cohort, which keeps
 *    `images_dev` until darc_destroy.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Calls enqueue work on it and return without waiting,
 *    unless they write a *_host output.
 *  - Sampling is trilinear with border padding: each coordinate of the
 *    sample point x + u(x) is clamped to [0, n_a - 1] (the paper does not
 *    define the interpolation; this is the reading taken).
 *  - Return value: DARC_OK (0) or a negative darc_status.  On an argument
 *    or shape error nothing is enqueued and no state changes.
 *    darc_last_error() returns a thread-local message for the last failure.
 */
#ifndef DARC_H_
#define DARC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DARC_OK = 0,
    DARC_ERR_ARG = -1,        /* null pointer, bad index, bad option          */
    DARC_ERR_SHAPE = -2,      /* a dimension < 2, an even or oversized window */
    DARC_ERR_OOM = -3,        /* device allocation failed                      */
    DARC_ERR_CUDA = -4,       /* a CUDA call failed (message has the detail)   */
    DARC_ERR_NONFINITE = -5,  /* a loss came out NaN/Inf; that step's update was skipped */
    DARC_ERR_IO = -6,         /* darc_save / darc_load file error              */
    DARC_ERR_INTERNAL = -7
} darc_status;

/* Dissimilarities (Sec. "Dissimilarity metrics"): point-wise MSE and L1
 * (closed-form atlas: mean, voxel-wise median), patch-wise local NCC and
 * SSIM over w^3 windows (atlas by mini-batch Adam). */
typedef enum { DARC_MSE = 0, DARC_LNCC = 1, DARC_L1 = 2, DARC_SSIM = 3 } darc_dissim;

/* Method settings.  Defaults (darc_default_config) follow the paper where it
 * gives a number: T = 7 squarings (Sec. "Diffeomorphisms"); Adam lr 1e-2 for
 * velocities and atlas, K3 = 20 atlas epochs (Sec. "Experiments"). */
typedef struct {
    int dissim;            /* darc_dissim                                         */
    int ncc_window;        /* odd edge w of the NCC / SSIM window, 3..17          */
    int n_squarings;       /* T, 0..20                                            */
    float lambda;          /* weight of the diffusion regulariser (Eq. 2)         */
    float lr, beta1, beta2, adam_eps;   /* Adam                                   */
    float ncc_eps;         /* NCC denominator stabiliser                          */
    int inner_steps;       /* K2: Adam steps per subject per sweep (Algorithm 1)  */
    int atlas_epochs;      /* K3: epochs of atlas SGD (NCC)                        */
    int atlas_batch;       /* atlas SGD mini-batch                                 */
    int center_mode;       /* 0: centre the velocities (the only mode built)       */
    int checkpoint_stride; /* 0: keep u_1..u_T for the adjoint; k > 0: keep every
                              k-th and recompute the rest in the adjoint           */
    int subject_batch;     /* subjects per launch in darc_subject_step (0 = all)  */
    int reset_each_sweep;  /* 1: restart v and Adam each sweep (literal Algorithm 1) */
    unsigned long long seed; /* atlas mini-batch shuffle                           */
    int adjoint;           /* darc_adjoint: how the squarings' adjoint forms the
                              transpose of the interpolation                      */
} darc_config;

/* The transpose of trilinear sampling in the adjoint of each squaring
 * (Sec. "Diffeomorphisms", the backward of Exp).  SCATTER: every source adds
 * its 8 corner weights with float atomics into a buffer its forward squaring
 * cleared.  GATHER: every voxel collects the sources whose displacement is
 * below one voxel on each axis from its 27 neighbours and is written once;
 * the others are scattered afterwards, so the result is bitwise
 * reproducible where all displacements are sub-voxel.  Both give the same
 * gradient up to float rounding order. */
typedef enum { DARC_ADJOINT_SCATTER = 0, DARC_ADJOINT_GATHER = 1 } darc_adjoint;

/* Per-sweep statistics (Sec. "Evaluation metrics"; Table 1's centrality). */
typedef struct {
    double loss_data;           /* mean over subjects of L at their last inner step   */
    double loss_reg;            /* mean over subjects of R at their last inner step   */
    double centrality_before;   /* mean_x |1/n sum_i v_i(x)| before the activation     */
    double centrality_after;    /* the same after it                                  */
    double atlas_loss;          /* NCC atlas SGD: mean loss of its last epoch (else 0) */
    int nonfinite_subjects;     /* subjects whose update was skipped (NaN/Inf loss)    */
} darc_sweep_stats;

typedef struct darc_cohort darc_cohort;

void darc_default_config(darc_config* cfg);
const char* darc_last_error(void);
const char* darc_version(void);

/* ===================================================================== */
/* Cohort API (Eq. 3; Algorithm 1)                                        */
/* ===================================================================== */

/* Creates a cohort of n subjects of D x H x W voxels.  images_dev [n][V]
 * stays owned by the caller and must outlive the cohort.  Allocates v, Adam
 * m/s (zero), the atlas A^0 = 1/n sum_i I_i (Algorithm 1 "initialize()";
 * reading: the MSE closed form at v = 0) and all scratch.  stream: the
 * caller's stream; every later call on the cohort is ordered after the work
 * already on it and before the work enqueued on it afterwards.
 * Errors: ARG, SHAPE, OOM, CUDA. */
int darc_init_cohort(darc_cohort** out, const darc_config* cfg, int n, int D, int H, int W,
                     const float* images_dev, void* stream);

/* `steps` Adam steps of subjects first..first+count-1 against the frozen
 * atlas (Eq. 3, lines 1..n; Algorithm 1 diffeo_pairwise_reg body): per step
 * phi = Exp(v), E = L(I o phi, A) + lambda R(u_T), dE/dv by the hand-written
 * adjoint, Adam.  loss_host (nullable) [count] receives each subject's E at
 * its last step (this waits for the stream).  A subject whose loss is not
 * finite keeps its v; the call then returns DARC_ERR_NONFINITE when
 * loss_host is given (otherwise the next darc_sweep reports it).
 * Errors: ARG, CUDA, NONFINITE. */
int darc_subject_step(darc_cohort* c, int first, int count, int steps, float* loss_host);

/* One outer iteration of Algorithm 1: every subject takes inner_steps steps
 * (darc_subject_step), then darc_update_atlas.  stats (nullable) is filled
 * after waiting for the stream.  Errors: ARG, CUDA, NONFINITE. */
int darc_sweep(darc_cohort* c, darc_sweep_stats* stats);

/* Enqueues, without waiting, a copy of every subject's losses at its last
 * step into out_dev float [n][2] = (L, R) (the values darc_sweep's stats
 * average), ordered on the caller's stream after the work already enqueued
 * on the cohort: a driver can read step k's losses while step k + 1 runs.
 * Non-finite losses are copied as they are (the next darc_sweep with stats
 * reports them).  Errors: ARG, CUDA. */
int darc_sweep_losses(darc_cohort* c, float* out_dev);

/* Centrality activation hat v_i = v_i - 1/n sum_j v_j (Eq. 3 line n+1) on
 * the stored velocities, then the atlas re-estimate (Eq. 3 last line): MSE,
 * A = 1/n sum_i I_i o Exp(hat v_i) (Sec. "Dissimilarity metrics", closed
 * form); local NCC, atlas_epochs epochs of mini-batch Adam on A over the
 * warped cohort (Algorithm 1 SGD_for_atlas).  stats (nullable): the
 * centrality and atlas fields are filled (waits).  Errors: CUDA. */
int darc_update_atlas(darc_cohort* c, darc_sweep_stats* stats);

/* One-shot segmentation (Eq. oneshot): out[i] = labels o Exp(-v_i) for
 * i = first..first+count-1, nearest voxel r(p)_a = clamp(floor(p_a + 1/2),
 * 0, n_a - 1).  atlas_labels_dev uint8 [V]; out_dev uint8 [count][V].
 * Errors: ARG, CUDA. */
int darc_propagate_labels(darc_cohort* c, const uint8_t* atlas_labels_dev, uint8_t* out_dev,
                          int first, int count);

/* Diffeomorphism report (Sec. "Evaluation metrics": the folding rate
 * |J|<0 %; Sec. "Diffeomorphisms": Exp(-v) is the inverse of Exp(v)) for
 * subjects first..first+count-1 from their current velocities:
 * stats_host float [count][4] = {fraction of voxels with
 * det(I + grad u) <= 0 for u = Exp(v); mean and max over voxels of
 * |r(x)|, r the displacement of Exp(-v) o Exp(v) (zero for an exact
 * inverse; trilinear composition); min det}.  Uses the cohort's scratch;
 * the cohort's state is unchanged.  Waits for its work.
 * Errors: ARG, OOM, CUDA. */
int darc_diffeo_report(darc_cohort* c, int first, int count, float* stats_host);

/* PCA shape model (Sec. "Shape synthesis"): the principal components of
 * the cohort's current velocities, from the eigenpairs of the n x n Gram
 * matrix of the centred velocities (Jacobi rotations on the host).
 * eigvals_host double [n]: the eigenvalues lambda_k of the sample
 * covariance (1/(n - 1)), descending (at most n - 1 are nonzero);
 * weights_host (nullable) double [n][n]: row k = the subject weights e_k of
 * mode k, U_k = sum_i e_k[i] (v_i - mean) / sqrt((n - 1) lambda_k), signed so
 * that its largest-magnitude entry is positive.  Kept in the cohort for
 * darc_shape_sample.  Waits for its work.  Errors: ARG, OOM, CUDA. */
int darc_shape_pca(darc_cohort* c, double* eigvals_host, double* weights_host);

/* The host eigensolver behind darc_shape_pca: a_host [n][n] symmetric ->
 * mu_host [n] descending, e_host [n][n] (row k the unit eigenvector of
 * mu_k, largest-magnitude entry positive).  Host memory only; needs no GPU.
 * Errors: ARG. */
int darc_sym_eigen(const double* a_host, int n, double* mu_host, double* e_host);

/* New velocities v_out_dev [m][3][V] = mean + sum_{j<p} sqrt(lambda_j)
 * z_host[k][j] U_j (Sec. "Shape synthesis", alpha_j ~ N(0, lambda_j) drawn
 * by the caller as standard normal z_host [m][p]); phi_new = Exp(v_out).
 * Requires darc_shape_pca; 0 <= p <= n - 1.  Waits for its work.
 * Errors: ARG, CUDA. */
int darc_shape_sample(darc_cohort* c, const double* z_host, int m, int p, float* v_out_dev);

/* Copies of the state.  Velocity and atlas layouts as above.  set_velocity
 * zeroes subject i's Adam moments and step count (a warm start).
 * set_atlas replaces A (and its NCC window statistics).  Errors: ARG, CUDA. */
int darc_get_atlas(darc_cohort* c, float* out_dev);
int darc_set_atlas(darc_cohort* c, const float* atlas_dev);
int darc_get_velocity(darc_cohort* c, int i, float* out_dev);
int darc_set_velocity(darc_cohort* c, int i, const float* v_dev);
/* Adam state of subject i: m, s [3][V] each and the step count. */
int darc_get_adam_state(darc_cohort* c, int i, float* m_dev, float* s_dev, int* step_host);
int darc_cohort_info(darc_cohort* c, int* n, int* D, int* H, int* W, darc_config* cfg);

/* Checkpoint / resume: v, m, s, step counts, A, sweep index and config to a
 * file; darc_load rebuilds a cohort on images_dev.  Errors: IO, ARG, OOM. */
int darc_save(darc_cohort* c, const char* path);
int darc_load(darc_cohort** out, const char* path, const float* images_dev, void* stream);

void darc_destroy(darc_cohort* c);

/* ===================================================================== */
/* Sharded cohorts: hooks around the exchange steps of Eq. 3              */
/* ===================================================================== */
/* When the subjects of one cohort are split over several GPUs (each rank a
 * darc_cohort of its own subjects, same atlas), the subject updates stay
 * local (Eq. 3: uncoupled given A) and only the centrality activation and
 * the atlas re-estimate need the whole cohort.  These calls split them so a
 * caller can put a sum all-reduce (e.g. NCCL) between the halves; on one
 * rank, with an identity in between, they compute what darc_update_atlas
 * computes (up to summation order).  All are stream-ordered like the rest. */

/* sum_dev [3][V] <- sum of this rank's velocities (fixed order). */
int darc_velocity_sum(darc_cohort* c, float* sum_dev);
/* v_i <- v_i - sum_dev / n_total for every subject of this rank (sum_dev
 * [3][V] = the all-reduced darc_velocity_sum, n_total = subjects of all
 * ranks).  Errors: ARG, CUDA. */
int darc_centrality_apply(darc_cohort* c, const float* sum_dev, long long n_total);
/* MSE atlas: acc_dev double [V] <- sum over this rank's subjects of
 * I_i o Exp(v_i) (after the centrality activation). */
int darc_atlas_partial(darc_cohort* c, double* acc_dev);
/* A <- acc_dev / n_total (acc_dev = the all-reduced partial sums). */
int darc_atlas_set_sum(darc_cohort* c, const double* acc_dev, long long n_total);
/* NCC atlas SGD (Algorithm 1 SGD_for_atlas) split per mini-batch: begin
 * warps this rank's subjects and resets the atlas optimiser; grad writes
 * g_dev [V] = sum over this rank's mini-batch `batch` of epoch `epoch` of
 * dL_i/dA and loss_dev float [1] = the sum of their losses (the order of the
 * rank's subjects is its own shuffle, seeded with cfg.seed + rank_seed);
 * apply takes one Adam step with the all-reduced sum divided by the global
 * batch size; end refreshes the atlas window statistics.  A mini-batch of
 * at most 16 subjects takes the single-GPU update's fused box passes (per
 * sub-batch of up to four subjects one forward and one adjoint pass; the
 * last writes g_dev instead of stepping the atlas).  All four calls
 * only enqueue work on the cohort's stream: a driver keeps the losses on the
 * device and synchronises once per atlas update.
 * Returns DARC_ERR_ARG for an epoch/batch outside the schedule. */
int darc_atlas_sgd_begin(darc_cohort* c, int sweep, unsigned long long rank_seed);
int darc_atlas_sgd_grad(darc_cohort* c, int epoch, int batch, float* g_dev, float* loss_dev);
int darc_atlas_sgd_apply(darc_cohort* c, const float* g_dev, int global_batch);
int darc_atlas_sgd_end(darc_cohort* c);
/* number of mini-batches per epoch of this rank: ceil(n / atlas_batch) */
int darc_atlas_batches(darc_cohort* c);

/* ===================================================================== */
/* Measurement                                                             */
/* ===================================================================== */

/* Kernel families timed by the profiling switch. */
typedef enum {
    DARC_K_EXP_SQUARE = 0,      /* one squaring of Exp (24 B/voxel/subject)            */
    DARC_K_EXP_ADJOINT = 1,     /* adjoint of one squaring: the gather (36 B/voxel)    */
    DARC_K_WARP = 2,            /* warp (20 B/voxel/subject)                           */
    DARC_K_LNCC_FWD = 3,        /* local-NCC forward (28 B/voxel/subject)              */
    DARC_K_LNCC_BWD_WARP_REG = 4,/* NCC adjoint + warp adjoint + regulariser (48 B)    */
    DARC_K_MSE_WARP_REG = 5,    /* fused MSE step (32 B/voxel/subject)                 */
    DARC_K_ADAM = 6,            /* Adam on the velocities (84 B/voxel/subject)         */
    DARC_K_ATLAS = 7,           /* everything of the atlas re-estimate                 */
    DARC_K_EXP_FAR = 8,         /* far-source scatter after the gather adjoint (no
                                 * algorithmic bytes of its own: the step's 36 B
                                 * are counted on DARC_K_EXP_ADJOINT)                 */
    DARC_K_COUNT = 9
} darc_kernel_id;

/* on != 0: later calls on the cohort launch every kernel directly (no graph
 * replay) and bracket each launch of the families above with CUDA events on
 * the cohort's stream.  Off by default.  Errors: ARG. */
int darc_set_profiling(darc_cohort* c, int on);

/* Sums over the launches recorded since the last read (then cleared):
 * total_ms = summed event time, launches, bytes = algorithmic bytes (each
 * field read or written once, per the byte counts above).  Waits for the
 * cohort's stream.  Errors: ARG, CUDA. */
int darc_profile_read(darc_cohort* c, int kernel_id, double* total_ms, long long* launches,
                      double* bytes);

/* Kernels launched by the cohort so far (graph replays count each node). */
long long darc_launch_count(darc_cohort* c);

/* ===================================================================== */
/* Operator API: the kernels of one subject step, for B subjects at once. */
/* Used by the autograd wrappers and by parity tests.  `work_dev` is      */
/* caller-owned scratch of at least the size the matching *_workspace     */
/* query returns (bytes, 256-byte aligned).                                */
/* ===================================================================== */

/* Scaling and squaring (Sec. "Diffeomorphisms"): u_0 = sign 2^-T v,
 * u_{t+1}(x) = u_t(x) + S(u_t, x + u_t(x)).  v_dev [B][3][V]; u_dev
 * [T][B][3][V] receives u_1..u_T (u_T last).  sign = +1 for Exp(v), -1 for
 * Exp(-v).  T = 0 is an error (u_0 is v scaled; nothing to store).
 * Errors: ARG, SHAPE, CUDA. */
int darc_exp_forward(const float* v_dev, float* u_dev, int B, int D, int H, int W, int T,
                     float sign, void* stream);

/* Adjoint of darc_exp_forward: gv = dE/dv given gT = dE/du_T.  Each squaring
 * sends its incoming gradient to u_t(x) (identity), through dS/dp (Jacobian
 * term) and to the 8 interpolation corners (transpose of the interpolation,
 * a scatter).  u_dev as written by darc_exp_forward.  gv_dev [B][3][V] may
 * alias gT_dev.  work_dev: darc_exp_backward_workspace(B, D, H, W) bytes.
 * Errors: ARG, SHAPE, CUDA. */
size_t darc_exp_backward_workspace(int B, int D, int H, int W);
int darc_exp_backward(const float* v_dev, const float* u_dev, const float* gT_dev, float* gv_dev,
                      void* work_dev, int B, int D, int H, int W, int T, float sign, void* stream);

/* Warp (Eq. 2, "I o phi"): out[b](x) = S(I[b], x + u[b](x)).  I_dev [B][V]
 * (or [V] when I_batch_stride_zero != 0: one image for every b), u_dev
 * [B][3][V], out_dev [B][V].  Errors: ARG, SHAPE, CUDA. */
int darc_warp(const float* I_dev, int I_batch_stride_zero, const float* u_dev, float* out_dev,
              int B, int D, int H, int W, void* stream);

/* Adjoint of the warp with respect to u: gu[b](x) = gW[b](x) dS(I[b], p)/dp
 * at p = x + u[b](x); the derivative is 0 along a clamped axis.
 * Errors: ARG, SHAPE, CUDA. */
int darc_warp_backward(const float* I_dev, int I_batch_stride_zero, const float* u_dev,
                       const float* gW_dev, float* gu_dev, int B, int D, int H, int W,
                       void* stream);

/* MSE (Sec. "Dissimilarity metrics"; reading: mean over voxels)
 * L_b = 1/V sum_x (J[b](x) - A(x))^2.  J_dev [B][V], A_dev [V], loss_dev
 * float [B], gJ_dev (nullable) [B][V] = dL_b/dJ[b].  work_dev:
 * darc_loss_workspace(B, D, H, W).  Errors: ARG, SHAPE, CUDA. */
size_t darc_loss_workspace(int B, int D, int H, int W);
int darc_mse(const float* J_dev, const float* A_dev, float* loss_dev, float* gJ_dev,
             void* work_dev, int B, int D, int H, int W, void* stream);

/* L1 (Sec. "Dissimilarity metrics", point-wise): L_b = 1/V sum_x
 * |J[b](x) - A(x)|; gJ_dev (nullable) [B][V] = sign(J - A) / V (0 where
 * equal).  Layout and workspace as darc_mse.  Errors: ARG, SHAPE, CUDA. */
int darc_l1(const float* J_dev, const float* A_dev, float* loss_dev, float* gJ_dev,
            void* work_dev, int B, int D, int H, int W, void* stream);

/* The L1 atlas closed form (Sec. "Dissimilarity metrics"): out_dev[x] =
 * median over i of X_dev[i][x], X_dev [n][D*H*W].  Reading for even n: the
 * lower middle value (sorted s_0 <= ... <= s_{n-1}, s_{(n-1)/2}); the result
 * is always one of the inputs.  1 <= n <= 1600.  Errors: ARG, SHAPE, CUDA. */
int darc_median(const float* X_dev, int n, int D, int H, int W, float* out_dev, void* stream);

/* Local NCC (Sec. "Dissimilarity metrics", patch-wise NCC; reading: squared
 * correlation over the w^3 window with zero padding, normalised by w^3,
 * denominator + eps): L_b = -1/V sum_x cc_b(x).  gJ_dev (nullable) [B][V] =
 * dL_b/dJ[b]; gA_dev (nullable) [V] = sum_b dL_b/dA.  work_dev:
 * darc_lncc_workspace(B, D, H, W).  Errors: ARG, SHAPE, CUDA. */
size_t darc_lncc_workspace(int B, int D, int H, int W);
int darc_lncc(const float* J_dev, const float* A_dev, int window, float eps, float* loss_dev,
              float* gJ_dev, float* gA_dev, void* work_dev, int B, int D, int H, int W,
              void* stream);

/* SSIM (Sec. "Dissimilarity metrics", patch-wise; reading: Wang et al.'s
 * structural similarity over the same w^3 windows as darc_lncc, zero
 * padding, normalised by w^3, C1 = 1e-4, C2 = 9e-4 for intensities on
 * [0, 1]): L_b = -1/V sum_x ssim_b(x).  Gradients, layouts and workspace
 * (darc_lncc_workspace) as darc_lncc.  Errors: ARG, SHAPE, CUDA. */
int darc_ssim(const float* J_dev, const float* A_dev, int window, float* loss_dev, float* gJ_dev,
              float* gA_dev, void* work_dev, int B, int D, int H, int W, void* stream);

/* Diffusion regulariser (Eq. 2 second term; reading: forward differences of
 * the displacement, mean over the voxel pairs of each axis, mean over the
 * three axes).  u_dev [B][3][V], loss_dev float [B], gu_dev (nullable)
 * [B][3][V] = dR_b/du[b].  work_dev: darc_loss_workspace.
 * Errors: ARG, SHAPE, CUDA. */
int darc_diffusion_reg(const float* u_dev, float* loss_dev, float* gu_dev, void* work_dev, int B,
                       int D, int H, int W, void* stream);

/* One subject energy and gradient without the optimiser step (Eq. 2 for
 * each of B subjects, as in darc_subject_step): energy_dev float [B][2]
 * receives {L, R}; gv_dev [B][3][V] = dE/dv.  A_dev [V].  cfg supplies
 * dissim, window, T, lambda, ncc_eps, checkpoint_stride.  work_dev:
 * darc_subject_grad_workspace(cfg, B, D, H, W).  Errors: ARG, SHAPE, CUDA. */
size_t darc_subject_grad_workspace(const darc_config* cfg, int B, int D, int H, int W);
int darc_subject_grad(const darc_config* cfg, const float* I_dev, const float* A_dev,
                      const float* v_dev, float* energy_dev, float* gv_dev, void* work_dev, int B,
                      int D, int H, int W, void* stream);

/* Adam (Sec. "Experiments"; reading: PyTorch defaults, bias corrected):
 * m = b1 m + (1-b1) g, s = b2 s + (1-b2) g^2,
 * theta -= lr (m / (1 - b1^k)) / (sqrt(s / (1 - b2^k)) + eps).
 * theta, m, s, g: float [N]; k >= 1 is the 1-based step.  Errors: ARG, CUDA. */
int darc_adam(float* theta_dev, float* m_dev, float* s_dev, const float* g_dev, size_t N, int k,
              float lr, float beta1, float beta2, float eps, void* stream);

/* Centrality activation (Eq. 3): v[i] -= 1/n sum_j v[j] for v_dev [n][3][V];
 * metrics_dev (nullable) double [2] = mean_x |1/n sum_i v_i(x)| before and
 * after.  work_dev: darc_centrality_workspace(n, D, H, W).
 * Errors: ARG, CUDA. */
size_t darc_centrality_workspace(int n, int D, int H, int W);
int darc_centrality(float* v_dev, double* metrics_dev, void* work_dev, int n, int D, int H, int W,
                    void* stream);

/* MSE atlas closed form (Sec. "Dissimilarity metrics"):
 * A = 1/n sum_i I_i o Exp(v_i).  I_dev [n][V], v_dev [n][3][V], A_dev [V].
 * work_dev: darc_atlas_mean_workspace(n, D, H, W).  Errors: ARG, CUDA. */
size_t darc_atlas_mean_workspace(int n, int D, int H, int W);
int darc_atlas_mean(const float* I_dev, const float* v_dev, float* A_dev, void* work_dev, int n,
                    int D, int H, int W, int T, void* stream);

/* Label gather of Eq. oneshot given u = the displacement of Exp(-v):
 * out[b](x) = labels[r(x + u[b](x))].  Errors: ARG, CUDA. */
int darc_label_gather(const uint8_t* labels_dev, const float* u_dev, uint8_t* out_dev, int B,
                      int D, int H, int W, void* stream);

/* Dice score of one-shot segmentation (Sec. "Evaluation metrics"; Table 3):
 * for each of B label maps a_dev, b_dev [B][V] (uint8) and each label
 * l = 1..n_labels-1 (0 is the background), dice_host[b][l - 1] =
 * 2 |a = l and b = l| / (|a = l| + |b = l|), or -1 where the label occurs in
 * neither map.  n_labels 2..256.  work_dev: darc_dice_workspace(B,
 * n_labels) bytes (counters).  Waits for the stream (host output).
 * Errors: ARG, CUDA. */
size_t darc_dice_workspace(int B, int n_labels);
int darc_dice(const uint8_t* a_dev, const uint8_t* b_dev, int B, long long V, int n_labels, void* work_dev,
              double* dice_host, void* stream);

/* Mesh vertices moved by a forward map (Sec. "Shape synthesis"): out_dev
 * [P][3] = pts_dev[p] + S(u_dev, pts_dev[p]) for points in (z, y, x) voxel
 * coordinates and a displacement u_dev [3][D][H][W] (trilinear, border
 * padded).  Errors: ARG, CUDA. */
int darc_warp_points(const float* u_dev, int D, int H, int W, const float* pts_dev, long long P, float* out_dev,
                     void* stream);

/* Composition of two maps given as displacements (Sec. "Diffeomorphisms"):
 * out[b](x) = a[b](x) + S(b_dev[b], x + a[b](x)), the displacement of
 * phi_b o phi_a; trilinear, border padded.  All [B][3][V]; out must not
 * alias a or b.  Errors: ARG, CUDA. */
int darc_compose(const float* a_dev, const float* b_dev, float* out_dev, int B, int D, int H, int W, void* stream);

/* Folding report (Sec. "Evaluation metrics", |J|<0 %): det(I + grad u) by
 * central differences (one-sided on faces) into det_dev (nullable) [B][V];
 * count_dev (nullable) unsigned long long [B] = voxels with det <= 0.
 * Errors: ARG, CUDA. */
int darc_jacobian_det(const float* u_dev, float* det_dev, unsigned long long* count_dev, int B,
                      int D, int H, int W, void* stream);

/* ===================================================================== */
/* Learned warm start: BF16 tensor-core kernels (an addition to the       */
/* method; the paper has no counterpart)                                  */
/* ===================================================================== */

/* C = A B^T on the 5th-generation tensor cores: A_dev bf16 [M][K], B_dev
 * bf16 [N][K] (K contiguous in both), C_dev fp32 [M][N]; fp32 accumulation
 * in tensor memory.  M % 128 == 0, N % 16 == 0 with 16 <= N <= 256,
 * K % 16 == 0.  Errors: ARG, CUDA. */
int darc_gemm_bf16(const void* A_dev, const void* B_dev, float* C_dev, int M, int N, int K, void* stream);

/* 3x3x3 'same' convolution (zero padding) on the tensor cores, BF16
 * operands, FP32 accumulation:
 *   z[v][co] = bias[co] + sum_{tap, ci} in[v + off(tap)][ci] * W[co][tap][ci]
 *   off(tap) = (tap/9 - 1, (tap/3)%3 - 1, tap%3 - 1) in (z, y, x).
 * Volumes are bf16 channels-last with a one-voxel zero border:
 * [batch][D+2][H+2][W+2][stride]; the border of the input must be zero and
 * the border of the output is not written.  in_dev: channels [0, cin)
 * read; wt_dev: weights packed by darc_conv3d_pack_weights (flip 0);
 * bias_dev: fp32 [cout] or null.  Epilogue: act = 1 applies a leaky ReLU of
 * slope `slope`; gate_dev (same geometry, stride gate_stride, or null)
 * multiplies each result by 1 where gate > 0 and by `slope` elsewhere (the
 * data gradient through a leaky ReLU whose output is the gate).  Output:
 * out_dev, channels [0, cout) -- or, when out_f32_dev is non-null, fp32
 * planar without border [batch][cout][D*H*W].  np: cout rounded up to 16.
 * The data gradient of a layer is this call on dL/dz (cin = its cout
 * rounded up to 16) with weights packed with flip 1 and np = its cin.
 * Requirements: cin % 16 == 0, in_stride % 8 == 0, np % 16 == 0 with
 * 16 <= np <= 256, cout <= np, W small enough for two shared-memory stages
 * (W <= 581 at np = 256), 16-byte aligned in_dev and wt_dev.
 * Errors: ARG, SHAPE, CUDA. */
int darc_conv3d(const void* in_dev, int in_stride, int cin, const void* wt_dev, const float* bias_dev, void* out_dev,
                int out_stride, int cout, float* out_f32_dev, const void* gate_dev, int gate_stride, int act,
                float slope, int batch, int D, int H, int W, int np, void* stream);

/* Bytes of packed bf16 weights for a convolution with conv_cin input
 * channels and nrows output rows (both multiples of 16; 0 otherwise). */
size_t darc_conv3d_packed_bytes(int conv_cin, int nrows);

/* Packs fp32 weights w_dev [>= cout][kp] (k = tap * cin + ci, zero past
 * 27 cin) for darc_conv3d: flip = 0 the layer itself (conv_cin = cin,
 * nrows = cout rounded up to 16); flip = 1 its data gradient, the
 * transposed, mirrored kernel W'[ci][tap][co] = W[co][26 - tap][ci]
 * (conv_cin = cout rounded up to 16, nrows = cin).  packed_dev: 16-byte
 * aligned, darc_conv3d_packed_bytes(conv_cin, nrows) bytes.
 * Errors: ARG, SHAPE, CUDA. */
int darc_conv3d_pack_weights(const float* w_dev, int kp, int cin, int cout, int flip, void* packed_dev, void* stream);

/* Weight and bias gradients of darc_conv3d (same padded geometry):
 *   dw[co][k] = sum_v gz[v][co] * in[v + off(tap)][ci], k = tap*cin + ci  (fp32 [np][27 cin])
 *   db[co]    = sum_v gz[v][co]                                         (fp32 [cout], db_dev may be null)
 * gz_dev: gradient wrt the pre-activation (zero border), stride gz_stride,
 * cout % 8 == 0 channels read, cout / 8 dividing 256 when db_dev is given;
 * cin % 16 == 0; np % 16 == 0 with cout <= np <= 128.  Split-K partial sums
 * go to work_dev (fp32, work_bytes) and are added in a fixed order, so the
 * result is deterministic.  Errors: ARG (also: workspace smaller than one
 * split), SHAPE, CUDA. */
int darc_conv3d_wgrad(const void* in_dev, int in_stride, int cin, const void* gz_dev, int gz_stride, int cout,
                      float* dw_dev, float* db_dev, int batch, int D, int H, int W, int np, void* work_dev,
                      size_t work_bytes, void* stream);

/* Half-resolution image (mean of each 2x2x2 block): I_dev fp32 [B][D][H][W]
 * with even D, H, W -> out_dev [B][D/2][H/2][W/2].  Errors: ARG, CUDA. */
int darc_resample_half(const float* I_dev, int B, int D, int H, int W, float* out_dev, void* stream);

/* Full-resolution velocity from a half-resolution one: trilinear
 * interpolation at ((x + 1/2)/2 - 1/2) of the half grid (clamped), values
 * doubled because the voxel unit halves.  vh_dev fp32 [B][3][Dh][Hh][Wh] ->
 * v_dev [B][3][2Dh][2Hh][2Wh].  Errors: ARG, CUDA. */
int darc_upsample_velocity(const float* vh_dev, int B, int Dh, int Hh, int Wh, float* v_dev, void* stream);

/* The warm-start network: a 3-D U-Net with 4 levels of 16, 32, 64, 128
 * channels (two 3x3x3 conv + leaky ReLU 0.2 per level, 2x average pooling
 * down, nearest 2x up, skip connections by channel concatenation, a 3x3x3
 * head to 3 channels).  Input: (subject, atlas) at the network's
 * resolution D x H x W (each a multiple of 8, >= 16); output: a velocity
 * field fp32 [B][3][D][H][W] in voxel units of that grid.  BF16 weights
 * and activations, FP32 accumulation and FP32 master weights (Adam with
 * PyTorch's defaults beta = (0.9, 0.999), eps = 1e-8).  Weights are
 * He-normal from `seed` (SplitMix64 + Box-Muller).  The handle owns every
 * buffer for batches up to max_batch; calls on one handle must be ordered.
 * Errors: ARG, SHAPE, OOM, CUDA. */
typedef struct darc_unet darc_unet;
int darc_unet_create(darc_unet** out, int D, int H, int W, int max_batch, unsigned long long seed);
void darc_unet_destroy(darc_unet* u);
/* subj_dev fp32 [B][D][H][W], atlas_dev fp32 [D][H][W] (shared by the
 * batch) -> v_dev fp32 [B][3][D][H][W]. */
int darc_unet_forward(darc_unet* u, const float* subj_dev, const float* atlas_dev, int B, float* v_dev, void* stream);
/* One Adam step on loss = mean over B*3*D*H*W of (net(subj, atlas) -
 * target)^2, target_dev fp32 [B][3][D][H][W].  loss_host (may be null)
 * receives the loss of the forward pass before the update (the call then
 * synchronises the stream). */
int darc_unet_train_step(darc_unet* u, const float* subj_dev, const float* atlas_dev, const float* target_dev, int B,
                         float lr, float* loss_host, void* stream);
/* The same loss and its gradients without an update (read them with
 * darc_unet_layer_params). */
int darc_unet_gradients(darc_unet* u, const float* subj_dev, const float* atlas_dev, const float* target_dev, int B,
                        float* loss_host, void* stream);
/* Layer l in 0..14 (encoder 0-7, decoder 8-13, head 14): padded input
 * channels cin (multiple of 8), cout, and the weight matrix shape [np][kp]
 * with k = tap*cin + ci (cin rounded up to 16). */
int darc_unet_layer_info(darc_unet* u, int layer, int* cin, int* cout, int* kp, int* np);
/* set = 0: copy the fp32 master weights [np][kp], bias [cout] and the last
 * gradients out (null pointers skip); set = 1: load w and b (refreshing the
 * bf16 copies).  Synchronises the device. */
int darc_unet_layer_params(darc_unet* u, int layer, float* w_dev, float* b_dev, float* dw_dev, float* db_dev, int set);
/* Weights and Adam state to / from a file (little-endian, magic
 * "DARCUNT1").  Errors: ARG, IO, CUDA. */
int darc_unet_save(darc_unet* u, const char* path);
int darc_unet_load(darc_unet* u, const char* path);

/* ===================================================================== */
/* Allocation-free adjoint (the paper has no counterpart)                 */
/* ===================================================================== */

/* For callers that cannot allocate device memory -- a plug-in handed its
 * device buffers by a host application that owns the allocator, or a
 * process whose device memory is committed to a fixed budget -- and so
 * cannot supply the workspace darc_exp_backward needs.  Same arguments and
 * result as darc_exp_backward without the workspace: the scratch lives in a
 * file-scope device array of DARC_NOALLOC_SCRATCH_BYTES (64 MiB) that every
 * GPU which loads the library holds until the process exits.
 *  - Limit: B*D*H*W <= DARC_NOALLOC_MAX_VOXELS (the adjoint alternates
 *    between two gradient buffers of B*3*D*H*W floats); a larger call
 *    returns DARC_ERR_ARG and a message naming the limit.
 *  - The first call on a device looks up the array's device address (one
 *    cudaGetSymbolAddress with that device current); make that first call
 *    before any stream capture on the device.  Under CUDA's default lazy
 *    module loading the driver also commits the 64 MiB only then (at load
 *    time with CUDA_MODULE_LOADING=EAGER), so that first call can fail
 *    with DARC_ERR_CUDA when the device is full: a caller on a fixed budget
 *    should make one call at start-up.
 *  - gv_dev may equal gT_dev (the result replaces the incoming gradient);
 *    any other overlap of gv_dev with v_dev, u_dev or gT_dev returns
 *    DARC_ERR_ARG.
 *  - All calls share the one array, which keeps the last call's contents;
 *    each call clears what it accumulates into before using it.  Calls
 *    whose work overlaps on the GPU (other streams, unordered threads) race
 *    on the array: order them on one stream.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * Errors: ARG, SHAPE, CUDA. */
#define DARC_NOALLOC_SCRATCH_BYTES (64u << 20)
#define DARC_NOALLOC_MAX_VOXELS 2796202
int darc_exp_backward_noalloc(const float* v_dev, const float* u_dev, const float* gT_dev,
                              float* gv_dev, int B, int D, int H, int W, int T, float sign,
                              void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DARC_H_ */
