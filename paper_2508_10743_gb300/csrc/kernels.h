// kernels.h -- host launchers of the libdarc kernels (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "common.cuh"

namespace darc_impl {

// records `msg` as the thread's darc_last_error() and returns `code`
int report_error(int code, const std::string& msg);

// ---- scaling and squaring (k_exp.cu) ----
// dst[b] = u + S(u, x + u(x)) with u = scale * src[b]; B fields of [3][V].
cudaError_t exp_square(const float* src, float scale, float* dst, int B, const Vol& v,
                       cudaStream_t s);
// Adjoint of one squaring: gout[b] += out_scale * (identity + Jacobian +
// transpose-interpolation terms of gin[b]); u = scale * src[b].
// gout must hold zeros (or a sum to add to) before the call.
cudaError_t exp_square_adjoint(const float* src, float scale, const float* gin, float* gout,
                               float out_scale, int B, const Vol& v, cudaStream_t s);
// The same adjoint onto interleaved gradients: gout [B][V] float4 (z, y, x,
// 0), 16-byte aligned and cleared (or holding a sum to add to); gin is
// interleaved the same way (gin_interleaved != 0) or planar [B][3][V]; the
// field src likewise packed (src_packed != 0) or planar.
cudaError_t exp_square_adjoint4(const float* src, int src_packed, float scale, const float* gin, int gin_interleaved,
                                float4* gout, float out_scale, int B, const Vol& v, cudaStream_t s);
// Scatter-free adjoint of one squaring (k_exp_gather.cu): gout = out_scale *
// (identity + Jacobian terms + transpose terms of the near sources, |u_a| < 1
// on every axis), written once with plain stores (no clearing needed); the
// 32 x 8 x 8 tiles holding far sources are marked in flags
// (exp_far_flags(B, v) ints).  exp_adjoint_far then adds the far sources'
// transpose terms onto gout with atomics, visiting marked tiles only and
// clearing their marks.  gin / gout: interleaved [B][V] float4 (z, y, x, 0)
// (16-byte aligned) when *_interleaved, else planar [B][3][V]; src packed
// likewise when src_packed; u = scale * src.
size_t exp_far_flags(int B, const Vol& v);
cudaError_t exp_adjoint_gather(const float* src, int src_packed, float scale, const float* gin, int gin_interleaved,
                               float* gout, int gout_interleaved, float out_scale, int* flags, int B, const Vol& v,
                               cudaStream_t s);
cudaError_t exp_adjoint_far(const float* src, int src_packed, float scale, const float* gin, int gin_interleaved,
                            float* gout, int gout_interleaved, float out_scale, int* flags, int B, const Vol& v,
                            cudaStream_t s);
// g [B][3][V] from an interleaved gradient g4 [B][V] float4 (z, y, x, 0)
cudaError_t unpack_field(const float4* g4, float* g, int B, const Vol& v, cudaStream_t s);
// One squaring written packed: dst [B][V] float4 (z, y, x, 0), 16-byte
// aligned; src planar [B][3][V] or packed the same way (src_packed != 0).
// zero (may be null): another [B][V] float4 buffer set to zero on the way.
cudaError_t exp_square_packed(const float* src, int src_packed, float scale, float4* dst, int B, const Vol& v,
                              cudaStream_t s, float4* zero = nullptr);

// ---- images (k_image.cu) ----
cudaError_t warp(const float* I, size_t I_bstride, const float* u, float* out, int B, const Vol& v,
                 cudaStream_t s);
// the same with u packed, [B][V] float4 (z, y, x, 0), 16-byte aligned
cudaError_t warp_packed(const float* I, size_t I_bstride, const float4* u, float* out, int B, const Vol& v,
                        cudaStream_t s);
cudaError_t warp_backward(const float* I, size_t I_bstride, const float* u, const float* gW,
                          float* gu, int B, const Vol& v, cudaStream_t s);
// partials: double [B][nblk] laid out per subject, nblk = voxel_blocks(v)
int voxel_blocks(const Vol& v);
// l1 = 0: MSE (d^2, 2d); l1 = 1: L1 (|d|, sign d)
cudaError_t mse_partials(const float* J, const float* A, float* gJ, double* partials, int B,
                         const Vol& v, int l1, cudaStream_t s);
cudaError_t reg_partials(const float* u, float* gu, double* partials, int B, const Vol& v,
                         cudaStream_t s);
// fused point-wise subject step (l1 = 0: MSE, 1: L1): from u_T and I: W,
// the loss, its gradient through the warp, plus lambda * the regulariser
// gradient -> gT; partials [B][nblk][2]
cudaError_t mse_warp_reg(const float* I, size_t I_bstride, const float* A, const float* uT,
                         float lambda, float* gT, double* partials, int B, const Vol& v,
                         int l1, cudaStream_t s, int uT_packed = 0);
// out[l] = lower median over the n rows of X [n][V]; median_threads(n) == 0:
// n too large for the shared-memory columns (cudaErrorInvalidValue)
int median_threads(int n);
cudaError_t median(const float* X, int n, long long V, float* out, cudaStream_t s);
cudaError_t label_gather(const uint8_t* labels, const float* u, uint8_t* out, int B, const Vol& v,
                         cudaStream_t s);
// counts [B][nl][3] (cleared by the caller) += {|a = l|, |b = l|, |a = l and
// b = l|} over the V voxels of each of the B label maps; nl <= 256
cudaError_t label_overlap(const uint8_t* a, const uint8_t* b, int B, long long V, int nl,
                          unsigned long long* counts, cudaStream_t s);
// ---- PCA shape synthesis (k_shape.cu) ----
// mean[l] = 1/n sum_i v[i][l], v [n][M]
cudaError_t field_mean(const float* v, int n, long long M, float* mean, cudaStream_t s);
// G [n][n] = centred Gram matrix of the rows of v; partial: gram_splits(n) * n * n doubles
int gram_splits(int n);
cudaError_t gram(const float* v, const float* mean, int n, long long M, double* partial, double* G, cudaStream_t s);
// out[k] = mean + sum_i coef[k][i] (v_i - mean), k < m <= 8, coef float [m][n]
cudaError_t combine_fields(const float* v, const float* mean, int n, long long M, const float* coef, int m,
                           float* out, cudaStream_t s);
// out[p] = pts[p] + S(u, pts[p]), u [3][V], points [P][3] (z, y, x)
cudaError_t warp_points(const float* u, const Vol& v, const float* pts, long long P, float* out, cudaStream_t s);
// displacement of phi_b o phi_a: out = a + S(b, x + a)  ([B][3][V])
cudaError_t compose(const float* a, const float* b, float* out, int B, const Vol& v, cudaStream_t s);
// stats[b][4] = {fraction det(I + grad u) <= 0, mean |r|, max |r|, min det};
// partials: B * voxel_blocks(v) * 4 doubles
cudaError_t diffeo_stats(const float* u, const float* r, double* partials, float* stats, int B, const Vol& v,
                         cudaStream_t s);
cudaError_t jacobian_det(const float* u, float* det, unsigned long long* count, int B,
                         const Vol& v, cudaStream_t s);

// ---- reductions and optimiser (k_optim.cu) ----
// out[b * out_stride + k] = scale * sum_j partials[(b * nblk + j) * nval + k], k < nval
cudaError_t reduce_partials(const double* partials, int nblk, int nval, double scale, float* out,
                            int out_stride, int B, cudaStream_t s);
// cohort bookkeeping after a subject step: loss[b] = {L, R}; finite check;
// step counts and Adam bias factors for subjects first..first+B-1
// pL / pR: per-subject partial sums of L and R, element (b, j) at
// p[(b * nblk + j) * stride]
cudaError_t finish_step(const double* pL, int nblkL, int strideL, const double* pR, int nblkR,
                        int strideR, float* loss, int* flags, int* k, float2* bias,
                        int* nonfinite_total, float lr, float beta1, float beta2, int B,
                        cudaStream_t s);
// Adam on B fields [3][V] with per-subject factors bias[b] = {lr/c1, 1/sqrt(c2)};
// skipped where flags[b] != 0 (flags may be null)
cudaError_t adam_fields(float* theta, float* m, float* s_, const float* g, float g_scale,
                        const float2* bias, const int* flags, float beta1, float beta2, float eps,
                        int B, long long N, cudaStream_t st);
// The same for B fields [3][V] (B x V voxels) with interleaved gradients g
// [B][V] float4 (z, y, x, 0), scale 1
cudaError_t adam_fields_g4(float* theta, float* m, float* s_, const float4* g, const float2* bias, const int* flags,
                           float beta1, float beta2, float eps, int B, long long V, cudaStream_t st);
cudaError_t adam_flat(float* theta, float* m, float* s_, const float* g, size_t N, float lr_c1,
                      float inv_sqrt_c2, float beta1, float beta2, float eps, cudaStream_t st);
int centrality_blocks(const Vol& v);
cudaError_t centrality(float* v_all, int n, const Vol& v, double* partials, double* metrics,
                       cudaStream_t s);
// acc[l] (double) += sum over b of S(I[idx_b], x + u[b](x)) in fixed b order
cudaError_t warp_accumulate(const float* I, const int* subj, const float* u, double* acc, int B,
                            const Vol& v, cudaStream_t s);
cudaError_t image_mean_accumulate(const float* I, int n, double* acc, const Vol& v,
                                  cudaStream_t s);
cudaError_t finalize_mean(const double* acc, double inv_n, float* A, const Vol& v, cudaStream_t s);
// Adam step of the atlas SGD with the mini-batch mean gradient
// g = scale * (gshared + sum_b gsubj[b]) (gshared may be null)
cudaError_t atlas_adam(float* A, float* m, float* s_, const float* gshared, const float* gsubj,
                       int B, float scale, float lr_c1, float inv_sqrt_c2, float beta1, float beta2,
                       float eps, const Vol& v, cudaStream_t st);

// out[l] = scale * sum over B fields of v[b] [3][V] (fixed order, double sums)
cudaError_t field_sum(const float* v, int B, float* out, const Vol& vol, cudaStream_t s);
// v[b] -= scale * sum for B fields
cudaError_t field_subtract(float* v, int B, const float* sum, float scale, const Vol& vol, cudaStream_t s);
// out[l] = scale * (gshared[l] + sum_b gsubj[b][l])
cudaError_t combine_grad(const float* gshared, const float* gsubj, int B, float scale, float* out,
                         const Vol& v, cudaStream_t s);

// ---- tensor-core kernels (k_unet.cu) ----
cudaError_t gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, cudaStream_t s);
// a D x H x W volume stored with a one-voxel zero border: padded row of
// (z, y, x) = ((z + 1) Hp + y + 1) Wp + x + 1, Vp rows per volume
struct PadVol {
    int D, H, W, Wp, Hp;
    long long P, Vp;            // rows per padded plane, per padded volume
};
PadVol make_pad(int D, int H, int W);
// one 3x3x3 'same' convolution over padded channels-last bf16 volumes (see
// darc_conv3d in darc.h for the fields)
struct ConvDesc {
    const void* in;               // [batch][D+2][H+2][W+2][in_stride], channels [0, cin), cin % 16 == 0
    int in_stride, cin;
    const void* wt;               // packed by pack_weights (cin / 16 chunks, np rows)
    const float* bias;
    void* out;                    // same geometry, channels [0, cout) at out
    int out_stride, cout;
    float* out_f32;               // planar fp32 [batch][cout][D * H * W] (replaces out)
    const void* gate;             // same geometry: multiply by the leaky-ReLU slope where gate <= 0
    int gate_stride;
    int act;
    float slope;
    int batch, D, H, W, np;
};
cudaError_t conv3_forward(const ConvDesc& d, cudaStream_t s);
// whether two pipeline stages of a conv of this width and np fit in shared memory
bool conv_fits(int W, int np);
// bf16 elements of packed weights for a convolution with conv_cin input
// channels (multiple of 16) and nrows output rows (np)
size_t packed_weight_elems(int conv_cin, int nrows);
// pack fp32 masters w[co][k] (k = tap cin + ci, kp per row) for the forward
// (flip 0: conv_cin = cin, nrows = np) or the data gradient (flip 1:
// conv_cin = cout rounded up to 16, nrows = cin)
cudaError_t pack_weights(const float* w, int kp, int cin, int cout, int conv_cin, int nrows, int flip, void* out,
                         cudaStream_t s);
// dw [np][kp] fp32 = sum_q gz[q][co] in[q + off(tap)][ci] over the padded
// rows of the interior planes; partial: splits x kp x np floats
cudaError_t conv3_wgrad(const void* in, int in_stride, int cin, const void* gz, int gz_stride, int cout, float* partial,
                        int splits, float* dw, int batch, int D, int H, int W, int kp, int np, cudaStream_t s);
// CTAs of one split of the weight gradient's window kernel (callers size
// their splits so a launch has about four CTAs per SM)
int wgrad_ctas_per_split(int cin);
int wgrad_resident_ctas(int np);
// db[c] = sum over rows of gz[v][c]; (cout + 7) / 8 must divide 256; work:
// bias_grad_work_floats(cout) floats
int bias_grad_work_floats(int cout);
cudaError_t bias_grad(const void* gz, int stride, long long nvox, int cout, float* db, float* work, cudaStream_t s);
// 2x pooling / nearest upsampling between padded volumes; D, H, W: the fine grid
cudaError_t pool2(const void* x, int xs, void* y, int ys, int C, int B, int D, int H, int W, cudaStream_t s);
cudaError_t pool2_adjoint(const void* gy, int gys, const void* x, int xs, void* gx, int gxs, int C, float slope, int B,
                          int D, int H, int W, cudaStream_t s);
cudaError_t up2(const void* x, int xs, void* y, int ys, int C, int B, int D, int H, int W, cudaStream_t s);
cudaError_t up2_adjoint(const void* gy, int gys, void* gx, int gxs, int C, int B, int D, int H, int W, cudaStream_t s);
// 16-channel padded network input from planar fp32 subjects [B][V] and atlas [V]
cudaError_t pack_input(const float* subj, const float* atlas, void* x, int B, int D, int H, int W, cudaStream_t s);
int velocity_loss_blocks(long long n);
// pred, target planar [batch][3][V]; g padded channels-last, stride gs
cudaError_t velocity_loss(const float* pred, const float* target, int B, int D, int H, int W, void* g, int gs,
                          double* partials, cudaStream_t s);
cudaError_t upsample_velocity(const float* vh, int Dh, int Hh, int Wh, float* v, int D, int H, int W, int B,
                              cudaStream_t s);
cudaError_t downsample_image(const float* I, int D, int H, int W, float* Ih, int B, cudaStream_t s);

// ---- local NCC (k_lncc.cu) ----
// Box sums need scratch P of B x (channels <= 3) x V floats for the 2-D sums.
// Z-pass blocks per image of a box-sum launch of B images (its loss
// partials are laid out [B][box_blocks(v, B)]); at most box_blocks_max(v)
int box_blocks(const Vol& v, int B);
int box_blocks_max(const Vol& v);
// XY strip height and Z chunk of a launch of B images
int box_yc(const Vol& v, int B);
int box_zc(const Vol& v, int B);
// window statistics of the atlas: stats[0] = Box(A), stats[1] = Box(A^2)
cudaError_t atlas_stats(const float* A, float* stats, int r, const Vol& v, float* P, cudaStream_t s);
// forward: box sums of J, J^2, J*A; the patch metric m (metric 0: local
// NCC cc, 1: SSIM); loss partials [B][nblk] of -m/V; per-voxel coefficients
// coef [B][3][V]: wrt_atlas = 0 -> dm/d(S_J, S_JJ, S_JA), 1 -> dm/d(S_A,
// S_AA, S_JA).  J rows are J + subj[b]*V when subj != null.
cudaError_t lncc_forward(const float* J, const int* subj, const float* A, const float* stats,
                         int r, float eps, int wrt_atlas, int metric, float* coef, double* partials, int B,
                         const Vol& v, float* P, cudaStream_t s);
// backward: g = -1/V [Box(c0) + 2 X Box(c1) + Y Box(c2)], X = J (Y = A) or,
// for wrt_atlas, X = A (Y = J); writes g [B][V]
cudaError_t lncc_backward(const float* J, const int* subj, const float* A, const float* coef,
                          int r, int wrt_atlas, float* g, int B, const Vol& v, float* P, cudaStream_t s);
// backward fused with the warp adjoint and the regulariser:
// gT = gJ * dS(I, x + uT)/dp + lambda dR/du_T; reg partials [B][nblk]
// (uT_packed != 0: uT is packed, [B][V] float4 (z, y, x, 0), 16-byte aligned)
cudaError_t lncc_backward_warp_reg(const float* J, const float* A, const float* coef, int r,
                                   const float* I, size_t I_bstride, const float* uT,
                                   float lambda, float* gT, double* partials, int B, const Vol& v,
                                   float* P, cudaStream_t s, int uT_packed = 0);
cudaError_t sum_images(const float* g, int B, float* out, const Vol& v, cudaStream_t s);
// Box(J_b), Box(J_b^2) of B images: stats [B][2][V]
cudaError_t image_stats(const float* J, float* stats, int B, int r, const Vol& v, float* P, cudaStream_t s);
// atlas SGD for a mini-batch (rows subj[0..nb)): coefficients wrt the atlas,
// loss partials [nb][nblk]
cudaError_t atlas_sgd_forward(const float* J, const float* jstats, const int* subj, const float* A,
                              const float* astats, int r, float eps, int metric, float* coef, double* partials,
                              int nb, const Vol& v, float* P, cudaStream_t s);
// gshared [V] = Box(sum a) + 2 A Box(sum b); gsubj [nb][V] = J_b Box(g_b)
cudaError_t atlas_sgd_backward(const float* J, const int* subj, const float* A, const float* coef,
                               int r, float* gshared, float* gsubj, int nb, const Vol& v, float* P,
                               cudaStream_t s);

// The same mini-batch step in box passes when the subjects' rows are known
// on the host (nb <= ATLAS_FUSED_MAX): sub-batches of at most ATLAS_SUB_MAX
// subjects (atlas_sub_batches(nb) of them, sizes differing by one at most),
// each one forward pass and one adjoint pass.  Forward: coef [2 + nb][V]
// (sum_b dm/dS_A, sum_b dm/dS_AA, dm_b/dS_JA), loss partials [nb][nblk],
// P >= (2 + ATLAS_SUB_MAX) V floats.  Adjoint: the sub-batches' gradients
// add up in gacc [V] (unused for one sub-batch), the last pass takes the
// Adam step of A (scale multiplies the gradient, as in atlas_adam; A, m, s
// updated in place).
constexpr int ATLAS_SUB_MAX = 4;
constexpr int ATLAS_FUSED_MAX = 16;
int atlas_sub_batches(int nb);
struct AtlasStepArgs {
    float* A;
    float* m;
    float* s;
    float scale, lr_c1, isc2, b1, b2, eps;
};
cudaError_t atlas_sgd_fused_forward(const float* const* Jrows, const float* const* jsrows, int nb, const float* A,
                                    int r, float eps, int metric, float* coef, double* partials, const Vol& v,
                                    float* P, cudaStream_t s);
cudaError_t atlas_sgd_fused_adam(const float* const* Jrows, int nb, const float* coef, int r, float* A, float* m,
                                 float* s_, float scale, float lr_c1, float isc2, float b1, float b2, float eps,
                                 float* gacc, const Vol& v, float* P, cudaStream_t s);
// the same adjoint passes writing g [V] = scale * the batch's summed gradient
// instead of stepping A (a sharded cohort sums g over its ranks first)
cudaError_t atlas_sgd_fused_grad(const float* const* Jrows, int nb, const float* coef, int r, const float* A,
                                 float scale, float* g, float* gacc, const Vol& v, float* P, cudaStream_t s);

}  // namespace darc_impl
