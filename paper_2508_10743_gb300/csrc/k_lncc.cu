// k_lncc.cu -- patch-wise dissimilarities (local NCC, SSIM): forward and
// adjoint (sm_103a).
//
// Patch-wise NCC (arXiv 2508.10743, Sec. "Dissimilarity metrics"), read as
// the squared correlation over the w^3 window centred at each voxel, zero
// padding outside the volume, normalised by N = w^3:
//   P = S_JA - S_J S_A / N, sJ = S_JJ - S_J^2 / N, sA = S_AA - S_A^2 / N,
//   cc = P^2 / (sJ sA + eps),  L = -1/V sum_x cc(x).
// SSIM (same section) over the same windows and sums: mu = S/N, var and
// cov from the second moments, ssim = (2 muJ muA + C1)(2 cov + C2) /
// ((muJ^2 + muA^2 + C1)(varJ + varA + C2)), L = -1/V sum_x ssim(x).
// The adjoint is again a box sum (the zero-padded box filter is
// self-adjoint):  dL/dJ(y) = -1/V [Box(a) + 2 J(y) Box(b) + A(y) Box(g)]
// with a = dcc/dS_J, b = dcc/dS_JJ, g = dcc/dS_JA (mirror for A).
//
// Every box sum is two kernels sharing an `Op` (input channels, epilogue):
// an XY kernel, one warp per plane strip of 32 columns, stages each row with
// its halo in warp-private shared memory, sums x windows from it and keeps a
// running y sum (lane-private ring of the last w rows), writing the 2-D
// window sums; a Z kernel, one thread per column, keeps a running z sum over
// chunks of 32 planes and applies the epilogue.  Zero padding throughout.
#include "kernels.h"

#include <algorithm>
#include <type_traits>

namespace darc_impl {
namespace {

// XY pass: a block of XW warps covers a 32-column strip, YC output rows and
// XW consecutive planes (one plane per warp).
#ifndef DARC_BOX_XW
#define DARC_BOX_XW 8
#endif
#ifndef DARC_BOX_YC
#define DARC_BOX_YC 64
#endif
#ifndef DARC_BOX_YC_WIDE_BATCH
#define DARC_BOX_YC_WIDE_BATCH 192
#endif
constexpr int XW = DARC_BOX_XW, YC = DARC_BOX_YC;
// strip height for launches of eight or more images (enough blocks without
// splitting the columns as finely)
constexpr int YC_WIDE = DARC_BOX_YC_WIDE_BATCH;
// Z pass: 32 x 8 columns per block, ZC output planes per thread; the
// entering and leaving values of ZU planes are loaded ahead of their sums:
// four planes for one or two channels, two for three or more (whose wider
// state and epilogues need the registers for occupancy); ZMINB > 0 asks for
// that many resident blocks per SM (a register cap).
#ifndef DARC_BOX_ZC
#define DARC_BOX_ZC 32
#endif
#ifndef DARC_BOX_ZU_NARROW
#define DARC_BOX_ZU_NARROW 4
#endif
#ifndef DARC_BOX_ZU_WIDE
#define DARC_BOX_ZU_WIDE 2
#endif
#ifndef DARC_BOX_ZMINB
#define DARC_BOX_ZMINB 0
#endif
constexpr int ZX = 32, ZY = 8, ZC = DARC_BOX_ZC;
// Small launches (one small image) would leave most SMs idle with these
// tiles: the XY strip and the Z chunk shrink (down to 16 rows, 8 planes)
// until a launch has at least two blocks per SM.
#ifndef DARC_BOX_MIN_BLOCKS
#define DARC_BOX_MIN_BLOCKS (2 * 152)
#endif
constexpr int BOX_MIN_BLOCKS = DARC_BOX_MIN_BLOCKS, YC_MIN = 16, ZC_MIN = 8;

size_t xy_smem_bytes(int nch, int r)
{
    const int w = 2 * r + 1;
    return sizeof(float) * (size_t)XW * ((size_t)nch * (32 + 2 * r) + (size_t)(w + 1) * nch * 32);
}

// P[b][c] = 2-D window sums (x, y) of the input channels of every plane.
// WT: the window edge when known at compile time (the x sums unroll), or 0.
template <int NCH, class Op, int WT>
__global__ void __launch_bounds__(XW * 32) box_xy_kernel(Op op, Vol v, int r, float* __restrict__ P, int nzb,
                                                         int yc)
{
    extern __shared__ float sm[];
    const int w = WT > 0 ? WT : 2 * r + 1, LXW = 32 + 2 * r, NR = w + 1;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int b = blockIdx.z / nzb;
    const int z = (blockIdx.z % nzb) * XW + wp;
    if (z >= v.D) return;                          // whole warp; no block-level barrier below
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * yc;
    const int x = x0 + lane;
    float* row = sm + (size_t)wp * (NCH * LXW + NR * NCH * 32);
    float* ring = row + NCH * LXW;
    const int yend = min(y0 + yc, v.H);
    float ys[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) ys[c] = 0.f;
    // a row with its halo is at most 32 + 2 * 8 values: two per lane; the
    // next row is loaded into registers while the current one is summed
    float pre[2][NCH];
    auto fetch = [&](int yi) {
        const bool yin = yi >= 0 && yi < v.H;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int j = lane + 32 * k, xx = x0 - r + j;
            if (j < LXW && yin && xx >= 0 && xx < v.W) {
                op.load(b, ((long long)z * v.H + yi) * v.W + xx, pre[k]);
            } else {
#pragma unroll
                for (int c = 0; c < NCH; ++c) pre[k][c] = 0.f;
            }
        }
    };
    fetch(y0 - r);
    for (int yi = y0 - r; yi < yend + r; ++yi) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int j = lane + 32 * k;
            if (j < LXW) {
#pragma unroll
                for (int c = 0; c < NCH; ++c) row[c * LXW + j] = pre[k][c];
            }
        }
        if (yi + 1 < yend + r) fetch(yi + 1);
        __syncwarp();
        const int slot = (yi - (y0 - r)) % NR, old = (slot + 1) % NR;
        const bool drop = yi - w >= y0 - r;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const float* rr = row + c * LXW + lane;
            float xsum = 0.f;
            if constexpr (WT > 0) {
#pragma unroll
                for (int d = 0; d < WT; ++d) xsum += rr[d];
            } else {
                for (int d = 0; d < w; ++d) xsum += rr[d];
            }
            ys[c] += xsum;
            if (drop) ys[c] -= ring[(old * NCH + c) * 32 + lane];
            ring[(slot * NCH + c) * 32 + lane] = xsum;     // lane-private
        }
        __syncwarp();
        const int yo = yi - r;
        if (yo >= y0 && x < v.W) {
            const long long l = ((long long)z * v.H + yo) * v.W + x;
#pragma unroll
            for (int c = 0; c < NCH; ++c) P[((size_t)b * NCH + c) * v.V + l] = ys[c];
        }
    }
}

// Number of block reductions an Op's epilogue feeds: 1 (emit returns the
// value) unless the Op declares kNRed, whose emit_n adds kNRed values.
template <class Op, class = void>
struct NRed {
    static constexpr int value = 1;
    static constexpr bool multi = false;
};
template <class Op>
struct NRed<Op, std::void_t<decltype(Op::kNRed)>> {
    static constexpr int value = Op::kNRed;
    static constexpr bool multi = true;
};

// 3-D window sums along z from the 2-D sums, then the Op's epilogue
// Resident blocks per SM an Op asks of its Z pass (a register cap), else ZMINB.
template <class Op, class = void>
struct ZMinBlocks {
    static constexpr int value = DARC_BOX_ZMINB;
};
template <class Op>
struct ZMinBlocks<Op, std::void_t<decltype(Op::kZMinBlocks)>> {
    static constexpr int value = Op::kZMinBlocks;
};

template <int NCH, class Op>
__global__ void __launch_bounds__(ZX * ZY, ZMinBlocks<Op>::value)
box_z_kernel(Op op, Vol v, int r, const float* __restrict__ P, int nzc, int zlen)
{
    __shared__ double red[32];
    const int x = blockIdx.x * ZX + threadIdx.x;
    const int y = blockIdx.y * ZY + threadIdx.y;
    const int b = blockIdx.z / nzc, zc = blockIdx.z % nzc;
    const int z0 = zc * zlen, z1 = min(v.D, z0 + zlen);
    constexpr int ZU = NCH >= 3 ? DARC_BOX_ZU_WIDE : DARC_BOX_ZU_NARROW;
    constexpr int NR = NRed<Op>::value;
    float acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = 0.f;
    if (x < v.W && y < v.H) {
        const long long col = (long long)y * v.W + x, plane = (long long)v.H * v.W;
        const float* Pb = P + (size_t)b * NCH * v.V;
        float S[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            float s = 0.f;
            for (int q = max(z0 - r, 0); q <= min(z0 + r, v.D - 1); ++q) s += __ldg(Pb + c * v.V + q * plane + col);
            S[c] = s;
        }
        // ZU planes at a time: their entering and leaving planes are loaded
        // first (out-of-range ones as exact zeros), then summed in order
        for (int zo = z0; zo < z1; zo += ZU) {
            float add[ZU][NCH], drp[ZU][NCH];
#pragma unroll
            for (int u = 0; u < ZU; ++u) {
                const int zz = zo + u;
                const bool step = zz > z0 && zz < z1;
                const int qa = zz + r, qd = zz - r - 1;
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    add[u][c] = (step && qa < v.D) ? __ldg(Pb + c * v.V + qa * plane + col) : 0.f;
                    drp[u][c] = (step && qd >= 0) ? __ldg(Pb + c * v.V + qd * plane + col) : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < ZU; ++u) {
                const int zz = zo + u;
                if (zz >= z1) break;
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    S[c] += add[u][c];
                    S[c] -= drp[u][c];
                }
                if constexpr (!NRed<Op>::multi)
                    acc[0] += op.emit(b, zz, y, x, zz * plane + col, S);
                else
                    op.emit_n(b, zz, y, x, zz * plane + col, S, acc);
            }
        }
    }
    if (Op::kReduces) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const double s2 = block_sum(acc[k], red);
            if (threadIdx.x == 0 && threadIdx.y == 0)
                op.partial(b * NR + k, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zc), s2);
        }
    }
}

// ---------------------------------------------------------------------------
// Box(f) and Box(f^2) of each image of a batch: stats[b] = {Box f_b, Box f_b^2}
struct StatsOp {
    static constexpr bool kReduces = false;
    const float* A;
    float* stats;
    long long V;
    __device__ void load(int b, long long l, float* o) const
    {
        const float a = __ldg(A + (size_t)b * V + l);
        o[0] = a;
        o[1] = a * a;
    }
    __device__ float emit(int b, int, int, int, long long l, const float* S) const
    {
        float* sb = stats + (size_t)b * 2 * V;
        sb[l] = S[0];
        sb[V + l] = S[1];
        return 0.f;
    }
    __device__ void partial(int, int, double) const {}
};

struct CCTerms {
    float cc, c0, c1, c2;
};

// cc and its derivatives from the five window sums (wrt J, or wrt A)
__device__ __forceinline__ CCTerms cc_terms(float SJ, float SJJ, float SJA, float SA, float SAA,
                                            float invN, float eps, bool wrt_atlas)
{
    const float P = SJA - SJ * SA * invN;
    const float vJ = fmaxf(SJJ - SJ * SJ * invN, 0.f);
    const float vA = fmaxf(SAA - SA * SA * invN, 0.f);
    const float Q = fmaf(vJ, vA, eps);
    const float iQ = 1.f / Q;
    CCTerms t;
    t.cc = P * P * iQ;
    const float dP = 2.f * P * iQ;
    if (!wrt_atlas) {
        const float dvJ = -t.cc * vA * iQ;
        t.c0 = dP * (-SA * invN) + dvJ * (-2.f * SJ * invN);
        t.c1 = dvJ;
    } else {
        const float dvA = -t.cc * vJ * iQ;
        t.c0 = dP * (-SJ * invN) + dvA * (-2.f * SA * invN);
        t.c1 = dvA;
    }
    t.c2 = dP;
    return t;
}

// SSIM over the same window from the same five sums (Wang et al. 2004,
// C1 = (0.01)^2, C2 = (0.03)^2 for intensities on [0, 1]), and its
// derivatives wrt the sums of the differentiated image X (J, or A when
// wrt_atlas): c0 = dssim/dS_X, c1 = dssim/dS_XX, c2 = dssim/dS_XY.
__device__ __forceinline__ CCTerms ssim_terms(float SJ, float SJJ, float SJA, float SA, float SAA,
                                              float invN, bool wrt_atlas)
{
    constexpr float C1 = 1.0e-4f, C2 = 9.0e-4f;
    const float mJ = SJ * invN, mA = SA * invN;
    const float vJ = SJJ * invN - mJ * mJ, vA = SAA * invN - mA * mA;
    const float cJA = SJA * invN - mJ * mA;
    const float a1 = fmaf(2.f * mJ, mA, C1), a2 = fmaf(2.f, cJA, C2);
    const float b1 = mJ * mJ + mA * mA + C1, b2 = vJ + vA + C2;
    const float ib1 = 1.f / b1, ib2 = 1.f / b2, ib = ib1 * ib2;
    CCTerms t;
    t.cc = a1 * a2 * ib;
    const float mX = wrt_atlas ? mA : mJ, mY = wrt_atlas ? mJ : mA;
    t.c0 = 2.f * invN * (mY * (a2 - a1) * ib - mX * t.cc * (ib1 - ib2));
    t.c1 = -t.cc * invN * ib2;
    t.c2 = 2.f * invN * a1 * ib;
    return t;
}

// the patch-wise metric of a launch: 0 = local NCC, 1 = SSIM
__device__ __forceinline__ CCTerms patch_terms(int metric, float SJ, float SJJ, float SJA, float SA, float SAA,
                                               float invN, float eps, bool wrt_atlas)
{
    return metric ? ssim_terms(SJ, SJJ, SJA, SA, SAA, invN, wrt_atlas)
                  : cc_terms(SJ, SJJ, SJA, SA, SAA, invN, eps, wrt_atlas);
}

struct FwdOp {
    static constexpr bool kReduces = true;
    const float* J;
    const int* subj;
    const float* A;
    const float* stats;
    float* coef;
    double* partials;
    int nblk;
    long long V;
    float invN, eps, negInvV;
    int wrt_atlas, metric;
    __device__ const float* row(int b) const { return J + (size_t)(subj ? subj[b] : b) * V; }
    __device__ void load(int b, long long l, float* o) const
    {
        const float j = __ldg(row(b) + l), a = __ldg(A + l);
        o[0] = j;
        o[1] = j * j;
        o[2] = j * a;
    }
    __device__ float emit(int b, int, int, int, long long l, const float* S) const
    {
        const CCTerms t = patch_terms(metric, S[0], S[1], S[2], __ldg(stats + l), __ldg(stats + V + l), invN,
                                      eps, wrt_atlas != 0);
        float* cb = coef + (size_t)b * 3 * V;
        cb[l] = t.c0;
        cb[V + l] = t.c1;
        cb[2 * V + l] = t.c2;
        return t.cc * negInvV;
    }
    __device__ void partial(int b, int blk, double s) const { partials[(size_t)b * nblk + blk] = s; }
};

struct BwdOp {
    static constexpr bool kReduces = false;
    const float* J;
    const int* subj;
    const float* A;
    const float* coef;
    float* g;
    long long V;
    float negInvV;
    int wrt_atlas;
    __device__ void load(int b, long long l, float* o) const
    {
        const float* cb = coef + (size_t)b * 3 * V;
        o[0] = __ldg(cb + l);
        o[1] = __ldg(cb + V + l);
        o[2] = __ldg(cb + 2 * V + l);
    }
    __device__ float emit(int b, int, int, int, long long l, const float* S) const
    {
        const float j = __ldg(J + (size_t)(subj ? subj[b] : b) * V + l), a = __ldg(A + l);
        const float X = wrt_atlas ? a : j, Y = wrt_atlas ? j : a;
        g[(size_t)b * V + l] = negInvV * (S[0] + 2.f * X * S[1] + Y * S[2]);
        return 0.f;
    }
    __device__ void partial(int, int, double) const {}
};

// U: the layout of u_T (PlanarField or PackedField)
// three resident blocks per SM for its Z pass (at most 85 registers): the
// epilogue's gathers and neighbour loads want occupancy more than registers
#ifndef DARC_WR_MINB
#define DARC_WR_MINB 3
#endif
template <class U>
struct BwdWarpRegOp {
    static constexpr bool kReduces = true;
    static constexpr int kZMinBlocks = DARC_WR_MINB;
    const float* J;
    const float* A;
    const float* coef;
    const float* I;
    size_t I_bstride;
    U uT;
    float* gT;
    double* partials;
    int nblk;
    Vol v;
    float negInvV, lambda;
    RegW rw;
    __device__ void load(int b, long long l, float* o) const
    {
        const float* cb = coef + (size_t)b * 3 * v.V;
        o[0] = __ldg(cb + l);
        o[1] = __ldg(cb + v.V + l);
        o[2] = __ldg(cb + 2 * v.V + l);
    }
    __device__ float emit(int b, int z, int y, int x, long long l, const float* S) const
    {
        const float j = __ldg(J + (size_t)b * v.V + l), a = __ldg(A + l);
        const float gJ = negInvV * (S[0] + 2.f * j * S[1] + a * S[2]);
        const U ub = uT.subject(b);
        const float3 d3 = ub.own((int)l);
        const Cell c = make_cell(z, y, x, d3.x, d3.y, d3.z, v);
        float dz, dy, dx;
        tri_grad(I + (size_t)b * I_bstride, c, v, dz, dy, dx);
        // diffusion regulariser at x (pairs counted at their lower voxel)
        float g[3];
        const float val = reg_at_field(ub, v, z, y, x, (int)l, rw, g);
        float* gb = gT + (size_t)b * 3 * v.V;
        gb[l] = fmaf(gJ, dz, lambda * g[0]);
        gb[v.V + l] = fmaf(gJ, dy, lambda * g[1]);
        gb[2 * v.V + l] = fmaf(gJ, dx, lambda * g[2]);
        return val;
    }
    __device__ void partial(int b, int blk, double s) const { partials[(size_t)b * nblk + blk] = s; }
};

// Atlas SGD, forward for one mini-batch: only Box(J A) depends on the atlas;
// Box(J), Box(J^2) come from the per-sweep cache, Box(A), Box(A^2) from the
// atlas statistics.  Writes d cc / d(S_A, S_AA, S_JA) per subject.
struct AtlasFwdOp {
    static constexpr bool kReduces = true;
    const float* J;        // warped cohort [n][V]
    const float* jstats;   // [n][2][V]
    const int* subj;
    const float* A;
    const float* astats;   // [2][V]
    float* coef;           // [nb][3][V]
    double* partials;
    int nblk;
    long long V;
    float invN, eps, negInvV;
    int metric;
    __device__ void load(int b, long long l, float* o) const
    {
        o[0] = __ldg(J + (size_t)subj[b] * V + l) * __ldg(A + l);
    }
    __device__ float emit(int b, int, int, int, long long l, const float* S) const
    {
        const float* js = jstats + (size_t)subj[b] * 2 * V;
        const CCTerms t = patch_terms(metric, __ldg(js + l), __ldg(js + V + l), S[0], __ldg(astats + l),
                                      __ldg(astats + V + l), invN, eps, true);
        float* cb = coef + (size_t)b * 3 * V;
        cb[l] = t.c0;
        cb[V + l] = t.c1;
        cb[2 * V + l] = t.c2;
        return t.cc * negInvV;
    }
    __device__ void partial(int b, int blk, double s) const { partials[(size_t)b * nblk + blk] = s; }
};

// Atlas SGD, adjoint part shared by the batch: Box is linear, so
// sum_b [Box(a_b) + 2 A Box(b_b)] = Box(sum_b a_b) + 2 A Box(sum_b b_b).
struct AtlasBwdSharedOp {
    static constexpr bool kReduces = false;
    const float* coef;     // [nb][3][V]
    int nb;
    const float* A;
    float* out;            // [V]
    long long V;
    __device__ void load(int, long long l, float* o) const
    {
        float sa = 0.f, sb = 0.f;
        for (int b = 0; b < nb; ++b) {
            sa += __ldg(coef + (size_t)b * 3 * V + l);
            sb += __ldg(coef + (size_t)b * 3 * V + V + l);
        }
        o[0] = sa;
        o[1] = sb;
    }
    __device__ float emit(int, int, int, int, long long l, const float* S) const
    {
        out[l] = S[0] + 2.f * __ldg(A + l) * S[1];
        return 0.f;
    }
    __device__ void partial(int, int, double) const {}
};

// Atlas SGD, adjoint part of each subject: J_b Box(g_b).
struct AtlasBwdSubjOp {
    static constexpr bool kReduces = false;
    const float* coef;     // [nb][3][V]
    const float* J;
    const int* subj;
    float* out;            // [nb][V]
    long long V;
    __device__ void load(int b, long long l, float* o) const
    {
        o[0] = __ldg(coef + (size_t)b * 3 * V + 2 * V + l);
    }
    __device__ float emit(int b, int, int, int, long long l, const float* S) const
    {
        out[(size_t)b * V + l] = __ldg(J + (size_t)subj[b] * V + l) * S[0];
        return 0.f;
    }
    __device__ void partial(int, int, double) const {}
};

// Atlas SGD, one box pass per sub-batch of NB <= 4 subjects of a mini-batch
// (rows known on the host): channels Box(A), Box(A^2) and Box(J_b A) for
// each b.  The epilogue evaluates the NB patch metrics and keeps what the
// adjoint needs.  Because Box is linear, the two coefficients that multiply
// terms shared by the batch are summed over b here (and over the earlier
// sub-batches when `accum`): coef [2][V] = {sum_b dm_b/dS_A, sum_b
// dm_b/dS_AA}, coefb [NB][V] = dm_b/dS_JA; loss partials [NB][nblk].
template <int NB, bool ACC>
struct AtlasFwdFusedOp {
    static constexpr bool kReduces = true;
    static constexpr int kNRed = NB;
    const float* J[NB];    // warped subject b [V]
    const float* js[NB];   // its window statistics [2][V]
    const float* A;
    float* coef;
    float* coefb;
    double* partials;
    int nblk;
    long long V;
    float invN, eps, negInvV;
    int metric;
    __device__ void load(int, long long l, float* o) const
    {
        const float a = __ldg(A + l);
        o[0] = a;
        o[1] = a * a;
#pragma unroll
        for (int b = 0; b < NB; ++b) o[2 + b] = __ldg(J[b] + l) * a;
    }
    __device__ void emit_n(int, int, int, int, long long l, const float* S, float* acc) const
    {
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const CCTerms t = patch_terms(metric, __ldg(js[b] + l), __ldg(js[b] + V + l), S[2 + b], S[0], S[1],
                                          invN, eps, true);
            s0 += t.c0;
            s1 += t.c1;
            coefb[(size_t)b * V + l] = t.c2;
            acc[b] += t.cc * negInvV;
        }
        if (ACC) {
            s0 = coef[l] + s0;
            s1 = coef[V + l] + s1;
        }
        coef[l] = s0;
        coef[V + l] = s1;
    }
    __device__ void partial(int b, int blk, double s) const { partials[(size_t)b * nblk + blk] = s; }
};

// Atlas SGD, the adjoint of a mini-batch, one box pass per sub-batch:
//   g = Box(sum a) + 2 A Box(sum b) + sum_b J_b Box(g_b)
// SHARED (the first sub-batch) adds the terms shared by the batch, later
// sub-batches add to the running sum `gin`.  The last pass either takes the
// Adam step with g * scale (m != null: A, m, s updated in place, each read
// and written only at the thread's own voxel) or writes g * gscale to gout
// (a sharded cohort sums g over its ranks before the step); earlier passes
// write the running sum to gout.  The XY pass reads the coefficients alone.
template <int NB, bool SHARED, bool ADAM>
struct AtlasBwdStepOp {
    static constexpr bool kReduces = false;
    const float* J[NB];
    const float* coef;     // [2][V] shared coefficients (SHARED)
    const float* coefb;    // [NB][V] this sub-batch's
    float* A;
    float* m;
    float* s;
    const float* gin;
    float* gout;
    long long V;
    float gscale, scale, lr_c1, isc2, b1, b2, eps;
    __device__ void load(int, long long l, float* o) const
    {
        if (SHARED) {
            o[0] = __ldg(coef + l);
            o[1] = __ldg(coef + V + l);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) o[(SHARED ? 2 : 0) + b] = __ldg(coefb + (size_t)b * V + l);
    }
    __device__ float emit(int, int, int, int, long long l, const float* S) const
    {
        float a = A[l];
        float g = SHARED ? S[0] + 2.f * a * S[1] : gin[l];
        // each subject's term rounded on its own, as a separate product
#pragma unroll
        for (int b = 0; b < NB; ++b) g += __fmul_rn(__ldg(J[b] + l), S[(SHARED ? 2 : 0) + b]);
        if (ADAM) {
            float mm = m[l], ss = s[l];
            adam1(a, mm, ss, g * scale, b1, b2, lr_c1, isc2, eps);
            A[l] = a;
            m[l] = mm;
            s[l] = ss;
        } else {
            gout[l] = g * gscale;
        }
        return 0.f;
    }
    __device__ void partial(int, int, double) const {}
};

template <int NCH, class Op, int WT>
cudaError_t launch_xy(const Op& op, int B, const Vol& v, int r, float* P, cudaStream_t s)
{
    static bool attr_set = false;   // once per instantiation, sized for its largest window
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(box_xy_kernel<NCH, Op, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)xy_smem_bytes(NCH, WT > 0 ? WT / 2 : 8));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int nzb = div_up(v.D, XW);
    const int yc = box_yc(v, B);
    box_xy_kernel<NCH, Op, WT><<<dim3(div_up(v.W, 32), div_up(v.H, yc), nzb * B), XW * 32, xy_smem_bytes(NCH, r),
                                 s>>>(op, v, r, P, nzb, yc);
    return cudaGetLastError();
}

template <int NCH, class Op>
cudaError_t launch_box(const Op& op, int B, const Vol& v, int r, float* P, cudaStream_t s)
{
    // windows of 3 to 9 voxels (the workloads' own) get their unrolled XY pass
    cudaError_t e;
    switch (r) {
    case 1: e = launch_xy<NCH, Op, 3>(op, B, v, r, P, s); break;
    case 2: e = launch_xy<NCH, Op, 5>(op, B, v, r, P, s); break;
    case 3: e = launch_xy<NCH, Op, 7>(op, B, v, r, P, s); break;
    case 4: e = launch_xy<NCH, Op, 9>(op, B, v, r, P, s); break;
    default: e = launch_xy<NCH, Op, 0>(op, B, v, r, P, s); break;
    }
    if (e != cudaSuccess) return e;
    const int zlen = box_zc(v, B), nzc = div_up(v.D, zlen);
    box_z_kernel<NCH, Op><<<dim3(div_up(v.W, ZX), div_up(v.H, ZY), nzc * B), dim3(ZX, ZY), 0, s>>>(op, v, r, P, nzc,
                                                                                                 zlen);
    return cudaGetLastError();
}

__global__ void sum_images_kernel(const float* __restrict__ g, int B, float* __restrict__ out,
                                  long long V)
{
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < V;
         l += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < B; ++b) s += __ldg(g + (size_t)b * V + l);
        out[l] = s;
    }
}

}  // namespace

int box_yc(const Vol& v, int B)
{
    int yc = B >= 8 ? YC_WIDE : YC;
    while (yc > YC_MIN && (long long)div_up(v.W, 32) * div_up(v.H, yc) * div_up(v.D, XW) * B < BOX_MIN_BLOCKS)
        yc /= 2;
    return std::max(yc, YC_MIN);
}

int box_zc(const Vol& v, int B)
{
    int zc = ZC;
    while (zc > ZC_MIN && (long long)div_up(v.W, ZX) * div_up(v.H, ZY) * div_up(v.D, zc) * B < BOX_MIN_BLOCKS) zc /= 2;
    return std::max(zc, ZC_MIN);
}

int box_blocks(const Vol& v, int B) { return div_up(v.W, ZX) * div_up(v.H, ZY) * div_up(v.D, box_zc(v, B)); }

int box_blocks_max(const Vol& v) { return div_up(v.W, ZX) * div_up(v.H, ZY) * div_up(v.D, ZC_MIN); }

cudaError_t atlas_stats(const float* A, float* stats, int r, const Vol& v, float* P, cudaStream_t s)
{
    StatsOp op{A, stats, v.V};
    return launch_box<2>(op, 1, v, r, P, s);
}

cudaError_t image_stats(const float* J, float* stats, int B, int r, const Vol& v, float* P, cudaStream_t s)
{
    StatsOp op{J, stats, v.V};
    return launch_box<2>(op, B, v, r, P, s);
}

cudaError_t atlas_sgd_forward(const float* J, const float* jstats, const int* subj, const float* A,
                              const float* astats, int r, float eps, int metric, float* coef, double* partials,
                              int nb, const Vol& v, float* P, cudaStream_t s)
{
    const int w = 2 * r + 1;
    AtlasFwdOp op{J, jstats, subj, A, astats, coef, partials, box_blocks(v, nb), v.V,
                  (float)(1.0 / ((double)w * w * w)), eps, (float)(-1.0 / (double)v.V), metric};
    return launch_box<1>(op, nb, v, r, P, s);
}

cudaError_t atlas_sgd_backward(const float* J, const int* subj, const float* A, const float* coef,
                               int r, float* gshared, float* gsubj, int nb, const Vol& v, float* P,
                               cudaStream_t s)
{
    AtlasBwdSharedOp shared{coef, nb, A, gshared, v.V};
    cudaError_t e = launch_box<2>(shared, 1, v, r, P, s);
    if (e != cudaSuccess) return e;
    AtlasBwdSubjOp each{coef, J, subj, gsubj, v.V};
    return launch_box<1>(each, nb, v, r, P, s);
}

namespace {
template <int NB, bool ACC>
cudaError_t atlas_fused_fwd_nb(const float* const* Jrows, const float* const* jsrows, const float* A, int r,
                               float eps, int metric, float* coef, float* coefb, double* partials, const Vol& v,
                               float* P, cudaStream_t s)
{
    const int w = 2 * r + 1;
    AtlasFwdFusedOp<NB, ACC> op{};
    for (int b = 0; b < NB; ++b) {
        op.J[b] = Jrows[b];
        op.js[b] = jsrows[b];
    }
    op.A = A;
    op.coef = coef;
    op.coefb = coefb;
    op.partials = partials;
    op.nblk = box_blocks(v, 1);
    op.V = v.V;
    op.invN = (float)(1.0 / ((double)w * w * w));
    op.eps = eps;
    op.negInvV = (float)(-1.0 / (double)v.V);
    op.metric = metric;
    return launch_box<2 + NB>(op, 1, v, r, P, s);
}

template <int NB, bool SHARED, bool ADAM>
cudaError_t atlas_step_nb(const float* const* Jrows, const float* coef, const float* coefb, int r,
                          const AtlasStepArgs& q, const float* gin, float* gout, float gscale, const Vol& v, float* P,
                          cudaStream_t s)
{
    AtlasBwdStepOp<NB, SHARED, ADAM> op{};
    for (int b = 0; b < NB; ++b) op.J[b] = Jrows[b];
    op.coef = coef;
    op.coefb = coefb;
    op.A = q.A;
    op.m = q.m;
    op.s = q.s;
    op.gin = gin;
    op.gout = gout;
    op.V = v.V;
    op.gscale = gscale;
    op.scale = q.scale;
    op.lr_c1 = q.lr_c1;
    op.isc2 = q.isc2;
    op.b1 = q.b1;
    op.b2 = q.b2;
    op.eps = q.eps;
    return launch_box<(SHARED ? 2 : 0) + NB>(op, 1, v, r, P, s);
}

template <bool SHARED, bool ADAM>
cudaError_t atlas_step_pass(const float* const* Jrows, int nb, const float* coef, const float* coefb, int r,
                            const AtlasStepArgs& q, const float* gin, float* gout, float gscale, const Vol& v,
                            float* P, cudaStream_t s)
{
    switch (nb) {
    case 1: return atlas_step_nb<1, SHARED, ADAM>(Jrows, coef, coefb, r, q, gin, gout, gscale, v, P, s);
    case 2: return atlas_step_nb<2, SHARED, ADAM>(Jrows, coef, coefb, r, q, gin, gout, gscale, v, P, s);
    case 3: return atlas_step_nb<3, SHARED, ADAM>(Jrows, coef, coefb, r, q, gin, gout, gscale, v, P, s);
    case 4: return atlas_step_nb<4, SHARED, ADAM>(Jrows, coef, coefb, r, q, gin, gout, gscale, v, P, s);
    default: return cudaErrorInvalidValue;
    }
}

// sub-batch k of K over nb subjects: first subject and size (sizes differ by one at most)
void atlas_sub_batch(int nb, int k, int& off, int& cnt)
{
    const int K = atlas_sub_batches(nb);
    off = (int)((long long)nb * k / K);
    cnt = (int)((long long)nb * (k + 1) / K) - off;
}

}  // namespace

int atlas_sub_batches(int nb) { return (nb + ATLAS_SUB_MAX - 1) / ATLAS_SUB_MAX; }

cudaError_t atlas_sgd_fused_forward(const float* const* Jrows, const float* const* jsrows, int nb, const float* A,
                                    int r, float eps, int metric, float* coef, double* partials, const Vol& v,
                                    float* P, cudaStream_t s)
{
    if (nb < 1 || nb > ATLAS_FUSED_MAX) return cudaErrorInvalidValue;
    const int K = atlas_sub_batches(nb), nblk = box_blocks(v, 1);
    for (int k = 0; k < K; ++k) {
        int off, cnt;
        atlas_sub_batch(nb, k, off, cnt);
        float* coefb = coef + (size_t)(2 + off) * v.V;
        double* pk = partials + (size_t)off * nblk;
        cudaError_t e;
        const float* const* J = Jrows + off;
        const float* const* js = jsrows + off;
        if (k == 0) {
            switch (cnt) {
            case 1: e = atlas_fused_fwd_nb<1, false>(J, js, A, r, eps, metric, coef, coefb, pk, v, P, s); break;
            case 2: e = atlas_fused_fwd_nb<2, false>(J, js, A, r, eps, metric, coef, coefb, pk, v, P, s); break;
            case 3: e = atlas_fused_fwd_nb<3, false>(J, js, A, r, eps, metric, coef, coefb, pk, v, P, s); break;
            case 4: e = atlas_fused_fwd_nb<4, false>(J, js, A, r, eps, metric, coef, coefb, pk, v, P, s); break;
            default: e = cudaErrorInvalidValue;
            }
        } else {
            switch (cnt) {
            case 1: e = atlas_fused_fwd_nb<1, true>(J, js, A, r, eps, metric, coef, coefb, pk, v, P, s); break;
            case 2: e = atlas_fused_fwd_nb<2, true>(J, js, A, r, eps, metric, coef, coefb, pk, v, P, s); break;
            case 3: e = atlas_fused_fwd_nb<3, true>(J, js, A, r, eps, metric, coef, coefb, pk, v, P, s); break;
            case 4: e = atlas_fused_fwd_nb<4, true>(J, js, A, r, eps, metric, coef, coefb, pk, v, P, s); break;
            default: e = cudaErrorInvalidValue;
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {
cudaError_t atlas_backward_passes(const float* const* Jrows, int nb, const float* coef, int r,
                                  const AtlasStepArgs& q, float* gacc, float* gout, float gscale, bool adam,
                                  const Vol& v, float* P, cudaStream_t s)
{
    if (nb < 1 || nb > ATLAS_FUSED_MAX) return cudaErrorInvalidValue;
    const int K = atlas_sub_batches(nb);
    if (K > 1 && !gacc) return cudaErrorInvalidValue;
    for (int k = 0; k < K; ++k) {
        int off, cnt;
        atlas_sub_batch(nb, k, off, cnt);
        const float* coefb = coef + (size_t)(2 + off) * v.V;
        const bool last = k == K - 1;
        float* go = last ? gout : gacc;
        const float gs = last ? gscale : 1.f;
        const float* const* J = Jrows + off;
        const float* gin = k == 0 ? nullptr : gacc;
        cudaError_t e;
        if (adam && last)
            e = k == 0 ? atlas_step_pass<true, true>(J, cnt, coef, coefb, r, q, gin, go, gs, v, P, s)
                       : atlas_step_pass<false, true>(J, cnt, coef, coefb, r, q, gin, go, gs, v, P, s);
        else
            e = k == 0 ? atlas_step_pass<true, false>(J, cnt, coef, coefb, r, q, gin, go, gs, v, P, s)
                       : atlas_step_pass<false, false>(J, cnt, coef, coefb, r, q, gin, go, gs, v, P, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t atlas_sgd_fused_adam(const float* const* Jrows, int nb, const float* coef, int r, float* A, float* m,
                                 float* s_, float scale, float lr_c1, float isc2, float b1, float b2, float eps,
                                 float* gacc, const Vol& v, float* P, cudaStream_t s)
{
    const AtlasStepArgs q{A, m, s_, scale, lr_c1, isc2, b1, b2, eps};
    return atlas_backward_passes(Jrows, nb, coef, r, q, gacc, nullptr, 1.f, true, v, P, s);
}

cudaError_t atlas_sgd_fused_grad(const float* const* Jrows, int nb, const float* coef, int r, const float* A,
                                 float scale, float* g, float* gacc, const Vol& v, float* P, cudaStream_t s)
{
    const AtlasStepArgs q{const_cast<float*>(A), nullptr, nullptr, 1.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    return atlas_backward_passes(Jrows, nb, coef, r, q, gacc, g, scale, false, v, P, s);
}

cudaError_t lncc_forward(const float* J, const int* subj, const float* A, const float* stats,
                         int r, float eps, int wrt_atlas, int metric, float* coef, double* partials, int B,
                         const Vol& v, float* P, cudaStream_t s)
{
    const int w = 2 * r + 1;
    FwdOp op{J, subj, A, stats, coef, partials, box_blocks(v, B), v.V,
             (float)(1.0 / ((double)w * w * w)), eps, (float)(-1.0 / (double)v.V), wrt_atlas, metric};
    return launch_box<3>(op, B, v, r, P, s);
}

cudaError_t lncc_backward(const float* J, const int* subj, const float* A, const float* coef,
                          int r, int wrt_atlas, float* g, int B, const Vol& v, float* P, cudaStream_t s)
{
    BwdOp op{J, subj, A, coef, g, v.V, (float)(-1.0 / (double)v.V), wrt_atlas};
    return launch_box<3>(op, B, v, r, P, s);
}

cudaError_t lncc_backward_warp_reg(const float* J, const float* A, const float* coef, int r,
                                   const float* I, size_t I_bstride, const float* uT,
                                   float lambda, float* gT, double* partials, int B, const Vol& v,
                                   float* P, cudaStream_t s, int uT_packed)
{
    auto w = [&](int n) { return (float)(1.0 / (3.0 * (double)v.V * (double)(n - 1) / (double)n)); };
    const RegW rw{w(v.D), w(v.H), w(v.W)};
    const float negInvV = (float)(-1.0 / (double)v.V);
    if (uT_packed) {
        if (reinterpret_cast<uintptr_t>(uT) & 15) return cudaErrorMisalignedAddress;
        BwdWarpRegOp<PackedField> op{J, A, coef, I, I_bstride, PackedField{reinterpret_cast<const float4*>(uT), v.V},
                                     gT, partials, box_blocks(v, B), v, negInvV, lambda, rw};
        return launch_box<3>(op, B, v, r, P, s);
    }
    BwdWarpRegOp<PlanarField> op{J, A, coef, I, I_bstride, PlanarField{uT, v.V}, gT, partials, box_blocks(v, B), v,
                                 negInvV, lambda, rw};
    return launch_box<3>(op, B, v, r, P, s);
}

cudaError_t sum_images(const float* g, int B, float* out, const Vol& v, cudaStream_t s)
{
    const int blocks = (int)std::min<long long>((v.V + 255) / 256, 152LL * 16);
    sum_images_kernel<<<blocks, 256, 0, s>>>(g, B, out, v.V);
    return cudaGetLastError();
}

}  // namespace darc_impl
