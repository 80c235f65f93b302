// k_lncc.cu -- local (windowed) NCC forward and adjoint (sm_103a).
//
// Patch-wise NCC (arXiv 2508.10743, Sec. "Dissimilarity metrics"), read as
// the squared correlation over the w^3 window centred at each voxel, zero
// padding outside the volume, normalised by N = w^3:
//   P = S_JA - S_J S_A / N, sJ = S_JJ - S_J^2 / N, sA = S_AA - S_A^2 / N,
//   cc = P^2 / (sJ sA + eps),  L = -1/V sum_x cc(x).
// The adjoint is again a box sum (the zero-padded box filter is
// self-adjoint):  dL/dJ(y) = -1/V [Box(a) + 2 J(y) Box(b) + A(y) Box(g)]
// with a = dcc/dS_J, b = dcc/dS_JJ, g = dcc/dS_JA (mirror for A).
//
// One kernel template streams a 32 x 16 (x, y) column tile through z: each
// input plane (with an r-voxel halo, zero outside) is staged in shared
// memory, summed along x and then y, and its 2-D window sums go into a ring
// of w planes; every output plane sums its w ring entries afresh (no
// running sum, so no drift along z).  An `Op` supplies the per-voxel input
// channels and consumes the window sums.
#include "kernels.h"

#include <algorithm>

namespace darc_impl {
namespace {

constexpr int BX = 32, BY = 16, BNT = 256, ZCHUNK = 32;

template <int NCH>
size_t box_smem_bytes(int r)
{
    const int w = 2 * r + 1, LX = BX + 2 * r, LY = BY + 2 * r;
    return sizeof(float) * ((size_t)NCH * LY * LX + (size_t)NCH * LY * BX + (size_t)w * NCH * BY * BX);
}

template <int NCH, class Op>
__global__ void __launch_bounds__(BNT) box_kernel(Op op, Vol v, int r, int nzc)
{
    extern __shared__ float sm[];
    __shared__ double red[32];
    const int w = 2 * r + 1, LX = BX + 2 * r, LY = BY + 2 * r;
    float* tile = sm;                               // [NCH][LY][LX]
    float* xs = tile + NCH * LY * LX;               // [NCH][LY][BX]
    float* ring = xs + NCH * LY * BX;               // [w][NCH][BY][BX]
    const int tid = threadIdx.x;
    const int b = blockIdx.z / nzc, zc = blockIdx.z % nzc;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int z0 = zc * ZCHUNK, z1 = min(v.D, z0 + ZCHUNK);
    float acc = 0.f;
    for (int zi = z0 - r; zi < z1 + r; ++zi) {
        const bool zin = (zi >= 0) && (zi < v.D);
        for (int e = tid; e < LY * LX; e += BNT) {
            const int ly = e / LX, lx = e - ly * LX;
            const int y = y0 - r + ly, x = x0 - r + lx;
            float vals[NCH];
            if (zin && y >= 0 && y < v.H && x >= 0 && x < v.W) {
                op.load(b, ((long long)zi * v.H + y) * v.W + x, vals);
            } else {
#pragma unroll
                for (int c = 0; c < NCH; ++c) vals[c] = 0.f;
            }
#pragma unroll
            for (int c = 0; c < NCH; ++c) tile[(c * LY + ly) * LX + lx] = vals[c];
        }
        __syncthreads();
        for (int e = tid; e < LY * BX; e += BNT) {
            const int ly = e / BX, tx = e - ly * BX;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const float* row = tile + (c * LY + ly) * LX + tx;
                float s = 0.f;
                for (int d = 0; d < w; ++d) s += row[d];
                xs[(c * LY + ly) * BX + tx] = s;
            }
        }
        __syncthreads();
        const int slot = (zi - (z0 - r)) % w;
        for (int e = tid; e < BY * BX; e += BNT) {
            const int ty = e / BX, tx = e - ty * BX;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const float* col = xs + (c * LY + ty) * BX + tx;
                float s = 0.f;
                for (int d = 0; d < w; ++d) s += col[d * BX];
                ring[((slot * NCH + c) * BY + ty) * BX + tx] = s;
            }
        }
        __syncthreads();
        const int zo = zi - r;
        if (zo >= z0) {
            for (int e = tid; e < BY * BX; e += BNT) {
                const int ty = e / BX, tx = e - ty * BX;
                const int y = y0 + ty, x = x0 + tx;
                if (y < v.H && x < v.W) {
                    float S[NCH];
#pragma unroll
                    for (int c = 0; c < NCH; ++c) {
                        float s = 0.f;
                        for (int k = 0; k < w; ++k) s += ring[((k * NCH + c) * BY + ty) * BX + tx];
                        S[c] = s;
                    }
                    acc += op.emit(b, zo, y, x, ((long long)zo * v.H + y) * v.W + x, S);
                }
            }
        }
    }
    if (Op::kReduces) {
        const double s = block_sum(acc, red);
        if (tid == 0)
            op.partial(b, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zc), s);
    }
}

// ---------------------------------------------------------------------------
struct AtlasStatsOp {
    static constexpr bool kReduces = false;
    const float* A;
    float* stats;
    long long V;
    __device__ void load(int, long long l, float* o) const
    {
        const float a = __ldg(A + l);
        o[0] = a;
        o[1] = a * a;
    }
    __device__ float emit(int, int, int, int, long long l, const float* S) const
    {
        stats[l] = S[0];
        stats[V + l] = S[1];
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
    int wrt_atlas;
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
        const CCTerms t = cc_terms(S[0], S[1], S[2], __ldg(stats + l), __ldg(stats + V + l), invN,
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

struct RegW {
    float z, y, x;
};

struct BwdWarpRegOp {
    static constexpr bool kReduces = true;
    const float* J;
    const float* A;
    const float* coef;
    const float* I;
    size_t I_bstride;
    const float* uT;
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
        const float* ub = uT + (size_t)b * 3 * v.V;
        const Cell c = make_cell(z, y, x, __ldg(ub + l), __ldg(ub + v.V + l), __ldg(ub + 2 * v.V + l), v);
        float dz, dy, dx;
        tri_grad(I + (size_t)b * I_bstride, c, v, dz, dy, dx);
        // diffusion regulariser at x (pairs counted at their lower voxel)
        const long long st[3] = {(long long)v.H * v.W, (long long)v.W, 1};
        const int q[3] = {z, y, x};
        const int n[3] = {v.D, v.H, v.W};
        const float ca[3] = {rw.z, rw.y, rw.x};
        float val = 0.f, g[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a2 = 0; a2 < 3; ++a2) {
            const bool up = q[a2] + 1 < n[a2];
            const bool dn = q[a2] > 0;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float* uc = ub + ch * v.V;
                const float cur = __ldg(uc + l);
                const float dup = up ? __ldg(uc + l + st[a2]) - cur : 0.f;
                const float ddn = dn ? cur - __ldg(uc + l - st[a2]) : 0.f;
                val = fmaf(ca[a2] * dup, dup, val);
                g[ch] = fmaf(2.f * ca[a2], ddn - dup, g[ch]);
            }
        }
        float* gb = gT + (size_t)b * 3 * v.V;
        gb[l] = fmaf(gJ, dz, lambda * g[0]);
        gb[v.V + l] = fmaf(gJ, dy, lambda * g[1]);
        gb[2 * v.V + l] = fmaf(gJ, dx, lambda * g[2]);
        return val;
    }
    __device__ void partial(int b, int blk, double s) const { partials[(size_t)b * nblk + blk] = s; }
};

template <int NCH, class Op>
cudaError_t launch_box(const Op& op, int B, const Vol& v, int r, cudaStream_t s)
{
    const size_t smem = box_smem_bytes<NCH>(r);
    static bool attr_set = false;   // once per instantiation, sized for the largest window (r = 8)
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(box_kernel<NCH, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)box_smem_bytes<NCH>(8));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int nzc = div_up(v.D, ZCHUNK);
    const dim3 grid(div_up(v.W, BX), div_up(v.H, BY), nzc * B);
    box_kernel<NCH, Op><<<grid, BNT, smem, s>>>(op, v, r, nzc);
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

int box_blocks(const Vol& v) { return div_up(v.W, BX) * div_up(v.H, BY) * div_up(v.D, ZCHUNK); }

cudaError_t atlas_stats(const float* A, float* stats, int r, const Vol& v, cudaStream_t s)
{
    AtlasStatsOp op{A, stats, v.V};
    return launch_box<2>(op, 1, v, r, s);
}

cudaError_t lncc_forward(const float* J, const int* subj, const float* A, const float* stats,
                         int r, float eps, int wrt_atlas, float* coef, double* partials, int B,
                         const Vol& v, cudaStream_t s)
{
    const int w = 2 * r + 1;
    FwdOp op{J, subj, A, stats, coef, partials, box_blocks(v), v.V,
             (float)(1.0 / ((double)w * w * w)), eps, (float)(-1.0 / (double)v.V), wrt_atlas};
    return launch_box<3>(op, B, v, r, s);
}

cudaError_t lncc_backward(const float* J, const int* subj, const float* A, const float* coef,
                          int r, int wrt_atlas, float* g, int B, const Vol& v, cudaStream_t s)
{
    BwdOp op{J, subj, A, coef, g, v.V, (float)(-1.0 / (double)v.V), wrt_atlas};
    return launch_box<3>(op, B, v, r, s);
}

cudaError_t lncc_backward_warp_reg(const float* J, const float* A, const float* coef, int r,
                                   const float* I, size_t I_bstride, const float* uT,
                                   float lambda, float* gT, double* partials, int B, const Vol& v,
                                   cudaStream_t s)
{
    auto w = [&](int n) { return (float)(1.0 / (3.0 * (double)v.V * (double)(n - 1) / (double)n)); };
    BwdWarpRegOp op{J, A, coef, I, I_bstride, uT, gT, partials, box_blocks(v), v,
                    (float)(-1.0 / (double)v.V), lambda, RegW{w(v.D), w(v.H), w(v.W)}};
    return launch_box<3>(op, B, v, r, s);
}

cudaError_t sum_images(const float* g, int B, float* out, const Vol& v, cudaStream_t s)
{
    const int blocks = (int)std::min<long long>((v.V + 255) / 256, 152LL * 16);
    sum_images_kernel<<<blocks, 256, 0, s>>>(g, B, out, v.V);
    return cudaGetLastError();
}

}  // namespace darc_impl
