// k_image.cu -- warp, MSE, diffusion regulariser, label gather, Jacobian
// (sm_103a).
//
// Warp (arXiv 2508.10743, Eq. 2 "I o phi"): W(x) = S(I, x + u(x)).
// MSE (Sec. "Dissimilarity metrics"; mean over voxels).
// Diffusion regulariser (Eq. 2, second term), read as forward differences
// of the displacement, a mean over each axis' voxel pairs and a mean over
// the three axes.
// One-shot label gather (Eq. oneshot) and the Jacobian determinant of the
// folding rate (Sec. "Evaluation metrics").
//
// Per-voxel kernels: 32 x 8 threads, each walking 4 z-planes; loss partial
// sums per block in float, stored as double, reduced in fixed order later.
#include "kernels.h"

#include <algorithm>

namespace darc_impl {
namespace {

RegW reg_weights(const Vol& v)
{
    auto w = [&](int n) { return (float)(1.0 / (3.0 * (double)v.V * (double)(n - 1) / (double)n)); };
    return RegW{w(v.D), w(v.H), w(v.W)};
}

// Value share of voxel x and dR/du_c(x) for a planar field.
__device__ __forceinline__ float reg_at(const float* __restrict__ u, const Vol& v, int z, int y,
                                        int x, long long l, const RegW& rw, float g[3])
{
    return reg_at_field(PlanarField{u, v.V}, v, z, y, x, (int)l, rw, g);
}

__device__ __forceinline__ int block_index_in_subject(int zt)
{
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zt);
}

// U: PlanarField or PackedField (the displacement's layout)
template <class U>
__global__ void __launch_bounds__(VT_THREADS)
warp_kernel(const float* __restrict__ I, size_t I_bstride, U u, float* __restrict__ out, Vol v, int nzt)
{
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    if (x >= v.W || y >= v.H) return;
    const float* Ib = I + (size_t)b * I_bstride;
    const U ub = u.subject(b);
    float* ob = out + (size_t)b * v.V;
    for (int k = 0; k < VT_Z; ++k) {
        const int z = zt * VT_Z + k;
        if (z >= v.D) break;
        const int l = (z * v.H + y) * v.W + x;
        const float3 d = ub.own(l);
        const Cell c = make_cell_warp(z, y, x, d.x, d.y, d.z, v);
        ob[l] = tri(Ib, c, v);
    }
}

__global__ void __launch_bounds__(VT_THREADS)
warp_backward_kernel(const float* __restrict__ I, size_t I_bstride, const float* __restrict__ u,
                     const float* __restrict__ gW, float* __restrict__ gu, Vol v, int nzt)
{
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    if (x >= v.W || y >= v.H) return;
    const float* Ib = I + (size_t)b * I_bstride;
    const float* ub = u + (size_t)b * 3 * v.V;
    const float* gb = gW + (size_t)b * v.V;
    float* ob = gu + (size_t)b * 3 * v.V;
    for (int k = 0; k < VT_Z; ++k) {
        const int z = zt * VT_Z + k;
        if (z >= v.D) break;
        const long long l = ((long long)z * v.H + y) * v.W + x;
        const Cell c = make_cell(z, y, x, __ldg(ub + l), __ldg(ub + v.V + l), __ldg(ub + 2 * v.V + l), v);
        float dz, dy, dx;
        tri_grad(Ib, c, v, dz, dy, dx);
        const float g = __ldg(gb + l);
        ob[l] = g * dz;
        ob[l + v.V] = g * dy;
        ob[l + 2 * v.V] = g * dx;
    }
}

// point-wise loss of d = W - A (Sec. "Dissimilarity metrics"): l1 = 0 -> d^2
// with derivative 2 d; l1 = 1 -> |d| with the subgradient sign(d) (0 at 0)
__device__ __forceinline__ float pw_loss(float d, int l1) { return l1 ? fabsf(d) : d * d; }
__device__ __forceinline__ float pw_grad(float d, int l1)
{
    return l1 ? (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) : 2.f * d;
}

__global__ void __launch_bounds__(VT_THREADS)
mse_kernel(const float* __restrict__ J, const float* __restrict__ A, float* __restrict__ gJ,
           double* __restrict__ partials, Vol v, int nzt, float invV, int l1)
{
    __shared__ double sh[32];
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    const float* Jb = J + (size_t)b * v.V;
    float acc = 0.f;
    if (x < v.W && y < v.H) {
        for (int k = 0; k < VT_Z; ++k) {
            const int z = zt * VT_Z + k;
            if (z >= v.D) break;
            const long long l = ((long long)z * v.H + y) * v.W + x;
            const float d = __ldg(Jb + l) - __ldg(A + l);
            acc = fmaf(invV, pw_loss(d, l1), acc);
            if (gJ) gJ[(size_t)b * v.V + l] = invV * pw_grad(d, l1);
        }
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        partials[(size_t)b * gridDim.x * gridDim.y * nzt + block_index_in_subject(zt)] = s;
}

__global__ void __launch_bounds__(VT_THREADS)
reg_kernel(const float* __restrict__ u, float* __restrict__ gu, double* __restrict__ partials,
           Vol v, int nzt, RegW rw)
{
    __shared__ double sh[32];
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    const float* ub = u + (size_t)b * 3 * v.V;
    float acc = 0.f;
    if (x < v.W && y < v.H) {
        for (int k = 0; k < VT_Z; ++k) {
            const int z = zt * VT_Z + k;
            if (z >= v.D) break;
            const long long l = ((long long)z * v.H + y) * v.W + x;
            float g[3];
            acc += reg_at(ub, v, z, y, x, l, rw, g);
            if (gu) {
                float* gb = gu + (size_t)b * 3 * v.V;
                gb[l] = g[0];
                gb[l + v.V] = g[1];
                gb[l + 2 * v.V] = g[2];
            }
        }
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        partials[(size_t)b * gridDim.x * gridDim.y * nzt + block_index_in_subject(zt)] = s;
}

// Point-wise subject step, fused: W = S(I, x + u_T), L = mean l(W - A)
// (MSE or L1), gT = (l'(W - A)/V) dS(I)/dp + lambda dR/du_T; partials {L, R}
// per block.
template <class U>
__global__ void __launch_bounds__(VT_THREADS)
mse_warp_reg_kernel(const float* __restrict__ I, size_t I_bstride, const float* __restrict__ A,
                    U uT, float lambda, float* __restrict__ gT,
                    double* __restrict__ partials, Vol v, int nzt, float invV, RegW rw, int l1)
{
    __shared__ double sh[32];
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    const float* Ib = I + (size_t)b * I_bstride;
    const U ub = uT.subject(b);
    float* gb = gT + (size_t)b * 3 * v.V;
    float accL = 0.f, accR = 0.f;
    if (x < v.W && y < v.H) {
        for (int k = 0; k < VT_Z; ++k) {
            const int z = zt * VT_Z + k;
            if (z >= v.D) break;
            const int l = (z * v.H + y) * v.W + x;
            const float3 d3 = ub.own(l);
            const Cell c = make_cell_warp(z, y, x, d3.x, d3.y, d3.z, v);
            float dz, dy, dx;
            const float Wv = tri_grad(Ib, c, v, dz, dy, dx);
            const float d = Wv - __ldg(A + l);
            accL = fmaf(invV, pw_loss(d, l1), accL);
            const float gW = invV * pw_grad(d, l1);
            float g[3];
            accR += reg_at_field(ub, v, z, y, x, l, rw, g);
            gb[l] = fmaf(gW, dz, lambda * g[0]);
            gb[l + v.V] = fmaf(gW, dy, lambda * g[1]);
            gb[l + 2 * v.V] = fmaf(gW, dx, lambda * g[2]);
        }
    }
    const double sL = block_sum(accL, sh);
    const double sR = block_sum(accR, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const size_t j = (size_t)b * gridDim.x * gridDim.y * nzt + block_index_in_subject(zt);
        partials[2 * j] = sL;
        partials[2 * j + 1] = sR;
    }
}

__global__ void __launch_bounds__(VT_THREADS)
label_gather_kernel(const uint8_t* __restrict__ lab, const float* __restrict__ u,
                    uint8_t* __restrict__ out, Vol v, int nzt)
{
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    if (x >= v.W || y >= v.H) return;
    const float* ub = u + (size_t)b * 3 * v.V;
    for (int k = 0; k < VT_Z; ++k) {
        const int z = zt * VT_Z + k;
        if (z >= v.D) break;
        const long long l = ((long long)z * v.H + y) * v.W + x;
        // nearest voxel: r(x + u) = x + floor(u + 1/2) for integer x, clamped
        const int q[3] = {z, y, x};
        const int n[3] = {v.D, v.H, v.W};
        int r[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float ua = fminf(fmaxf(__ldg(ub + a * v.V + l), -1.0e6f), 1.0e6f);
            int ra = q[a] + (int)floorf(ua + 0.5f);
            r[a] = min(max(ra, 0), n[a] - 1);
        }
        out[(size_t)b * v.V + l] = lab[((long long)r[0] * v.H + r[1]) * v.W + r[2]];
    }
}

// det(I + grad u) at voxel (z, y, x): central differences inside, one-sided
// on the faces
__device__ __forceinline__ float jac_det_at(const float* __restrict__ ub, const Vol& v, int z, int y, int x)
{
    const int n[3] = {v.D, v.H, v.W};
    const long long st[3] = {(long long)v.H * v.W, (long long)v.W, 1};
    const int q[3] = {z, y, x};
    const long long l = ((long long)z * v.H + y) * v.W + x;
    float J[3][3];
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
        long long lo = l, hi = l;
        float h;
        if (q[bb] == 0) { hi = l + st[bb]; h = 1.f; }
        else if (q[bb] == n[bb] - 1) { lo = l - st[bb]; h = 1.f; }
        else { lo = l - st[bb]; hi = l + st[bb]; h = 2.f; }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            J[a][bb] = (a == bb ? 1.f : 0.f) + (__ldg(ub + a * v.V + hi) - __ldg(ub + a * v.V + lo)) / h;
    }
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

__global__ void __launch_bounds__(VT_THREADS)
jacobian_kernel(const float* __restrict__ u, float* __restrict__ det,
                unsigned long long* __restrict__ count, Vol v, int nzt)
{
    __shared__ unsigned int nneg;
    if (threadIdx.x == 0 && threadIdx.y == 0) nneg = 0;
    __syncthreads();
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    const float* ub = u + (size_t)b * 3 * v.V;
    unsigned int mine = 0;
    if (x < v.W && y < v.H) {
        for (int k = 0; k < VT_Z; ++k) {
            const int z = zt * VT_Z + k;
            if (z >= v.D) break;
            const float d = jac_det_at(ub, v, z, y, x);
            if (det) det[(size_t)b * v.V + ((long long)z * v.H + y) * v.W + x] = d;
            mine += (d <= 0.f);
        }
    }
    if (mine) atomicAdd(&nneg, mine);
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && count && nneg)
        atomicAdd(count + b, (unsigned long long)nneg);
}

// voxel-wise lower median over n rows: out[l] = sorted_i X[i][l] at (n - 1)/2.
// One thread per voxel; its n values sit in its own column of shared memory
// (no barrier: a thread reads only what it wrote); the value whose rank
// window [#less, #less-or-equal) holds (n - 1)/2 is selected, so the result
// is one of the inputs, exactly.
__global__ void median_kernel(const float* __restrict__ X, int n, long long V, float* __restrict__ out)
{
    extern __shared__ float col[];
    const int t = threadIdx.x, bd = blockDim.x;
    const long long l = blockIdx.x * (long long)bd + t;
    if (l >= V) return;
    for (int i = 0; i < n; ++i) col[i * bd + t] = __ldg(X + (size_t)i * V + l);
    const int k = (n - 1) / 2;
    float m = col[t];
    for (int i = 0; i < n; ++i) {
        const float xi = col[i * bd + t];
        int lt = 0, le = 0;
        for (int j = 0; j < n; ++j) {
            const float xj = col[j * bd + t];
            lt += xj < xi;
            le += xj <= xi;
        }
        if (lt <= k && k < le) {
            m = xi;
            break;
        }
    }
    out[l] = m;
}

// displacement of phi_b o phi_a: out(x) = a(x) + S(b, x + a(x))
__global__ void __launch_bounds__(VT_THREADS)
compose_kernel(const float* __restrict__ a, const float* __restrict__ bf, float* __restrict__ out, Vol v, int nzt)
{
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    if (x >= v.W || y >= v.H) return;
    const float* a0 = a + (size_t)b * 3 * v.V;
    const float* b0 = bf + (size_t)b * 3 * v.V;
    float* o0 = out + (size_t)b * 3 * v.V;
    for (int k = 0; k < VT_Z; ++k) {
        const int z = zt * VT_Z + k;
        if (z >= v.D) break;
        const long long l = ((long long)z * v.H + y) * v.W + x;
        const float uz = __ldg(a0 + l), uy = __ldg(a0 + v.V + l), ux = __ldg(a0 + 2 * v.V + l);
        const Cell c = make_cell(z, y, x, uz, uy, ux, v);
        o0[l] = uz + tri(b0, c, v);
        o0[l + v.V] = uy + tri(b0 + v.V, c, v);
        o0[l + 2 * v.V] = ux + tri(b0 + 2 * v.V, c, v);
    }
}

// per block: {voxels with det(I + grad u) <= 0, sum |r|, max |r|, min det}
__global__ void __launch_bounds__(VT_THREADS)
diffeo_stats_kernel(const float* __restrict__ u, const float* __restrict__ r, double* __restrict__ partials, Vol v,
                    int nzt)
{
    __shared__ double sh[32];
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    const float* ub = u + (size_t)b * 3 * v.V;
    const float* rb = r + (size_t)b * 3 * v.V;
    float neg = 0.f, sum = 0.f, mx = 0.f, mn = 3.0e38f;
    if (x < v.W && y < v.H) {
        for (int k = 0; k < VT_Z; ++k) {
            const int z = zt * VT_Z + k;
            if (z >= v.D) break;
            const long long l = ((long long)z * v.H + y) * v.W + x;
            const float d = jac_det_at(ub, v, z, y, x);
            const float e = sqrtf(rb[l] * rb[l] + rb[v.V + l] * rb[v.V + l] + rb[2 * v.V + l] * rb[2 * v.V + l]);
            neg += (d <= 0.f);
            sum += e;
            mx = fmaxf(mx, e);
            mn = fminf(mn, d);
        }
    }
    const int nb = gridDim.x * gridDim.y * nzt;
    const int blk = (blockIdx.z % nzt) * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x;
    double* out = partials + ((size_t)b * nb + blk) * 4;
    const double s0 = block_sum(neg, sh);
    const double s1 = block_sum(sum, sh);
    const double s2 = -block_min(-mx, sh);
    const double s3 = block_min(mn, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        out[0] = s0;
        out[1] = s1;
        out[2] = s2;
        out[3] = s3;
    }
}

// stats[b] = {negative fraction, mean |r|, max |r|, min det} (fixed order)
__global__ void diffeo_stats_finish_kernel(const double* __restrict__ partials, int nb, long long V,
                                           float* __restrict__ stats)
{
    if (threadIdx.x != 0) return;
    const int b = blockIdx.x;
    double neg = 0.0, sum = 0.0, mx = 0.0, mn = 3.0e38;
    for (int j = 0; j < nb; ++j) {
        const double* p = partials + ((size_t)b * nb + j) * 4;
        neg += p[0];
        sum += p[1];
        mx = fmax(mx, p[2]);
        mn = fmin(mn, p[3]);
    }
    stats[4 * b + 0] = (float)(neg / (double)V);
    stats[4 * b + 1] = (float)(sum / (double)V);
    stats[4 * b + 2] = (float)mx;
    stats[4 * b + 3] = (float)mn;
}

dim3 vgrid(int B, const Vol& v, int& nzt)
{
    nzt = div_up(v.D, VT_Z);
    return dim3(div_up(v.W, VT_X), div_up(v.H, VT_Y), nzt * B);
}

}  // namespace

int voxel_blocks(const Vol& v) { return div_up(v.W, VT_X) * div_up(v.H, VT_Y) * div_up(v.D, VT_Z); }

cudaError_t warp(const float* I, size_t I_bstride, const float* u, float* out, int B, const Vol& v,
                 cudaStream_t s)
{
    int nzt;
    const dim3 g = vgrid(B, v, nzt);
    warp_kernel<PlanarField><<<g, dim3(VT_X, VT_Y), 0, s>>>(I, I_bstride, PlanarField{u, v.V}, out, v, nzt);
    return cudaGetLastError();
}

cudaError_t warp_packed(const float* I, size_t I_bstride, const float4* u, float* out, int B, const Vol& v,
                        cudaStream_t s)
{
    if (reinterpret_cast<uintptr_t>(u) & 15) return cudaErrorMisalignedAddress;
    int nzt;
    const dim3 g = vgrid(B, v, nzt);
    warp_kernel<PackedField><<<g, dim3(VT_X, VT_Y), 0, s>>>(I, I_bstride, PackedField{u, v.V}, out, v, nzt);
    return cudaGetLastError();
}

cudaError_t warp_backward(const float* I, size_t I_bstride, const float* u, const float* gW,
                          float* gu, int B, const Vol& v, cudaStream_t s)
{
    int nzt;
    const dim3 g = vgrid(B, v, nzt);
    warp_backward_kernel<<<g, dim3(VT_X, VT_Y), 0, s>>>(I, I_bstride, u, gW, gu, v, nzt);
    return cudaGetLastError();
}

cudaError_t mse_partials(const float* J, const float* A, float* gJ, double* partials, int B,
                         const Vol& v, int l1, cudaStream_t s)
{
    int nzt;
    const dim3 g = vgrid(B, v, nzt);
    mse_kernel<<<g, dim3(VT_X, VT_Y), 0, s>>>(J, A, gJ, partials, v, nzt, (float)(1.0 / (double)v.V), l1);
    return cudaGetLastError();
}

cudaError_t reg_partials(const float* u, float* gu, double* partials, int B, const Vol& v,
                         cudaStream_t s)
{
    int nzt;
    const dim3 g = vgrid(B, v, nzt);
    reg_kernel<<<g, dim3(VT_X, VT_Y), 0, s>>>(u, gu, partials, v, nzt, reg_weights(v));
    return cudaGetLastError();
}

cudaError_t mse_warp_reg(const float* I, size_t I_bstride, const float* A, const float* uT,
                         float lambda, float* gT, double* partials, int B, const Vol& v,
                         int l1, cudaStream_t s, int uT_packed)
{
    int nzt;
    const dim3 g = vgrid(B, v, nzt);
    const float invV = (float)(1.0 / (double)v.V);
    if (uT_packed) {
        if (reinterpret_cast<uintptr_t>(uT) & 15) return cudaErrorMisalignedAddress;
        mse_warp_reg_kernel<PackedField><<<g, dim3(VT_X, VT_Y), 0, s>>>(
            I, I_bstride, A, PackedField{reinterpret_cast<const float4*>(uT), v.V}, lambda, gT, partials, v, nzt,
            invV, reg_weights(v), l1);
    } else {
        mse_warp_reg_kernel<PlanarField><<<g, dim3(VT_X, VT_Y), 0, s>>>(
            I, I_bstride, A, PlanarField{uT, v.V}, lambda, gT, partials, v, nzt, invV, reg_weights(v), l1);
    }
    return cudaGetLastError();
}

namespace {

// Per-subject label overlaps for the Dice score (Sec. "Evaluation
// metrics"): counts[b][l] = {|a = l|, |b = l|, |a = l and b = l|}; block
// histograms in shared memory, flushed with one atomic per label.
__global__ void __launch_bounds__(256)
label_overlap_kernel(const uint8_t* __restrict__ a, const uint8_t* __restrict__ bl, long long V, int nl,
                     unsigned long long* __restrict__ counts)
{
    __shared__ unsigned int h[3][256];
    for (int k = threadIdx.x; k < 3 * 256; k += 256) (&h[0][0])[k] = 0u;
    __syncthreads();
    const int b = blockIdx.y;
    const uint8_t* pa = a + (size_t)b * V;
    const uint8_t* pb = bl + (size_t)b * V;
    for (long long l = blockIdx.x * 256LL + threadIdx.x; l < V; l += (long long)gridDim.x * 256) {
        const int x = __ldg(pa + l), y = __ldg(pb + l);
        atomicAdd(&h[0][x], 1u);
        atomicAdd(&h[1][y], 1u);
        if (x == y) atomicAdd(&h[2][x], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * nl; k += 256) {
        const int c = k / nl, lab = k - c * nl;
        if (h[c][lab]) atomicAdd(counts + ((size_t)b * nl + lab) * 3 + c, (unsigned long long)h[c][lab]);
    }
}

}  // namespace

cudaError_t label_overlap(const uint8_t* a, const uint8_t* b, int B, long long V, int nl,
                          unsigned long long* counts, cudaStream_t s)
{
    const int gx = (int)std::max<long long>(1, std::min<long long>((V + 255) / 256, 152LL * 8 / std::max(B, 1) + 1));
    label_overlap_kernel<<<dim3(gx, B), 256, 0, s>>>(a, b, V, nl, counts);
    return cudaGetLastError();
}

cudaError_t label_gather(const uint8_t* labels, const float* u, uint8_t* out, int B, const Vol& v,
                         cudaStream_t s)
{
    int nzt;
    const dim3 g = vgrid(B, v, nzt);
    label_gather_kernel<<<g, dim3(VT_X, VT_Y), 0, s>>>(labels, u, out, v, nzt);
    return cudaGetLastError();
}

int median_threads(int n)
{
    int bd = 256;
    while (bd > 32 && (size_t)n * bd * sizeof(float) > 48 * 1024) bd /= 2;
    return (size_t)n * bd * sizeof(float) <= 200 * 1024 ? bd : 0;
}

cudaError_t median(const float* X, int n, long long V, float* out, cudaStream_t s)
{
    const int bd = median_threads(n);
    if (bd == 0) return cudaErrorInvalidValue;
    const size_t smem = (size_t)n * bd * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(median_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    median_kernel<<<(unsigned)((V + bd - 1) / bd), bd, smem, s>>>(X, n, V, out);
    return cudaGetLastError();
}

cudaError_t compose(const float* a, const float* b, float* out, int B, const Vol& v, cudaStream_t s)
{
    int nzt;
    const dim3 g = vgrid(B, v, nzt);
    compose_kernel<<<g, dim3(VT_X, VT_Y), 0, s>>>(a, b, out, v, nzt);
    return cudaGetLastError();
}

cudaError_t diffeo_stats(const float* u, const float* r, double* partials, float* stats, int B, const Vol& v,
                         cudaStream_t s)
{
    int nzt;
    const dim3 g = vgrid(B, v, nzt);
    diffeo_stats_kernel<<<g, dim3(VT_X, VT_Y), 0, s>>>(u, r, partials, v, nzt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diffeo_stats_finish_kernel<<<B, 32, 0, s>>>(partials, voxel_blocks(v), v.V, stats);
    return cudaGetLastError();
}

cudaError_t jacobian_det(const float* u, float* det, unsigned long long* count, int B,
                         const Vol& v, cudaStream_t s)
{
    int nzt;
    const dim3 g = vgrid(B, v, nzt);
    jacobian_kernel<<<g, dim3(VT_X, VT_Y), 0, s>>>(u, det, count, v, nzt);
    return cudaGetLastError();
}

}  // namespace darc_impl
