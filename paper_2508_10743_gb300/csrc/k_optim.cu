// k_optim.cu -- loss reductions, Adam, centrality activation, atlas means
// (sm_103a).
//
// Adam (arXiv 2508.10743, Sec. "Experiments": Adam, lr 1e-2, for the
// velocities and the atlas; reading: PyTorch's defaults, bias corrected).
// Centrality activation (Eq. 3, line n+1): hat v_i = v_i - 1/n sum_j v_j.
// MSE atlas (Sec. "Dissimilarity metrics"): A = 1/n sum_i I_i o Exp(hat v_i).
// Every reduction sums in a fixed order (deterministic).
#include "kernels.h"

#include <algorithm>

namespace darc_impl {
namespace {

constexpr int RT = 256;

__global__ void __launch_bounds__(RT)
reduce_partials_kernel(const double* __restrict__ p, int nblk, int nval, double scale,
                       float* __restrict__ out, int out_stride)
{
    __shared__ double sh[32];
    const int b = blockIdx.x;
    for (int k = 0; k < nval; ++k) {
        double s = 0.0;
        for (int j = threadIdx.x; j < nblk; j += RT) s += p[((size_t)b * nblk + j) * nval + k];
        s = warp_sum(s);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < RT / 32; ++q) t += sh[q];
            out[(size_t)b * out_stride + k] = (float)(t * scale);
        }
        __syncthreads();
    }
}

__device__ double fixed_sum(const double* __restrict__ p, int nblk, int stride, int b, double* sh)
{
    double s = 0.0;
    for (int j = threadIdx.x; j < nblk; j += RT) s += p[((size_t)b * nblk + j) * stride];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < RT / 32; ++q) t += sh[q];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(RT)
finish_step_kernel(const double* __restrict__ pL, int nblkL, int strideL,
                   const double* __restrict__ pR, int nblkR, int strideR, float* __restrict__ loss,
                   int* __restrict__ flags, int* __restrict__ k, float2* __restrict__ bias,
                   int* __restrict__ nonfinite_total, float lr, float beta1, float beta2)
{
    __shared__ double sh[32];
    const int b = blockIdx.x;
    const double L = fixed_sum(pL, nblkL, strideL, b, sh);
    const double R = fixed_sum(pR, nblkR, strideR, b, sh);
    if (threadIdx.x == 0) {
        loss[2 * b] = (float)L;
        loss[2 * b + 1] = (float)R;
        const bool ok = isfinite(L) && isfinite(R);
        flags[b] = ok ? 0 : 1;
        if (ok) {
            const int kk = k[b] + 1;
            k[b] = kk;
            const double c1 = 1.0 - pow((double)beta1, (double)kk);
            const double c2 = 1.0 - pow((double)beta2, (double)kk);
            bias[b] = make_float2((float)((double)lr / c1), (float)(1.0 / sqrt(c2)));
        } else {
            atomicAdd(nonfinite_total, 1);
        }
    }
}

// grid (blocks over N/4, B); theta/m/s/g float4 when N % 4 == 0
__global__ void __launch_bounds__(RT)
adam_fields_kernel(float* __restrict__ th, float* __restrict__ m, float* __restrict__ s,
                   const float* __restrict__ g, float g_scale, const float2* __restrict__ bias,
                   const int* __restrict__ flags, float b1, float b2, float eps, long long N)
{
    const int b = blockIdx.y;
    if (flags && flags[b]) return;
    const float2 bf = bias[b];
    const size_t off = (size_t)b * N;
    if ((N & 3) == 0) {
        float4* th4 = reinterpret_cast<float4*>(th + off);
        float4* m4 = reinterpret_cast<float4*>(m + off);
        float4* s4 = reinterpret_cast<float4*>(s + off);
        const float4* g4 = reinterpret_cast<const float4*>(g + off);
        for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N / 4;
             e += (long long)gridDim.x * RT) {
            float4 t = th4[e], mm = m4[e], ss = s4[e];
            const float4 gg = __ldg(g4 + e);
            adam1(t.x, mm.x, ss.x, gg.x * g_scale, b1, b2, bf.x, bf.y, eps);
            adam1(t.y, mm.y, ss.y, gg.y * g_scale, b1, b2, bf.x, bf.y, eps);
            adam1(t.z, mm.z, ss.z, gg.z * g_scale, b1, b2, bf.x, bf.y, eps);
            adam1(t.w, mm.w, ss.w, gg.w * g_scale, b1, b2, bf.x, bf.y, eps);
            th4[e] = t;
            m4[e] = mm;
            s4[e] = ss;
        }
    } else {
        for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N;
             e += (long long)gridDim.x * RT) {
            float t = th[off + e], mm = m[off + e], ss = s[off + e];
            adam1(t, mm, ss, __ldg(g + off + e) * g_scale, b1, b2, bf.x, bf.y, eps);
            th[off + e] = t;
            m[off + e] = mm;
            s[off + e] = ss;
        }
    }
}

// The same step for B velocity fields [3][V] whose gradient is interleaved,
// one float4 (z, y, x, 0) per voxel; grid (blocks over V/4, B), four voxels
// a thread when V % 4 == 0.
__global__ void __launch_bounds__(RT)
adam_fields_g4_kernel(float* __restrict__ th, float* __restrict__ m, float* __restrict__ s,
                      const float4* __restrict__ g, const float2* __restrict__ bias,
                      const int* __restrict__ flags, float b1, float b2, float eps, long long V)
{
    const int b = blockIdx.y;
    if (flags && flags[b]) return;
    const float2 bf = bias[b];
    const size_t off = (size_t)b * 3 * V;
    const float4* gb = g + (size_t)b * V;
    if ((V & 3) == 0) {
        const long long V4 = V / 4;
        for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < V4; e += (long long)gridDim.x * RT) {
            float gv[3][4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 q = __ldg(gb + 4 * e + k);
                gv[0][k] = q.x;
                gv[1][k] = q.y;
                gv[2][k] = q.z;
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float4* th4 = reinterpret_cast<float4*>(th + off + (size_t)ch * V);
                float4* m4 = reinterpret_cast<float4*>(m + off + (size_t)ch * V);
                float4* s4 = reinterpret_cast<float4*>(s + off + (size_t)ch * V);
                float4 t = th4[e], mm = m4[e], ss = s4[e];
                adam1(t.x, mm.x, ss.x, gv[ch][0], b1, b2, bf.x, bf.y, eps);
                adam1(t.y, mm.y, ss.y, gv[ch][1], b1, b2, bf.x, bf.y, eps);
                adam1(t.z, mm.z, ss.z, gv[ch][2], b1, b2, bf.x, bf.y, eps);
                adam1(t.w, mm.w, ss.w, gv[ch][3], b1, b2, bf.x, bf.y, eps);
                th4[e] = t;
                m4[e] = mm;
                s4[e] = ss;
            }
        }
    } else {
        for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < V; e += (long long)gridDim.x * RT) {
            const float4 q = __ldg(gb + e);
            const float gq[3] = {q.x, q.y, q.z};
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const size_t i = off + (size_t)ch * V + e;
                float t = th[i], mm = m[i], ss = s[i];
                adam1(t, mm, ss, gq[ch], b1, b2, bf.x, bf.y, eps);
                th[i] = t;
                m[i] = mm;
                s[i] = ss;
            }
        }
    }
}

__global__ void __launch_bounds__(RT)
adam_flat_kernel(float* __restrict__ th, float* __restrict__ m, float* __restrict__ s,
                 const float* __restrict__ g, size_t N, float lr_c1, float isc2, float b1, float b2,
                 float eps)
{
    for (size_t e = blockIdx.x * (size_t)RT + threadIdx.x; e < N; e += (size_t)gridDim.x * RT) {
        float t = th[e], mm = m[e], ss = s[e];
        adam1(t, mm, ss, __ldg(g + e), b1, b2, lr_c1, isc2, eps);
        th[e] = t;
        m[e] = mm;
        s[e] = ss;
    }
}

// one thread per voxel: mean field over the n subjects (fixed order),
// subtract it, record |mean| before and after (block partials)
__global__ void __launch_bounds__(RT)
centrality_kernel(float* __restrict__ v, int n, long long V, double* __restrict__ partials)
{
    __shared__ double sh[32];
    float before = 0.f, after = 0.f;
    const long long l = blockIdx.x * (long long)RT + threadIdx.x;
    if (l < V) {
        const size_t st = (size_t)3 * V;
        float mean[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double sum = 0.0;
            for (int i = 0; i < n; ++i) sum += (double)v[i * st + a * V + l];
            mean[a] = (float)(sum / n);
        }
        before = sqrtf(mean[0] * mean[0] + mean[1] * mean[1] + mean[2] * mean[2]);
        float rest[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double sum = 0.0;
            for (int i = 0; i < n; ++i) {
                const float nv = v[i * st + a * V + l] - mean[a];
                v[i * st + a * V + l] = nv;
                sum += (double)nv;
            }
            rest[a] = (float)(sum / n);
        }
        after = sqrtf(rest[0] * rest[0] + rest[1] * rest[1] + rest[2] * rest[2]);
    }
    const double sb = block_sum(before, sh);
    const double sa = block_sum(after, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sb;
        partials[2 * blockIdx.x + 1] = sa;
    }
}

__global__ void __launch_bounds__(RT)
metrics_kernel(const double* __restrict__ partials, int nblk, double invV, double* __restrict__ out)
{
    __shared__ double sh[32];
    for (int k = 0; k < 2; ++k) {
        double s = 0.0;
        for (int j = threadIdx.x; j < nblk; j += RT) s += partials[2 * j + k];
        s = warp_sum(s);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < RT / 32; ++q) t += sh[q];
            out[k] = t * invV;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(VT_THREADS)
warp_accumulate_kernel(const float* __restrict__ I, const int* __restrict__ subj,
                       const float* __restrict__ u, double* __restrict__ acc, int B, Vol v, int nzt)
{
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z;
    if (x >= v.W || y >= v.H) return;
    for (int k = 0; k < VT_Z; ++k) {
        const int z = zt * VT_Z + k;
        if (z >= v.D) break;
        const long long l = ((long long)z * v.H + y) * v.W + x;
        double s = acc[l];
        for (int b = 0; b < B; ++b) {
            const float* ub = u + (size_t)b * 3 * v.V;
            const Cell c = make_cell(z, y, x, __ldg(ub + l), __ldg(ub + v.V + l), __ldg(ub + 2 * v.V + l), v);
            s += (double)tri(I + (size_t)subj[b] * v.V, c, v);
        }
        acc[l] = s;
    }
}

__global__ void __launch_bounds__(RT)
image_mean_kernel(const float* __restrict__ I, int n, double* __restrict__ acc, long long V)
{
    for (long long l = blockIdx.x * (long long)RT + threadIdx.x; l < V; l += (long long)gridDim.x * RT) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += (double)__ldg(I + (size_t)i * V + l);
        acc[l] = s;
    }
}

__global__ void __launch_bounds__(RT)
finalize_mean_kernel(const double* __restrict__ acc, double inv_n, float* __restrict__ A, long long V)
{
    for (long long l = blockIdx.x * (long long)RT + threadIdx.x; l < V; l += (long long)gridDim.x * RT)
        A[l] = (float)(acc[l] * inv_n);
}

__global__ void __launch_bounds__(RT)
atlas_adam_kernel(float* __restrict__ A, float* __restrict__ m, float* __restrict__ s,
                  const float* __restrict__ gsh, const float* __restrict__ g, int B, float scale,
                  float lr_c1, float isc2, float b1, float b2, float eps, long long V)
{
    for (long long l = blockIdx.x * (long long)RT + threadIdx.x; l < V; l += (long long)gridDim.x * RT) {
        float gs = gsh ? __ldg(gsh + l) : 0.f;
        for (int b = 0; b < B; ++b) gs += __ldg(g + (size_t)b * V + l);
        float a = A[l], mm = m[l], ss = s[l];
        adam1(a, mm, ss, gs * scale, b1, b2, lr_c1, isc2, eps);
        A[l] = a;
        m[l] = mm;
        s[l] = ss;
    }
}

__global__ void __launch_bounds__(RT)
field_sum_kernel(const float* __restrict__ v, int B, float* __restrict__ out, long long N)
{
    for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT) {
        double s = 0.0;
        for (int b = 0; b < B; ++b) s += (double)__ldg(v + (size_t)b * N + e);
        out[e] = (float)s;
    }
}

__global__ void __launch_bounds__(RT)
field_subtract_kernel(float* __restrict__ v, int B, const float* __restrict__ sum, float scale, long long N)
{
    for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < N; e += (long long)gridDim.x * RT) {
        const float mu = __ldg(sum + e) * scale;
        for (int b = 0; b < B; ++b) v[(size_t)b * N + e] -= mu;
    }
}

__global__ void __launch_bounds__(RT)
combine_grad_kernel(const float* __restrict__ gsh, const float* __restrict__ g, int B, float scale,
                    float* __restrict__ out, long long V)
{
    for (long long l = blockIdx.x * (long long)RT + threadIdx.x; l < V; l += (long long)gridDim.x * RT) {
        float s = gsh ? __ldg(gsh + l) : 0.f;
        for (int b = 0; b < B; ++b) s += __ldg(g + (size_t)b * V + l);
        out[l] = s * scale;
    }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + RT - 1) / RT, 152LL * 32)); }

}  // namespace

cudaError_t field_sum(const float* v, int B, float* out, const Vol& vol, cudaStream_t s)
{
    field_sum_kernel<<<grid_for(3 * vol.V), RT, 0, s>>>(v, B, out, 3 * vol.V);
    return cudaGetLastError();
}

cudaError_t field_subtract(float* v, int B, const float* sum, float scale, const Vol& vol, cudaStream_t s)
{
    field_subtract_kernel<<<grid_for(3 * vol.V), RT, 0, s>>>(v, B, sum, scale, 3 * vol.V);
    return cudaGetLastError();
}

cudaError_t combine_grad(const float* gshared, const float* gsubj, int B, float scale, float* out,
                         const Vol& v, cudaStream_t s)
{
    combine_grad_kernel<<<grid_for(v.V), RT, 0, s>>>(gshared, gsubj, B, scale, out, v.V);
    return cudaGetLastError();
}

cudaError_t reduce_partials(const double* partials, int nblk, int nval, double scale, float* out,
                            int out_stride, int B, cudaStream_t s)
{
    reduce_partials_kernel<<<B, RT, 0, s>>>(partials, nblk, nval, scale, out, out_stride);
    return cudaGetLastError();
}

cudaError_t finish_step(const double* pL, int nblkL, int strideL, const double* pR, int nblkR,
                        int strideR, float* loss, int* flags, int* k, float2* bias,
                        int* nonfinite_total, float lr, float beta1, float beta2, int B,
                        cudaStream_t s)
{
    finish_step_kernel<<<B, RT, 0, s>>>(pL, nblkL, strideL, pR, nblkR, strideR, loss, flags, k, bias,
                                        nonfinite_total, lr, beta1, beta2);
    return cudaGetLastError();
}

cudaError_t adam_fields(float* theta, float* m, float* s_, const float* g, float g_scale,
                        const float2* bias, const int* flags, float beta1, float beta2, float eps,
                        int B, long long N, cudaStream_t st)
{
    const long long work = (N % 4 == 0) ? N / 4 : N;
    const int gx = (int)std::max<long long>(1, std::min<long long>((work + RT - 1) / RT, 152LL * 8));
    adam_fields_kernel<<<dim3(gx, B), RT, 0, st>>>(theta, m, s_, g, g_scale, bias, flags, beta1,
                                                   beta2, eps, N);
    return cudaGetLastError();
}

cudaError_t adam_fields_g4(float* theta, float* m, float* s_, const float4* g, const float2* bias, const int* flags,
                           float beta1, float beta2, float eps, int B, long long V, cudaStream_t st)
{
    const long long work = (V % 4 == 0) ? V / 4 : V;
    const int gx = (int)std::max<long long>(1, std::min<long long>((work + RT - 1) / RT, 152LL * 8));
    adam_fields_g4_kernel<<<dim3(gx, B), RT, 0, st>>>(theta, m, s_, g, bias, flags, beta1, beta2, eps, V);
    return cudaGetLastError();
}

cudaError_t adam_flat(float* theta, float* m, float* s_, const float* g, size_t N, float lr_c1,
                      float inv_sqrt_c2, float beta1, float beta2, float eps, cudaStream_t st)
{
    adam_flat_kernel<<<grid_for((long long)N), RT, 0, st>>>(theta, m, s_, g, N, lr_c1, inv_sqrt_c2,
                                                            beta1, beta2, eps);
    return cudaGetLastError();
}

int centrality_blocks(const Vol& v) { return div_up(v.V, RT); }

cudaError_t centrality(float* v_all, int n, const Vol& v, double* partials, double* metrics,
                       cudaStream_t s)
{
    const int nb = centrality_blocks(v);
    centrality_kernel<<<nb, RT, 0, s>>>(v_all, n, v.V, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !metrics) return e;
    metrics_kernel<<<1, RT, 0, s>>>(partials, nb, 1.0 / (double)v.V, metrics);
    return cudaGetLastError();
}

cudaError_t warp_accumulate(const float* I, const int* subj, const float* u, double* acc, int B,
                            const Vol& v, cudaStream_t s)
{
    const int nzt = div_up(v.D, VT_Z);
    warp_accumulate_kernel<<<dim3(div_up(v.W, VT_X), div_up(v.H, VT_Y), nzt), dim3(VT_X, VT_Y), 0, s>>>(
        I, subj, u, acc, B, v, nzt);
    return cudaGetLastError();
}

cudaError_t image_mean_accumulate(const float* I, int n, double* acc, const Vol& v, cudaStream_t s)
{
    image_mean_kernel<<<grid_for(v.V), RT, 0, s>>>(I, n, acc, v.V);
    return cudaGetLastError();
}

cudaError_t finalize_mean(const double* acc, double inv_n, float* A, const Vol& v, cudaStream_t s)
{
    finalize_mean_kernel<<<grid_for(v.V), RT, 0, s>>>(acc, inv_n, A, v.V);
    return cudaGetLastError();
}

cudaError_t atlas_adam(float* A, float* m, float* s_, const float* gshared, const float* gsubj,
                       int B, float scale, float lr_c1, float inv_sqrt_c2, float beta1, float beta2,
                       float eps, const Vol& v, cudaStream_t st)
{
    atlas_adam_kernel<<<grid_for(v.V), RT, 0, st>>>(A, m, s_, gshared, gsubj, B, scale, lr_c1, inv_sqrt_c2,
                                                    beta1, beta2, eps, v.V);
    return cudaGetLastError();
}

}  // namespace darc_impl
