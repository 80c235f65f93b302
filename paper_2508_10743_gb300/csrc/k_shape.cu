// k_shape.cu -- PCA shape synthesis in velocity space (arXiv 2508.10743,
// Sec. "Shape synthesis"): the cohort's mean velocity, the Gram matrix of
// the centred velocities (whose eigenpairs give the covariance's principal
// components without forming the 3V x 3V covariance), new velocities as
// weighted sums of the subjects' fields, and the forward map applied to
// mesh vertices.
#include "kernels.h"

#include <algorithm>

namespace darc_impl {
namespace {

constexpr int GT = 16;          // Gram tile edge (rows i x rows j per block)
constexpr int GK = 64;          // elements of a row staged per round

// mean[l] = 1/n sum_i v[i][l] (fixed order)
__global__ void field_mean_kernel(const float* __restrict__ v, int n, long long M, float* __restrict__ mean)
{
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < M; l += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += __ldg(v + (size_t)i * M + l);
        mean[l] = (float)(s / n);
    }
}

// Partial Gram sums over one split of the elements: block (ti, tj, split)
// computes G[i][j] = sum_l (v_i - mean)(v_j - mean) for its 16 x 16 tile;
// each 64-element round is summed in float and added to a double.
__global__ void __launch_bounds__(GT * GT)
gram_kernel(const float* __restrict__ v, const float* __restrict__ mean, int n, long long M, long long chunk,
            double* __restrict__ partial)
{
    __shared__ float si[GT][GK + 1], sj[GT][GK + 1];
    const int tx = threadIdx.x % GT, ty = threadIdx.x / GT;
    const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
    const long long l0 = (long long)blockIdx.z * chunk, l1 = min(M, l0 + chunk);
    double acc = 0.0;
    for (long long lb = l0; lb < l1; lb += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += GT * GT) {
            const int r = e / GK, k = e % GK;
            const long long l = lb + k;
            const float m = l < l1 ? __ldg(mean + l) : 0.f;
            si[r][k] = (l < l1 && i0 + r < n) ? __ldg(v + (size_t)(i0 + r) * M + l) - m : 0.f;
            sj[r][k] = (l < l1 && j0 + r < n) ? __ldg(v + (size_t)(j0 + r) * M + l) - m : 0.f;
        }
        __syncthreads();
        float s = 0.f;
#pragma unroll 16
        for (int k = 0; k < GK; ++k) s = fmaf(si[ty][k], sj[tx][k], s);
        acc += s;
        __syncthreads();
    }
    const int i = i0 + ty, j = j0 + tx;
    if (i < n && j < n) partial[((size_t)blockIdx.z * n + i) * n + j] = acc;
}

__global__ void gram_reduce_kernel(const double* __restrict__ partial, int splits, int n, double* __restrict__ G)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    double s = 0.0;
    for (int q = 0; q < splits; ++q) s += partial[(size_t)q * n * n + e];
    G[e] = s;
}

// out[k][l] = mean[l] + sum_i coef[k][i] (v_i[l] - mean[l]), k < m <= 8
__global__ void combine_kernel(const float* __restrict__ v, const float* __restrict__ mean, int n, long long M,
                               const float* __restrict__ coef, int m, float* __restrict__ out)
{
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < M; l += (long long)gridDim.x * blockDim.x) {
        const float mu = __ldg(mean + l);
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int i = 0; i < n; ++i) {
            const float d = __ldg(v + (size_t)i * M + l) - mu;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < m) acc[k] = fmaf(__ldg(coef + k * n + i), d, acc[k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < m) out[(size_t)k * M + l] = mu + acc[k];
    }
}

// out[p] = pts[p] + S(u, pts[p]): points in (z, y, x) voxel coordinates
__global__ void warp_points_kernel(const float* __restrict__ u, Vol v, const float* __restrict__ pts, long long P,
                                   float* __restrict__ out)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float pz = pts[3 * p], py = pts[3 * p + 1], px = pts[3 * p + 2];
        // a cell from integer base 0 and the point as the displacement
        const Cell c = make_cell(0, 0, 0, pz, py, px, v);
        out[3 * p] = pz + tri(u, c, v);
        out[3 * p + 1] = py + tri(u + v.V, c, v);
        out[3 * p + 2] = px + tri(u + 2 * v.V, c, v);
    }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 8)); }

}  // namespace

cudaError_t field_mean(const float* v, int n, long long M, float* mean, cudaStream_t s)
{
    field_mean_kernel<<<grid_for(M), 256, 0, s>>>(v, n, M, mean);
    return cudaGetLastError();
}

int gram_splits(int n)
{
    const int t = (n + GT - 1) / GT;
    return std::max(1, std::min(608 / (t * t), 256));
}

cudaError_t gram(const float* v, const float* mean, int n, long long M, double* partial, double* G, cudaStream_t s)
{
    const int t = (n + GT - 1) / GT, splits = gram_splits(n);
    const long long chunk = ((M + splits - 1) / splits + GK - 1) / GK * GK;
    gram_kernel<<<dim3(t, t, splits), GT * GT, 0, s>>>(v, mean, n, M, chunk, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gram_reduce_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(partial, splits, n, G);
    return cudaGetLastError();
}

cudaError_t combine_fields(const float* v, const float* mean, int n, long long M, const float* coef, int m,
                           float* out, cudaStream_t s)
{
    combine_kernel<<<grid_for(M), 256, 0, s>>>(v, mean, n, M, coef, m, out);
    return cudaGetLastError();
}

cudaError_t warp_points(const float* u, const Vol& v, const float* pts, long long P, float* out, cudaStream_t s)
{
    warp_points_kernel<<<grid_for(P), 256, 0, s>>>(u, v, pts, P, out);
    return cudaGetLastError();
}

}  // namespace darc_impl
