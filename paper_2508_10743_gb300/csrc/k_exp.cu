// k_exp.cu -- scaling and squaring and its adjoint (sm_103a).
//
// Exp(v) by scaling and squaring (arXiv 2508.10743, Sec. "Diffeomorphisms":
// phi = Exp(v), seven squarings): u_0 = sign 2^-T v and
// u_{t+1}(x) = u_t(x) + S(u_t, x + u_t(x)).
//
// Forward: one thread per voxel, the 8 corners of each channel gathered
// through the read-only cache (neighbouring threads share cells, so the
// gathers hit L1).  Adjoint: the transpose of the interpolation is a
// scatter.  A block stages its sources' contributions in a shared-memory
// window that covers every cell its 32x8x4 tile of sources can reach
// (computed per block from the data), adds them there with shared atomics,
// and flushes the window to global memory with one atomic add per non-zero
// cell and channel.  A block whose window exceeds the budget scatters
// straight to global memory.
#include "kernels.h"

#include <climits>

namespace darc_impl {
namespace {

__global__ void __launch_bounds__(VT_THREADS)
exp_square_kernel(const float* __restrict__ src, float scale, float* __restrict__ dst, Vol v,
                  int nzt)
{
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt;
    const int b = blockIdx.z / nzt;
    if (x >= v.W || y >= v.H) return;
    const float* s0 = src + (size_t)b * 3 * v.V;
    const float* s1 = s0 + v.V;
    const float* s2 = s1 + v.V;
    float* d0 = dst + (size_t)b * 3 * v.V;
#pragma unroll 1
    for (int k = 0; k < VT_Z; ++k) {
        const int z = zt * VT_Z + k;
        if (z >= v.D) break;
        const long long l = ((long long)z * v.H + y) * v.W + x;
        const float uz = scale * __ldg(s0 + l), uy = scale * __ldg(s1 + l), ux = scale * __ldg(s2 + l);
        const Cell c = make_cell(z, y, x, uz, uy, ux, v);
        d0[l] = fmaf(scale, tri(s0, c, v), uz);
        d0[l + v.V] = fmaf(scale, tri(s1, c, v), uy);
        d0[l + 2 * v.V] = fmaf(scale, tri(s2, c, v), ux);
    }
}

// shared-memory window budget of the adjoint: cells x 3 channels x 4 B
constexpr int WIN_CELLS = 4096;
constexpr size_t WIN_BYTES = (size_t)WIN_CELLS * 3 * sizeof(float);

__global__ void __launch_bounds__(VT_THREADS)
exp_square_adjoint_kernel(const float* __restrict__ src, float scale, const float* __restrict__ gin,
                          float* __restrict__ gout, float out_scale, Vol v, int nzt)
{
    extern __shared__ float win[];           // [3][cells]
    __shared__ int bnd[6];                   // lo z,y,x ; hi z,y,x
    const int tid = threadIdx.y * VT_X + threadIdx.x;
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt;
    const int b = blockIdx.z / nzt;
    const bool xy_ok = (x < v.W) && (y < v.H);
    const float* s0 = src + (size_t)b * 3 * v.V;
    const float* s1 = s0 + v.V;
    const float* s2 = s1 + v.V;
    const float* g0 = gin + (size_t)b * 3 * v.V;
    float* o0 = gout + (size_t)b * 3 * v.V;

    if (tid < 3) bnd[tid] = INT_MAX;
    else if (tid < 6) bnd[tid] = INT_MIN;
    __syncthreads();

    // 1. window bounds: every corner touched and every source voxel itself
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    if (xy_ok) {
        for (int k = 0; k < VT_Z; ++k) {
            const int z = zt * VT_Z + k;
            if (z >= v.D) break;
            const long long l = ((long long)z * v.H + y) * v.W + x;
            const Cell c = make_cell(z, y, x, scale * __ldg(s0 + l), scale * __ldg(s1 + l),
                                     scale * __ldg(s2 + l), v);
            lo[0] = min(lo[0], min(z, c.iz)); hi[0] = max(hi[0], max(z, c.iz + 1));
            lo[1] = min(lo[1], min(y, c.iy)); hi[1] = max(hi[1], max(y, c.iy + 1));
            lo[2] = min(lo[2], min(x, c.ix)); hi[2] = max(hi[2], max(x, c.ix + 1));
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    if ((tid & 31) == 0) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bnd[a], lo[a]);
            atomicMax(&bnd[3 + a], hi[a]);
        }
    }
    __syncthreads();
    if (bnd[0] == INT_MAX) return;           // no voxel of this tile is inside the volume
    const int wz0 = bnd[0], wy0 = bnd[1], wx0 = bnd[2];
    const int ey = bnd[4] - wy0 + 1, ex = bnd[5] - wx0 + 1;
    const long long cells_ll = (long long)(bnd[3] - wz0 + 1) * ey * ex;
    const bool staged = cells_ll <= WIN_CELLS;
    const int cells = staged ? (int)cells_ll : 0;
    if (staged) {
        for (int e = tid; e < 3 * cells; e += VT_THREADS) win[e] = 0.f;
        __syncthreads();
    }

    // 2. contributions of each source voxel
    if (xy_ok) {
        for (int k = 0; k < VT_Z; ++k) {
            const int z = zt * VT_Z + k;
            if (z >= v.D) break;
            const long long l = ((long long)z * v.H + y) * v.W + x;
            const Cell c = make_cell(z, y, x, scale * __ldg(s0 + l), scale * __ldg(s1 + l),
                                     scale * __ldg(s2 + l), v);
            const float gz = __ldg(g0 + l), gy = __ldg(g0 + v.V + l), gx = __ldg(g0 + 2 * v.V + l);
            float dz0, dy0, dx0, dz1, dy1, dx1, dz2, dy2, dx2;
            tri_grad(s0, c, v, dz0, dy0, dx0);
            tri_grad(s1, c, v, dz1, dy1, dx1);
            tri_grad(s2, c, v, dz2, dy2, dx2);
            // identity + Jacobian term at the source voxel itself (scale: du_t = scale d src)
            const float lz = gz + scale * (gz * dz0 + gy * dz1 + gx * dz2);
            const float ly = gy + scale * (gz * dy0 + gy * dy1 + gx * dy2);
            const float lx = gx + scale * (gz * dx0 + gy * dx1 + gx * dx2);
            float w[8];
            tri_weights(c, w);
            const float gs[3] = {gz * out_scale, gy * out_scale, gx * out_scale};
            if (staged) {
                const int e0 = ((z - wz0) * ey + (y - wy0)) * ex + (x - wx0);
                atomicAdd(&win[e0], lz * out_scale);
                atomicAdd(&win[cells + e0], ly * out_scale);
                atomicAdd(&win[2 * cells + e0], lx * out_scale);
                const int cb = ((c.iz - wz0) * ey + (c.iy - wy0)) * ex + (c.ix - wx0);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int e = cb + ((q >> 2) & 1) * ey * ex + ((q >> 1) & 1) * ex + (q & 1);
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) atomicAdd(&win[ch * cells + e], w[q] * gs[ch]);
                }
            } else {
                atomicAdd(o0 + l, lz * out_scale);
                atomicAdd(o0 + v.V + l, ly * out_scale);
                atomicAdd(o0 + 2 * v.V + l, lx * out_scale);
                const long long sy = v.W, sz = (long long)v.H * v.W;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const long long e = c.base + ((q >> 2) & 1) * sz + ((q >> 1) & 1) * sy + (q & 1);
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) atomicAdd(o0 + ch * v.V + e, w[q] * gs[ch]);
                }
            }
        }
    }

    // 3. flush the window
    if (staged) {
        __syncthreads();
        for (int e = tid; e < cells; e += VT_THREADS) {
            const int wz = e / (ey * ex);
            const int rem = e - wz * ey * ex;
            const int wy = rem / ex;
            const int wx = rem - wy * ex;
            const long long l = ((long long)(wz0 + wz) * v.H + (wy0 + wy)) * v.W + (wx0 + wx);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float val = win[ch * cells + e];
                if (val != 0.f) atomicAdd(o0 + ch * v.V + l, val);
            }
        }
    }
}

dim3 voxel_grid(int B, const Vol& v, int& nzt)
{
    nzt = div_up(v.D, VT_Z);
    return dim3(div_up(v.W, VT_X), div_up(v.H, VT_Y), nzt * B);
}

}  // namespace

cudaError_t exp_square(const float* src, float scale, float* dst, int B, const Vol& v,
                       cudaStream_t s)
{
    int nzt;
    const dim3 grid = voxel_grid(B, v, nzt);
    exp_square_kernel<<<grid, dim3(VT_X, VT_Y), 0, s>>>(src, scale, dst, v, nzt);
    return cudaGetLastError();
}

cudaError_t exp_square_adjoint(const float* src, float scale, const float* gin, float* gout,
                               float out_scale, int B, const Vol& v, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(exp_square_adjoint_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)WIN_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int nzt;
    const dim3 grid = voxel_grid(B, v, nzt);
    exp_square_adjoint_kernel<<<grid, dim3(VT_X, VT_Y), WIN_BYTES, s>>>(src, scale, gin, gout,
                                                                        out_scale, v, nzt);
    return cudaGetLastError();
}

}  // namespace darc_impl
