// common.cuh -- device helpers shared by the libdarc kernels (sm_103a).
//
// Layout: a volume has D x H x W voxels (z, y, x), x fastest; an image is
// float [V]; a field is planar float [3][V] (channel a = component along
// axis a, voxel units); batches are subject-major.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace darc_impl {

struct Vol {
    int D, H, W;
    long long V;
};

inline Vol make_vol(int D, int H, int W) { return Vol{D, H, W, (long long)D * H * W}; }

// Geometry of the per-voxel kernels: a block of 32 x 8 threads covers a
// 32 (x) x 8 (y) x TZ (z) tile, each thread walking TZ planes.
constexpr int VT_X = 32, VT_Y = 8, VT_Z = 4, VT_THREADS = VT_X * VT_Y;

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// Cell of one axis of the sample point x + u for trilinear sampling with
// border padding: the coordinate is clamped to [0, n - 1]; the cell is
// i = min(floor(p), n - 2) and t = p - i.  The position is formed as the
// integer x plus floor(u) and the fraction u - floor(u), which is exact in
// float32, so large volume coordinates cost no precision.  `clamped` marks
// a coordinate strictly outside [0, n - 1] (derivative 0 along that axis).
__device__ __forceinline__ void axis_cell(int x, float u, int n, int& i, float& t, bool& clamped)
{
    u = fminf(fmaxf(u, -1.0e6f), 1.0e6f);   // keeps NaN/Inf inside int range (they end clamped)
    const float fl = floorf(u);
    const int ii = x + (int)fl;
    const float tt = u - fl;
    if (ii < 0) {
        i = 0; t = 0.f; clamped = true;
    } else if (ii >= n - 1) {
        clamped = (ii > n - 1) || (tt > 0.f);
        i = n - 2; t = 1.f;
    } else {
        i = ii; t = tt; clamped = false;
    }
}

struct Cell {
    int base;              // linear index of corner (iz, iy, ix) (V < 2^31)
    float tz, ty, tx;
    bool cz, cy, cx;       // clamped axes
    int iz, iy, ix;
};

__device__ __forceinline__ Cell make_cell(int z, int y, int x, float uz, float uy, float ux, const Vol& v)
{
    Cell c;
    axis_cell(z, uz, v.D, c.iz, c.tz, c.cz);
    axis_cell(y, uy, v.H, c.iy, c.ty, c.cy);
    axis_cell(x, ux, v.W, c.ix, c.tx, c.cx);
    c.base = (c.iz * v.H + c.iy) * v.W + c.ix;
    return c;
}

// make_cell in its unclamped form when every lane running it together has
// an unclamped cell on every axis (|u| < 1e6 and 0 <= x + floor(u) <= n - 2:
// make_cell's middle case, the same floats), else make_cell itself.
__device__ __forceinline__ Cell make_cell_warp(int z, int y, int x, float uz, float uy, float ux, const Vol& v)
{
    const float fz = floorf(uz), fy = floorf(uy), fx = floorf(ux);
    const bool finite = fabsf(uz) < 1.0e6f && fabsf(uy) < 1.0e6f && fabsf(ux) < 1.0e6f;
    const int iz = z + (finite ? (int)fz : 0), iy = y + (finite ? (int)fy : 0), ix = x + (finite ? (int)fx : 0);
    const bool inner = finite && (unsigned)iz <= (unsigned)(v.D - 2) && (unsigned)iy <= (unsigned)(v.H - 2) &&
                       (unsigned)ix <= (unsigned)(v.W - 2);
    if (__all_sync(__activemask(), inner)) {
        Cell c;
        c.iz = iz;
        c.iy = iy;
        c.ix = ix;
        c.tz = uz - fz;
        c.ty = uy - fy;
        c.tx = ux - fx;
        c.cz = c.cy = c.cx = false;
        c.base = (iz * v.H + iy) * v.W + ix;
        return c;
    }
    return make_cell(z, y, x, uz, uy, ux, v);
}

// Trilinear value at the cell from its 8 corner values (corner order
// (dz, dy, dx) = 000, 001, 010, ...).
__device__ __forceinline__ float tri_corners(const Cell& c, float f000, float f001, float f010, float f011,
                                             float f100, float f101, float f110, float f111)
{
    const float a00 = fmaf(c.tx, f001 - f000, f000);
    const float a01 = fmaf(c.tx, f011 - f010, f010);
    const float a10 = fmaf(c.tx, f101 - f100, f100);
    const float a11 = fmaf(c.tx, f111 - f110, f110);
    const float b0 = fmaf(c.ty, a01 - a00, a00);
    const float b1 = fmaf(c.ty, a11 - a10, a10);
    return fmaf(c.tz, b1 - b0, b0);
}

// The same value and dS/dp (0 along clamped axes) from the 8 corner values.
__device__ __forceinline__ float tri_grad_corners(const Cell& c, float f000, float f001, float f010, float f011,
                                                  float f100, float f101, float f110, float f111,
                                                  float& gz, float& gy, float& gx)
{
    const float d00 = f001 - f000, d01 = f011 - f010, d10 = f101 - f100, d11 = f111 - f110;
    const float a00 = fmaf(c.tx, d00, f000);
    const float a01 = fmaf(c.tx, d01, f010);
    const float a10 = fmaf(c.tx, d10, f100);
    const float a11 = fmaf(c.tx, d11, f110);
    const float b0 = fmaf(c.ty, a01 - a00, a00);
    const float b1 = fmaf(c.ty, a11 - a10, a10);
    gz = c.cz ? 0.f : (b1 - b0);
    const float e0 = a01 - a00, e1 = a11 - a10;
    gy = c.cy ? 0.f : fmaf(c.tz, e1 - e0, e0);
    const float h0 = fmaf(c.ty, d01 - d00, d00), h1 = fmaf(c.ty, d11 - d10, d10);
    gx = c.cx ? 0.f : fmaf(c.tz, h1 - h0, h0);
    return fmaf(c.tz, b1 - b0, b0);
}

// S(f, p): trilinear value at the cell.
__device__ __forceinline__ float tri(const float* __restrict__ f, const Cell& c, const Vol& v)
{
    const int sy = v.W, sz = v.H * v.W;
    const float* p = f + c.base;
    return tri_corners(c, __ldg(p), __ldg(p + 1), __ldg(p + sy), __ldg(p + sy + 1), __ldg(p + sz),
                       __ldg(p + sz + 1), __ldg(p + sz + sy), __ldg(p + sz + sy + 1));
}

// S(f, p) and dS/dp (0 along clamped axes).
__device__ __forceinline__ float tri_grad(const float* __restrict__ f, const Cell& c, const Vol& v,
                                          float& gz, float& gy, float& gx)
{
    const int sy = v.W, sz = v.H * v.W;
    const float* p = f + c.base;
    return tri_grad_corners(c, __ldg(p), __ldg(p + 1), __ldg(p + sy), __ldg(p + sy + 1), __ldg(p + sz),
                            __ldg(p + sz + 1), __ldg(p + sz + sy), __ldg(p + sz + sy + 1), gz, gy, gx);
}

// A displacement field in one of two layouts: planar [3][V] (channel a =
// axis a) or packed, one float4 (z, y, x, 0) per voxel.  own() reads the
// three channels at a voxel; sample() the trilinear values at a cell;
// grad() also the 3 x 3 derivatives d[channel][axis].  Both layouts give
// the same floats.
struct PlanarField {
    const float* p;
    long long V;
    __device__ PlanarField subject(int b) const { return PlanarField{p + (size_t)b * 3 * V, V}; }
    __device__ float3 own(int l) const { return make_float3(__ldg(p + l), __ldg(p + V + l), __ldg(p + 2 * V + l)); }
    __device__ float3 sample(const Cell& c, const Vol& v) const
    {
        return make_float3(tri(p, c, v), tri(p + V, c, v), tri(p + 2 * V, c, v));
    }
    __device__ void grad(const Cell& c, const Vol& v, float d[3][3]) const
    {
        tri_grad(p, c, v, d[0][0], d[0][1], d[0][2]);
        tri_grad(p + V, c, v, d[1][0], d[1][1], d[1][2]);
        tri_grad(p + 2 * V, c, v, d[2][0], d[2][1], d[2][2]);
    }
};

struct PackedField {
    const float4* p;
    long long V;
    __device__ PackedField subject(int b) const { return PackedField{p + (size_t)b * V, V}; }
    __device__ float3 own(int l) const
    {
        const float4 q = __ldg(p + l);
        return make_float3(q.x, q.y, q.z);
    }
    __device__ void corners(const Cell& c, const Vol& v, float4 f[8]) const
    {
        const int sy = v.W, sz = v.H * v.W;
        const float4* q = p + c.base;
        f[0] = __ldg(q);
        f[1] = __ldg(q + 1);
        f[2] = __ldg(q + sy);
        f[3] = __ldg(q + sy + 1);
        f[4] = __ldg(q + sz);
        f[5] = __ldg(q + sz + 1);
        f[6] = __ldg(q + sz + sy);
        f[7] = __ldg(q + sz + sy + 1);
    }
    __device__ float3 sample(const Cell& c, const Vol& v) const
    {
        float4 f[8];
        corners(c, v, f);
        return make_float3(tri_corners(c, f[0].x, f[1].x, f[2].x, f[3].x, f[4].x, f[5].x, f[6].x, f[7].x),
                           tri_corners(c, f[0].y, f[1].y, f[2].y, f[3].y, f[4].y, f[5].y, f[6].y, f[7].y),
                           tri_corners(c, f[0].z, f[1].z, f[2].z, f[3].z, f[4].z, f[5].z, f[6].z, f[7].z));
    }
    __device__ void grad(const Cell& c, const Vol& v, float d[3][3]) const
    {
        float4 f[8];
        corners(c, v, f);
        tri_grad_corners(c, f[0].x, f[1].x, f[2].x, f[3].x, f[4].x, f[5].x, f[6].x, f[7].x, d[0][0], d[0][1], d[0][2]);
        tri_grad_corners(c, f[0].y, f[1].y, f[2].y, f[3].y, f[4].y, f[5].y, f[6].y, f[7].y, d[1][0], d[1][1], d[1][2]);
        tri_grad_corners(c, f[0].z, f[1].z, f[2].z, f[3].z, f[4].z, f[5].z, f[6].z, f[7].z, d[2][0], d[2][1], d[2][2]);
    }
};

// J^T g for a packed field: with J = dS(u, p)/dp at the cell (3 x 3,
// channel by axis) and g a 3-vector, (J^T g)_a = d/dp_a of the trilinear
// interpolation of the corner dot products g . u(corner) (S is linear in the
// corner values), zero along clamped axes.
__device__ __forceinline__ float3 packed_jac_t(const PackedField& f, const Cell& c, const Vol& v, float3 g)
{
    float4 q[8];
    f.corners(c, v, q);
    float d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] = fmaf(g.x, q[k].x, fmaf(g.y, q[k].y, g.z * q[k].z));
    float jz, jy, jx;
    tri_grad_corners(c, d[0], d[1], d[2], d[3], d[4], d[5], d[6], d[7], jz, jy, jx);
    return make_float3(jz, jy, jx);
}

// J^T g of a planar field: the 3 x 3 derivatives, then the product
__device__ __forceinline__ float3 planar_jac_t(const PlanarField& f, const Cell& c, const Vol& v, float3 g)
{
    float d[3][3];
    f.grad(c, v, d);
    return make_float3(g.x * d[0][0] + g.y * d[1][0] + g.z * d[2][0], g.x * d[0][1] + g.y * d[1][1] + g.z * d[2][1],
                       g.x * d[0][2] + g.y * d[1][2] + g.z * d[2][2]);
}

__device__ __forceinline__ float3 field_jac_t(const PackedField& f, const Cell& c, const Vol& v, float3 g)
{
    return packed_jac_t(f, c, v, g);
}

__device__ __forceinline__ float3 field_jac_t(const PlanarField& f, const Cell& c, const Vol& v, float3 g)
{
    return planar_jac_t(f, c, v, g);
}

// The 8 trilinear weights in corner order (dz, dy, dx) = 000, 001, 010, ...
__device__ __forceinline__ void tri_weights(const Cell& c, float w[8])
{
    const float z0 = 1.f - c.tz, y0 = 1.f - c.ty, x0 = 1.f - c.tx;
    const float zy00 = z0 * y0, zy01 = z0 * c.ty, zy10 = c.tz * y0, zy11 = c.tz * c.ty;
    w[0] = zy00 * x0; w[1] = zy00 * c.tx;
    w[2] = zy01 * x0; w[3] = zy01 * c.tx;
    w[4] = zy10 * x0; w[5] = zy10 * c.tx;
    w[6] = zy11 * x0; w[7] = zy11 * c.tx;
}

// Diffusion regulariser weights per axis: 1 / (3 P_a), P_a = V (n_a - 1) /
// n_a voxel pairs along axis a.
struct RegW {
    float z, y, x;
};

// Value share of voxel x (pairs counted at their lower voxel) and gradient
// dR/du_c(x) of the diffusion regulariser, for a field in either layout.
template <class F>
__device__ __forceinline__ float reg_at_field(const F& f, const Vol& v, int z, int y, int x, int l, const RegW& rw,
                                              float g[3])
{
    const int st[3] = {v.H * v.W, v.W, 1};
    const int q[3] = {z, y, x};
    const int n[3] = {v.D, v.H, v.W};
    const float ca[3] = {rw.z, rw.y, rw.x};
    const float3 c3 = f.own(l);
    const float cur[3] = {c3.x, c3.y, c3.z};
    float val = 0.f;
    g[0] = g[1] = g[2] = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const bool up = q[a] + 1 < n[a];
        const bool dn = q[a] > 0;
        const float3 u3 = up ? f.own(l + st[a]) : c3;
        const float3 d3 = dn ? f.own(l - st[a]) : c3;
        const float uv[3] = {u3.x, u3.y, u3.z}, dv[3] = {d3.x, d3.y, d3.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float dup = up ? uv[c] - cur[c] : 0.f;
            const float ddn = dn ? cur[c] - dv[c] : 0.f;
            val = fmaf(ca[a] * dup, dup, val);
            g[c] = fmaf(2.f * ca[a], ddn - dup, g[c]);
        }
    }
    return val;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block sum of a float per thread (blockDim.x*y*z a multiple of 32, <= 1024)
// returned in double on thread 0; fixed order, so deterministic.
__device__ __forceinline__ double block_sum(float x, double* sh /* >= 32 doubles */)
{
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    double d = warp_sum((double)x);
    if ((tid & 31) == 0) sh[tid >> 5] = d;
    __syncthreads();
    double tot = 0.0;
    if (tid == 0)
        for (int k = 0; k < (nthr >> 5); ++k) tot += sh[k];
    __syncthreads();
    return tot;
}

// One Adam step of a parameter th with moments m, s and gradient g
// (Kingma & Ba 2015): lr_c1 = lr / (1 - beta1^k), isc2 = 1 / sqrt(1 - beta2^k).
__device__ __forceinline__ void adam1(float& th, float& m, float& s, float g, float b1, float b2,
                                      float lr_c1, float isc2, float eps)
{
    m = fmaf(b1, m, (1.f - b1) * g);
    s = fmaf(b2, s, (1.f - b2) * g * g);
    th -= lr_c1 * m / fmaf(sqrtf(s), isc2, eps);
}

// minimum over the block (valid in thread 0)
__device__ __forceinline__ double block_min(float x, double* sh /* >= 32 doubles */)
{
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    float m = x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) sh[tid >> 5] = m;
    __syncthreads();
    double r = 3.0e38;
    if (tid == 0)
        for (int k = 0; k < (nthr >> 5); ++k) r = fmin(r, sh[k]);
    __syncthreads();
    return r;
}

}  // namespace darc_impl
