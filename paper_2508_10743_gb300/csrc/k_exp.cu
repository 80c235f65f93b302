// k_exp.cu -- scaling and squaring and its adjoint (sm_103a).
//
// Exp(v) by scaling and squaring (arXiv 2508.10743, Sec. "Diffeomorphisms":
// phi = Exp(v), seven squarings): u_0 = sign 2^-T v and
// u_{t+1}(x) = u_t(x) + S(u_t, x + u_t(x)).
//
// Forward: one thread per voxel, the 8 corners of each channel gathered
// through the read-only cache (neighbouring threads share cells, so the
// gathers hit L1).  Adjoint: the transpose of the interpolation is a
// scatter, done with float atomics that the L2 resolves (measured faster on
// GB300 than staging the block's contributions in shared memory, which cost
// occupancy and barriers).  A warp is one x-row of 32 sources; neighbouring
// lanes usually share an x-corner, so a lane hands its upper x-corner
// contribution to the next lane when the cells coincide, and sends the two
// x-corners of a (z, y) pair as one 8-byte atomic when they are aligned.
// Along z, each thread walks consecutive planes and merges the upper-z
// corners of one source with the lower-z corners of the next in registers.
//
// Two field layouts: planar [3][V] (v, the public Exp forward, the
// allocation-free adjoint) and packed, one float4 (z, y, x, 0) a voxel (the
// subject update's squaring fields: a corner's three channels are one
// 16-byte gather; the adjoint chains' gradients: one 16-byte atomic).  Both read through the same trilinear
// corner arithmetic, so they give the same floats.
#include "kernels.h"

#include <algorithm>
#include <climits>

namespace darc_impl {
namespace {

#define DARC_PRAGMA(x) _Pragma(#x)
#define DARC_UNROLL(n) DARC_PRAGMA(unroll n)

// Squaring tiles: 32 x 8 x SQ_Z voxels per block, each thread walking SQ_Z
// planes, SQ_UNROLL of them with their gathers in flight together.
#ifndef DARC_SQ_Z
#define DARC_SQ_Z 4
#endif
#ifndef DARC_SQ_UNROLL
#define DARC_SQ_UNROLL 1
#endif
constexpr int SQ_Z = DARC_SQ_Z;

// Staged squaring of a packed field (u_t, t >= 1): a block of 32 x 8 threads
// walks SQS_Z planes of a 32 x 8 column tile, keeping planes z - 1, z and
// z + 1 of u_t with a one-voxel halo in shared memory (a ring of four: the
// next plane is copied in while the current one is sampled; one block
// barrier a plane).  A voxel whose cell lies in the staged box (every |u|
// below one voxel, or a clamped cell at the border) reads its 8 corners
// there, others through the read-only cache; the corner values and the
// interpolation are the same either way, so the result equals
// exp_square_kernel's bit for bit.  Off by default (DARC_SQ_STAGED=1 turns it
// on): the squaring is bound by its DRAM bytes, which staging does not
// change, and the halo copies and the barrier a plane cost more than the
// L1 hits they replace (brain sweep: 148 against 122 ms of squarings).
#ifndef DARC_SQ_STAGED
#define DARC_SQ_STAGED 0
#endif
#ifndef DARC_SQS_Z
#define DARC_SQS_Z 16
#endif
constexpr int SQS_Z = DARC_SQS_Z;
constexpr int SQS_TX = VT_X + 2, SQS_TY = VT_Y + 2;

__device__ __forceinline__ void sqs_copy16(float4* dst_smem, const float4* src, bool in)
{
    // 16-byte asynchronous copy into shared memory; zeros where !in
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 :: "r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem))), "l"(src), "r"(in ? 16 : 0)
                 : "memory");
}

__global__ void __launch_bounds__(VT_THREADS)
exp_square_staged_kernel(PackedField src_all, float scale, float4* __restrict__ dst, Vol v, int nzt,
                         float4* __restrict__ zero)
{
    __shared__ __align__(16) float4 tile[4][SQS_TY][SQS_TX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * VT_X + tx;
    const int x0 = blockIdx.x * VT_X, y0 = blockIdx.y * VT_Y;
    const int x = x0 + tx, y = y0 + ty;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    const int z0 = zt * SQS_Z;
    const PackedField f = src_all.subject(b);
    float4* d0 = dst + (size_t)b * v.V;
    const int plane = v.H * v.W;
    // plane zz into its ring slot by asynchronous copies (one commit group)
    auto stage = [&](int zz) {
        float4 (*t)[SQS_TX] = tile[(zz - z0 + 1) & 3];
        for (int e = tid; e < SQS_TY * SQS_TX; e += VT_THREADS) {
            const int ry = e / SQS_TX, rx = e - ry * SQS_TX;
            const int gy = y0 - 1 + ry, gx = x0 - 1 + rx;
            const bool in = zz >= 0 && zz < v.D && gy >= 0 && gy < v.H && gx >= 0 && gx < v.W;
            sqs_copy16(&t[ry][rx], in ? f.p + (size_t)zz * plane + gy * v.W + gx : f.p, in);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // planes z0 - 1 .. z0 + 2 (one commit group each); then each plane's
    // group is committed two planes before it is sampled
    stage(z0 - 1);
    stage(z0);
    stage(z0 + 1);
    stage(z0 + 2);
    const bool in_xy = x < v.W && y < v.H;
    for (int k = 0; k < SQS_Z; ++k) {
        const int z = z0 + k;
        if (z >= v.D) break;                         // uniform over the block
        // planes z - 1 .. z + 1 landed (the last group, plane z + 2, may be in flight)
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        if (in_xy) {
            const float4 o = tile[(k + 1) & 3][ty + 1][tx + 1];
            const float uz = scale * o.x, uy = scale * o.y, ux = scale * o.z;
            const Cell c = make_cell(z, y, x, uz, uy, ux, v);
            float4 q[8];
            if (c.iz >= z - 1 && c.iz <= z && c.iy >= y0 - 1 && c.iy <= y0 + VT_Y - 1 && c.ix >= x0 - 1 &&
                c.ix <= x0 + VT_X - 1) {
                const int sz = (c.iz - z0 + 1) & 3, ry = c.iy - y0 + 1, rx = c.ix - x0 + 1;
                const int sz1 = (sz + 1) & 3;
                q[0] = tile[sz][ry][rx];
                q[1] = tile[sz][ry][rx + 1];
                q[2] = tile[sz][ry + 1][rx];
                q[3] = tile[sz][ry + 1][rx + 1];
                q[4] = tile[sz1][ry][rx];
                q[5] = tile[sz1][ry][rx + 1];
                q[6] = tile[sz1][ry + 1][rx];
                q[7] = tile[sz1][ry + 1][rx + 1];
            } else {
                f.corners(c, v, q);
            }
            const float sx = tri_corners(c, q[0].x, q[1].x, q[2].x, q[3].x, q[4].x, q[5].x, q[6].x, q[7].x);
            const float sy = tri_corners(c, q[0].y, q[1].y, q[2].y, q[3].y, q[4].y, q[5].y, q[6].y, q[7].y);
            const float sz_ = tri_corners(c, q[0].z, q[1].z, q[2].z, q[3].z, q[4].z, q[5].z, q[6].z, q[7].z);
            const int l = z * plane + y * v.W + x;
            d0[l] = make_float4(fmaf(scale, sx, uz), fmaf(scale, sy, uy), fmaf(scale, sz_, ux), 0.f);
            if (zero) zero[(size_t)b * v.V + l] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // every thread is done with plane z - 1: its slot takes plane z + 3
        __syncthreads();
        stage(z + 3);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Src: PlanarField or PackedField; PACKED_OUT: u_{t+1} written packed
// (float4 a voxel) instead of planar.  zero (packed only, may be null): a
// packed buffer of the same shape cleared on the way.
template <class Src, bool PACKED_OUT>
__global__ void __launch_bounds__(VT_THREADS)
exp_square_kernel(Src src_all, float scale, float* __restrict__ dst, Vol v, int nzt,
                  float4* __restrict__ zero = nullptr)
{
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt;
    const int b = blockIdx.z / nzt;
    if (x >= v.W || y >= v.H) return;
    const Src f = src_all.subject(b);
    float* d0 = dst + (size_t)b * (PACKED_OUT ? 4 : 3) * v.V;
    DARC_UNROLL(DARC_SQ_UNROLL)
    for (int k = 0; k < SQ_Z; ++k) {
        const int z = zt * SQ_Z + k;
        if (z >= v.D) break;
        const int l = (z * v.H + y) * v.W + x;
        const float3 o = f.own(l);
        const float uz = scale * o.x, uy = scale * o.y, ux = scale * o.z;
        const Cell c = make_cell(z, y, x, uz, uy, ux, v);
        const float3 sm = f.sample(c, v);
        const float rz = fmaf(scale, sm.x, uz), ry = fmaf(scale, sm.y, uy), rx = fmaf(scale, sm.z, ux);
        if (PACKED_OUT) {
            reinterpret_cast<float4*>(d0)[l] = make_float4(rz, ry, rx, 0.f);
            if (zero) zero[(size_t)b * v.V + l] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            d0[l] = rz;
            d0[l + v.V] = ry;
            d0[l + 2 * v.V] = rx;
        }
    }
}

// Adjoint tiles: 32 x 8 x ADJ_Z sources per block (each thread walks ADJ_Z
// planes).  PAIR: lanes hand coinciding x-corners to their neighbour;
// VEC2: a lane's two x-corners go out as one 8-byte atomic when aligned;
// CARRY: a thread keeps its upper-z corners in registers and adds them to
// the lower-z corners of its next plane when the two cells coincide (the
// usual case for a smooth field), so most corners are sent once, not twice.
#ifndef DARC_ADJ_Z
#define DARC_ADJ_Z 16
#endif
#ifndef DARC_ADJ_PAIR
#define DARC_ADJ_PAIR 1
#endif
#ifndef DARC_ADJ_VEC2
#define DARC_ADJ_VEC2 1
#endif
#ifndef DARC_ADJ_CARRY
#define DARC_ADJ_CARRY 1
#endif
constexpr int ADJ_Z = DARC_ADJ_Z;
// planes per thread of the far-source scatter: its blocks are the gather's
// 32 x 8 x 8 mark tiles
constexpr int FAR_Z = 8;
// resident blocks per SM asked of the interleaved adjoint (a register cap)
#ifndef DARC_ADJ_MINB
#define DARC_ADJ_MINB 4
#endif
// rows of the interleaved adjoint's blocks (32 x ADJ_Y threads; the
// resident-block cap scales so that a multiprocessor keeps the same threads)
#ifndef DARC_ADJ_Y
#define DARC_ADJ_Y 8
#endif
constexpr int ADJ_Y = DARC_ADJ_Y;
// 1: the interleaved adjoint loads the next plane's displacement and
// gradient while it works on the current one
#ifndef DARC_ADJ_PREFETCH
#define DARC_ADJ_PREFETCH 1
#endif
constexpr unsigned FULL_MASK = 0xffffffffu;

// The two x-corners (a, a + 1) of one (z, y) corner pair, three channels.
// Every lane of the warp calls it (shuffles); inactive lanes pass act = false.
__device__ __forceinline__ void emit_xpair(float* const o[3], int a, bool act, const float lo[3],
                                           const float hi[3], int lane, int vec2)
{
    bool absorb = false, given = false;
    if (DARC_ADJ_PAIR) {
        const int pa = __shfl_up_sync(FULL_MASK, act ? a : -4, 1);
        absorb = act && lane > 0 && pa >= 0 && pa + 1 == a;
        given = __shfl_down_sync(FULL_MASK, absorb, 1) && lane < 31;
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float lo_v = lo[ch];
        if (DARC_ADJ_PAIR) {
            const float ph = __shfl_up_sync(FULL_MASK, hi[ch], 1);
            if (absorb) lo_v += ph;
        }
        if (!act) continue;
        if (given) {
            atomicAdd(o[ch] + a, lo_v);
        } else if (DARC_ADJ_VEC2 && vec2 && (a & 1) == 0) {
            atomicAdd(reinterpret_cast<float2*>(o[ch] + a), make_float2(lo_v, hi[ch]));
        } else {
            atomicAdd(o[ch] + a, lo_v);
            atomicAdd(o[ch] + a + 1, hi[ch]);
        }
    }
}

// Same without the lane exchange (divergent callers).
__device__ __forceinline__ void emit_plain(float* const o[3], int a, const float lo[3], const float hi[3],
                                           int vec2)
{
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        if (DARC_ADJ_VEC2 && vec2 && (a & 1) == 0) {
            atomicAdd(reinterpret_cast<float2*>(o[ch] + a), make_float2(lo[ch], hi[ch]));
        } else {
            atomicAdd(o[ch] + a, lo[ch]);
            atomicAdd(o[ch] + a + 1, hi[ch]);
        }
    }
}

__global__ void __launch_bounds__(VT_THREADS)
exp_square_adjoint_kernel(const float* __restrict__ src, float scale, const float* __restrict__ gin,
                          float* __restrict__ gout, float out_scale, Vol v, int nzt, int vec2)
{
    const int lane = threadIdx.x;
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt;
    const int b = blockIdx.z / nzt;
    const bool xy_ok = (x < v.W) && (y < v.H);
    const float* s0 = src + (size_t)b * 3 * v.V;
    const float* s1 = s0 + v.V;
    const float* s2 = s1 + v.V;
    const float* g0 = gin + (size_t)b * 3 * v.V;
    const float* g1 = g0 + v.V;
    const float* g2 = g1 + v.V;
    float* o[3];
    o[0] = gout + (size_t)b * 3 * v.V;
    o[1] = o[0] + v.V;
    o[2] = o[1] + v.V;
    const int plane = v.H * v.W;
    float cl[2][3], cu[2][3];        // carried upper-z pairs: [dy][channel] lower / upper x-corner
    int ca = -1;                     // base index of the carried pairs (-1: none)
    for (int k = 0; k < ADJ_Z; ++k) {
        const int z = zt * ADJ_Z + k;
        const bool active = xy_ok && z < v.D;
        if (!DARC_ADJ_PAIR && !DARC_ADJ_CARRY && !active) break;
        float w[8], gs[3] = {0.f, 0.f, 0.f};
        int cb = -4;
        if (active) {
            const int l = z * plane + y * v.W + x;
            const Cell c = make_cell(z, y, x, scale * __ldg(s0 + l), scale * __ldg(s1 + l),
                                     scale * __ldg(s2 + l), v);
            const float gz = __ldg(g0 + l), gy = __ldg(g1 + l), gx = __ldg(g2 + l);
            float dz0, dy0, dx0, dz1, dy1, dx1, dz2, dy2, dx2;
            tri_grad(s0, c, v, dz0, dy0, dx0);
            tri_grad(s1, c, v, dz1, dy1, dx1);
            tri_grad(s2, c, v, dz2, dy2, dx2);
            // identity + Jacobian term at the source voxel itself (scale: du_t = scale d src)
            atomicAdd(o[0] + l, (gz + scale * (gz * dz0 + gy * dz1 + gx * dz2)) * out_scale);
            atomicAdd(o[1] + l, (gy + scale * (gz * dy0 + gy * dy1 + gx * dy2)) * out_scale);
            atomicAdd(o[2] + l, (gx + scale * (gz * dx0 + gy * dx1 + gx * dx2)) * out_scale);
            tri_weights(c, w);
            gs[0] = gz * out_scale;
            gs[1] = gy * out_scale;
            gs[2] = gx * out_scale;
            cb = c.base;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) w[q] = 0.f;
        }
        // transpose of the interpolation: the 8 corners as 4 (dz, dy) pairs of x-corners
        if (DARC_ADJ_CARRY) {
            const bool merge = active && ca == cb;
            if (ca >= 0 && !merge) {                 // the carried corners are not this cell's: send them
                emit_plain(o, ca, cl[0], cu[0], vec2);
                emit_plain(o, ca + v.W, cl[1], cu[1], vec2);
            }
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                float lo[3], hi[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    lo[ch] = w[2 * dy] * gs[ch] + (merge ? cl[dy][ch] : 0.f);
                    hi[ch] = w[2 * dy + 1] * gs[ch] + (merge ? cu[dy][ch] : 0.f);
                }
                emit_xpair(o, cb + dy * v.W, active, lo, hi, lane, vec2);
            }
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    cl[dy][ch] = w[4 + 2 * dy] * gs[ch];
                    cu[dy][ch] = w[5 + 2 * dy] * gs[ch];
                }
            ca = active ? cb + plane : -1;
        } else {
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                float lo[3], hi[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    lo[ch] = w[q] * gs[ch];
                    hi[ch] = w[q + 1] * gs[ch];
                }
                emit_xpair(o, cb + ((q >> 2) & 1) * plane + ((q >> 1) & 1) * v.W, active, lo, hi, lane, vec2);
            }
        }
    }
    if (DARC_ADJ_CARRY) {
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) emit_xpair(o, ca + dy * v.W, ca >= 0, cl[dy], cu[dy], lane, vec2);
    }
}

// Interleaved gradient fields: one float4 (z, y, x, 0) per voxel, so that a
// corner's three channels leave as one 16-byte atomic.  The lane exchange
// and the z carry work as above on whole corners.
__device__ __forceinline__ void emit4_xpair(float4* o, int a, bool act, float4 lo, const float4& hi, int lane)
{
    const int pa = __shfl_up_sync(FULL_MASK, act ? a : -4, 1);
    const bool absorb = act && lane > 0 && pa >= 0 && pa + 1 == a;
    const bool given = __shfl_down_sync(FULL_MASK, absorb, 1) && lane < 31;
    const float hz = __shfl_up_sync(FULL_MASK, hi.x, 1);
    const float hy = __shfl_up_sync(FULL_MASK, hi.y, 1);
    const float hx = __shfl_up_sync(FULL_MASK, hi.z, 1);
    if (absorb) {
        lo.x += hz;
        lo.y += hy;
        lo.z += hx;
    }
    if (!act) return;
    atomicAdd(o + a, lo);
    if (!given) atomicAdd(o + a + 1, hi);
}

// Far-source scatter after the gather adjoint (k_exp_gather.cu): a block
// runs only if the gather marked its tile (the mark is cleared here), and
// only sources with |u_a| >= 1 on some axis (or not finite) scatter.
__device__ __forceinline__ bool far_tile(int* flags)
{
    __shared__ int mark;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const size_t bid = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        mark = flags[bid];
        if (mark) flags[bid] = 0;
    }
    __syncthreads();
    return mark != 0;
}

__device__ __forceinline__ bool near_source(float uz, float uy, float ux)
{
    return fabsf(uz) < 1.f && fabsf(uy) < 1.f && fabsf(ux) < 1.f;
}

// IN4: the incoming gradient is interleaved too (else planar [3][V]); the
// outgoing one is always interleaved [V] float4 per field.  FAR: only the
// transpose terms of far sources, in marked tiles (flags).
template <bool IN4, class Src, bool FAR = false>
__global__ void __launch_bounds__(FAR ? VT_THREADS : VT_X * ADJ_Y,
                                  FAR ? DARC_ADJ_MINB : DARC_ADJ_MINB * VT_Y / ADJ_Y)
exp_square_adjoint4_kernel(Src src_all, float scale, const float* __restrict__ gin,
                           float4* __restrict__ gout, float out_scale, Vol v, int nzt, int* flags = nullptr)
{
    if (FAR && !far_tile(flags)) return;
    constexpr int ZT = FAR ? FAR_Z : ADJ_Z;   // planes per thread
    constexpr int TY = FAR ? VT_Y : ADJ_Y;    // rows per block
    const int lane = threadIdx.x;
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int zt = blockIdx.z % nzt;
    const int b = blockIdx.z / nzt;
    const bool xy_ok = (x < v.W) && (y < v.H);
    const Src f = src_all.subject(b);
    const float* g0 = gin + (size_t)b * (IN4 ? 4 : 3) * v.V;
    float4* o = gout + (size_t)b * v.V;
    const int plane = v.H * v.W;
    float4 cl[2], cu[2];             // carried upper-z pairs: [dy] lower / upper x-corner
    int ca = -1;                     // base index of the carried pairs (-1: none)
    constexpr bool PF = DARC_ADJ_PREFETCH && !FAR;
    float3 u_nx = make_float3(0.f, 0.f, 0.f), g_nx = u_nx;   // the next plane's (prefetch)
    auto fetch = [&](int kk) {
        const int zz = zt * ZT + kk;
        if (xy_ok && zz < v.D) {
            const int ll = zz * plane + y * v.W + x;
            u_nx = f.own(ll);
            if (IN4) {
                const float4 q = __ldg(reinterpret_cast<const float4*>(g0) + ll);
                g_nx = make_float3(q.x, q.y, q.z);
            } else {
                g_nx = make_float3(__ldg(g0 + ll), __ldg(g0 + v.V + ll), __ldg(g0 + 2 * v.V + ll));
            }
        }
    };
    if (PF) fetch(0);
    for (int k = 0; k < ZT; ++k) {
        const int z = zt * ZT + k;
        bool active = xy_ok && z < v.D;
        float w[8];
        float4 gs = make_float4(0.f, 0.f, 0.f, 0.f);
        int cb = -4;
        float3 u = make_float3(0.f, 0.f, 0.f), gpf = u;
        const int l = z * plane + y * v.W + x;
        if (PF) {
            u = u_nx;
            gpf = g_nx;
            if (k + 1 < ZT) fetch(k + 1);
        } else if (active) {
            u = f.own(l);
            if (FAR && near_source(scale * u.x, scale * u.y, scale * u.z)) active = false;
        }
        if (active) {
            const Cell c = make_cell_warp(z, y, x, scale * u.x, scale * u.y, scale * u.z, v);
            float gz, gy, gx;
            if (PF) {
                gz = gpf.x;
                gy = gpf.y;
                gx = gpf.z;
            } else if (IN4) {
                const float4 g4 = __ldg(reinterpret_cast<const float4*>(g0) + l);
                gz = g4.x;
                gy = g4.y;
                gx = g4.z;
            } else {
                gz = __ldg(g0 + l);
                gy = __ldg(g0 + v.V + l);
                gx = __ldg(g0 + 2 * v.V + l);
            }
            if (!FAR) {
                // identity + Jacobian term at the source voxel itself (scale: du_t = scale d src)
                const float3 jt = field_jac_t(f, c, v, make_float3(gz, gy, gx));
                atomicAdd(o + l, make_float4(fmaf(scale, jt.x, gz) * out_scale, fmaf(scale, jt.y, gy) * out_scale,
                                             fmaf(scale, jt.z, gx) * out_scale, 0.f));
            }
            tri_weights(c, w);
            gs = make_float4(gz * out_scale, gy * out_scale, gx * out_scale, 0.f);
            cb = c.base;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) w[q] = 0.f;
        }
        const bool merge = active && ca == cb;
        if (ca >= 0 && !merge) {                     // the carried corners are not this cell's: send them
            atomicAdd(o + ca, cl[0]);
            atomicAdd(o + ca + 1, cu[0]);
            atomicAdd(o + ca + v.W, cl[1]);
            atomicAdd(o + ca + v.W + 1, cu[1]);
        }
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const float wl = w[2 * dy], wh = w[2 * dy + 1];
            float4 lo = make_float4(wl * gs.x, wl * gs.y, wl * gs.z, 0.f);
            const float4 hi = make_float4(wh * gs.x + (merge ? cu[dy].x : 0.f), wh * gs.y + (merge ? cu[dy].y : 0.f),
                                          wh * gs.z + (merge ? cu[dy].z : 0.f), 0.f);
            if (merge) {
                lo.x += cl[dy].x;
                lo.y += cl[dy].y;
                lo.z += cl[dy].z;
            }
            emit4_xpair(o, cb + dy * v.W, active, lo, hi, lane);
        }
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const float wl = w[4 + 2 * dy], wh = w[5 + 2 * dy];
            cl[dy] = make_float4(wl * gs.x, wl * gs.y, wl * gs.z, 0.f);
            cu[dy] = make_float4(wh * gs.x, wh * gs.y, wh * gs.z, 0.f);
        }
        ca = active ? cb + plane : -1;
    }
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) emit4_xpair(o, ca + dy * v.W, ca >= 0, cl[dy], cu[dy], lane);
}

// Far-source transpose terms onto planar gradients [B][3][V]: one atomic per
// corner and channel (far sources are few where this layout is used).
template <bool IN4, class Src>
__global__ void __launch_bounds__(VT_THREADS)
exp_far_planar_kernel(Src src_all, float scale, const float* __restrict__ gin, float* __restrict__ gout,
                      float out_scale, Vol v, int nzt, int* flags)
{
    if (!far_tile(flags)) return;
    const int x = blockIdx.x * VT_X + threadIdx.x;
    const int y = blockIdx.y * VT_Y + threadIdx.y;
    const int zt = blockIdx.z % nzt;
    const int b = blockIdx.z / nzt;
    if (x >= v.W || y >= v.H) return;
    const Src f = src_all.subject(b);
    const float* g0 = gin + (size_t)b * (IN4 ? 4 : 3) * v.V;
    float* o = gout + (size_t)b * 3 * v.V;
    const int plane = v.H * v.W;
    for (int k = 0; k < FAR_Z; ++k) {
        const int z = zt * FAR_Z + k;
        if (z >= v.D) break;
        const int l = z * plane + y * v.W + x;
        const float3 u = f.own(l);
        const float uz = scale * u.x, uy = scale * u.y, ux = scale * u.z;
        if (near_source(uz, uy, ux)) continue;
        const Cell c = make_cell(z, y, x, uz, uy, ux, v);
        float gz, gy, gx;
        if (IN4) {
            const float4 g4 = __ldg(reinterpret_cast<const float4*>(g0) + l);
            gz = g4.x;
            gy = g4.y;
            gx = g4.z;
        } else {
            gz = __ldg(g0 + l);
            gy = __ldg(g0 + v.V + l);
            gx = __ldg(g0 + 2 * v.V + l);
        }
        float w[8];
        tri_weights(c, w);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int a = c.base + ((q >> 2) & 1) * plane + ((q >> 1) & 1) * v.W + (q & 1);
            const float s = w[q] * out_scale;
            atomicAdd(o + a, s * gz);
            atomicAdd(o + v.V + a, s * gy);
            atomicAdd(o + 2 * v.V + a, s * gx);
        }
    }
}

// g[b][c][l] = g4[b][l].c: an interleaved gradient back to planar fields
__global__ void __launch_bounds__(256)
unpack_field_kernel(const float4* __restrict__ g4, float* __restrict__ g, long long V, long long n)
{
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
        const long long b = e / V, l = e - b * V;
        const float4 q = __ldg(g4 + e);
        float* gb = g + (size_t)b * 3 * V;
        gb[l] = q.x;
        gb[V + l] = q.y;
        gb[2 * V + l] = q.z;
    }
}

dim3 voxel_grid(int B, const Vol& v, int& nzt, int zt)
{
    nzt = div_up(v.D, zt);
    return dim3(div_up(v.W, VT_X), div_up(v.H, VT_Y), nzt * B);
}

}  // namespace

cudaError_t exp_square(const float* src, float scale, float* dst, int B, const Vol& v,
                       cudaStream_t s)
{
    int nzt;
    const dim3 grid = voxel_grid(B, v, nzt, SQ_Z);
    exp_square_kernel<PlanarField, false><<<grid, dim3(VT_X, VT_Y), 0, s>>>(PlanarField{src, v.V}, scale, dst, v,
                                                                            nzt);
    return cudaGetLastError();
}

cudaError_t exp_square_packed(const float* src, int src_packed, float scale, float4* dst, int B, const Vol& v,
                              cudaStream_t s, float4* zero)
{
    if ((reinterpret_cast<uintptr_t>(dst) & 15) || (src_packed && (reinterpret_cast<uintptr_t>(src) & 15)) ||
        (reinterpret_cast<uintptr_t>(zero) & 15))
        return cudaErrorMisalignedAddress;
    int nzt;
    const dim3 grid = voxel_grid(B, v, nzt, SQ_Z);
    float* d = reinterpret_cast<float*>(dst);
    if (src_packed && DARC_SQ_STAGED) {
        int nzs;
        const dim3 gs = voxel_grid(B, v, nzs, SQS_Z);
        exp_square_staged_kernel<<<gs, dim3(VT_X, VT_Y), 0, s>>>(
            PackedField{reinterpret_cast<const float4*>(src), v.V}, scale, dst, v, nzs, zero);
    } else if (src_packed)
        exp_square_kernel<PackedField, true><<<grid, dim3(VT_X, VT_Y), 0, s>>>(
            PackedField{reinterpret_cast<const float4*>(src), v.V}, scale, d, v, nzt, zero);
    else
        exp_square_kernel<PlanarField, true><<<grid, dim3(VT_X, VT_Y), 0, s>>>(PlanarField{src, v.V}, scale, d, v,
                                                                               nzt, zero);
    return cudaGetLastError();
}

cudaError_t exp_square_adjoint(const float* src, float scale, const float* gin, float* gout,
                               float out_scale, int B, const Vol& v, cudaStream_t s)
{
    int nzt;
    const dim3 grid = voxel_grid(B, v, nzt, ADJ_Z);
    // 8-byte atomics need every channel plane 8-byte aligned (V even, aligned base)
    const int vec2 = (v.V % 2 == 0) && ((reinterpret_cast<uintptr_t>(gout) & 7) == 0);
    exp_square_adjoint_kernel<<<grid, dim3(VT_X, VT_Y), 0, s>>>(src, scale, gin, gout, out_scale, v,
                                                                nzt, vec2);
    return cudaGetLastError();
}

template <class Src>
void launch_adjoint4(Src f, float scale, const float* gin, int gin_interleaved, float4* gout, float out_scale,
                     dim3 grid, const Vol& v, int nzt, cudaStream_t s)
{
    if (gin_interleaved)
        exp_square_adjoint4_kernel<true, Src><<<grid, dim3(VT_X, ADJ_Y), 0, s>>>(f, scale, gin, gout, out_scale, v, nzt);
    else
        exp_square_adjoint4_kernel<false, Src><<<grid, dim3(VT_X, ADJ_Y), 0, s>>>(f, scale, gin, gout, out_scale, v, nzt);
}

cudaError_t exp_square_adjoint4(const float* src, int src_packed, float scale, const float* gin, int gin_interleaved,
                                float4* gout, float out_scale, int B, const Vol& v, cudaStream_t s)
{
    if ((reinterpret_cast<uintptr_t>(gout) & 15) || (gin_interleaved && (reinterpret_cast<uintptr_t>(gin) & 15)) ||
        (src_packed && (reinterpret_cast<uintptr_t>(src) & 15)))
        return cudaErrorMisalignedAddress;
    int nzt;
    dim3 grid = voxel_grid(B, v, nzt, ADJ_Z);
    grid.y = div_up(v.H, ADJ_Y);
    if (src_packed)
        launch_adjoint4(PackedField{reinterpret_cast<const float4*>(src), v.V}, scale, gin, gin_interleaved, gout,
                        out_scale, grid, v, nzt, s);
    else
        launch_adjoint4(PlanarField{src, v.V}, scale, gin, gin_interleaved, gout, out_scale, grid, v, nzt, s);
    return cudaGetLastError();
}

template <class Src>
void launch_far(Src f, float scale, const float* gin, int in4, float* gout, int out4, float out_scale, int* flags,
                dim3 grid, const Vol& v, int nzt, cudaStream_t s)
{
    const dim3 block(VT_X, VT_Y);
    float4* g4 = reinterpret_cast<float4*>(gout);
    if (out4 && in4)
        exp_square_adjoint4_kernel<true, Src, true><<<grid, block, 0, s>>>(f, scale, gin, g4, out_scale, v, nzt, flags);
    else if (out4)
        exp_square_adjoint4_kernel<false, Src, true><<<grid, block, 0, s>>>(f, scale, gin, g4, out_scale, v, nzt, flags);
    else if (in4)
        exp_far_planar_kernel<true, Src><<<grid, block, 0, s>>>(f, scale, gin, gout, out_scale, v, nzt, flags);
    else
        exp_far_planar_kernel<false, Src><<<grid, block, 0, s>>>(f, scale, gin, gout, out_scale, v, nzt, flags);
}

cudaError_t exp_adjoint_far(const float* src, int src_packed, float scale, const float* gin, int gin_interleaved,
                            float* gout, int gout_interleaved, float out_scale, int* flags, int B, const Vol& v,
                            cudaStream_t s)
{
    static_assert(FAR_Z == 8 && VT_X == 32 && VT_Y == 8, "far-scatter blocks are the gather's 32 x 8 x 8 mark tiles");
    if ((src_packed && (reinterpret_cast<uintptr_t>(src) & 15)) ||
        (gin_interleaved && (reinterpret_cast<uintptr_t>(gin) & 15)) ||
        (gout_interleaved && (reinterpret_cast<uintptr_t>(gout) & 15)))
        return cudaErrorMisalignedAddress;
    int nzt;
    const dim3 grid = voxel_grid(B, v, nzt, FAR_Z);
    if (src_packed)
        launch_far(PackedField{reinterpret_cast<const float4*>(src), v.V}, scale, gin, gin_interleaved, gout,
                   gout_interleaved, out_scale, flags, grid, v, nzt, s);
    else
        launch_far(PlanarField{src, v.V}, scale, gin, gin_interleaved, gout, gout_interleaved, out_scale, flags, grid,
                   v, nzt, s);
    return cudaGetLastError();
}

cudaError_t unpack_field(const float4* g4, float* g, int B, const Vol& v, cudaStream_t s)
{
    const long long n = (long long)B * v.V;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    unpack_field_kernel<<<blocks, 256, 0, s>>>(g4, g, v.V, n);
    return cudaGetLastError();
}

}  // namespace darc_impl
