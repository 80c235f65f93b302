// k_exp_gather.cu -- the scatter-free adjoint of one squaring (sm_103a).
//
// One squaring of Exp (arXiv 2508.10743, Sec. "Diffeomorphisms") is
// u_{t+1}(x) = u_t(x) + S(u_t, x + u_t(x)).  With g = dL/du_{t+1}, its adjoint
//
//   dL/du_t(x) = g(x) + J(x)^T g(x) + sum_y w(y -> x) g(y)
//
// has a term at the voxel itself (J(x) = dS(u_t, p)/dp at p = x + u_t(x)) and
// the transpose of the interpolation: w(y -> x) is the trilinear weight that
// the sample point of y puts on the lattice point x.  Along each axis that
// weight is the hat max(0, 1 - |u_a(y) - (x_a - y_a)|), so a source whose
// displacement is below one voxel on every axis ("near") reaches only
// x - y in {-1, 0, 1}^3, and for |u_a| < 1 the three hats are max(u_a, 0),
// 1 - |u_a| and max(-u_a, 0) for x_a - y_a = +1, 0, -1.
//
// exp_gather_kernel writes every target once, with a plain store: the
// identity and Jacobian terms plus the near sources among its 27
// neighbours.  A block owns a 32 x 16 x 16 tile of targets; it stages one
// source plane at a time (the tile's 34 x 18 sources with a one-voxel halo,
// displacement and gradient) in shared memory and walks z.  A thread owns
// four targets of one (x) column and keeps their sums for the planes
// z - 1, z, z + 1 in registers, so every staged source is read by three
// lanes and the rows it reaches, not by all 27 of its targets.  At a face of
// the volume a source that points outward samples the face itself (border
// padding), which the hats reproduce with that axis' displacement set to 0.
//
// Far sources (|u_a| >= 1 on some axis, or not finite) are left out of the
// gather.  The gather marks each 32 x 8 x 8 tile that holds one, and the
// scatter that follows (exp_far_scatter in k_exp.cu) visits only those
// tiles and adds the far sources' transpose terms with atomics onto the
// stored values.  Stale marks only cost time: the scatter clears each mark
// it visits, and a source is scattered only if it is far.
#include "kernels.h"

namespace darc_impl {
namespace {

constexpr int GA_TX = 32;                  // targets along x per block (one per lane)
constexpr int GA_RY = 4;                   // target rows per thread
constexpr int GA_WARPS = 4;
constexpr int GA_TY = GA_RY * GA_WARPS;    // 16 target rows per block
constexpr int GA_TZ = 16;                  // target planes per block
constexpr int GA_SX = GA_TX + 2, GA_SY = GA_TY + 2;
constexpr int GA_HALO = 2 * GA_SX + 2 * GA_TY;   // halo sources of a staged plane
constexpr int GA_THREADS = 32 * GA_WARPS;
static_assert(GA_HALO <= GA_THREADS, "one halo source per thread at most");
// far-scatter tiles (the scatter's blocks): 32 x 8 x 8 voxels
constexpr int FT_X = 32, FT_Y = 8, FT_Z = 8;

// Staged source plane: per source (with a one-voxel halo) the hats of its
// displacement and its gradient, all zero for far or outside sources.
//   a = (hat z -1, hat z 0, hat z +1, u_y)    (hat a d: weight on x_a - y_a = d)
//   b = (g_z, g_y, g_x, hat y 0)
//   hx[d + 1] = hat x d
// u is taken with outward border moves zeroed.
struct GatherPlane {
    float4 a[GA_SY][GA_SX];
    float4 b[GA_SY][GA_SX];
    float hx[3][GA_SY][GA_SX];
};

// Paired FP32 arithmetic (FFMA2 / FADD2 / FMUL2 on sm_100 and later): two
// IEEE single operations per instruction, per lane identical to the scalar
// fmaf, + and *.
__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// gradient g at voxel l of subject field base g0
template <bool IN4>
__device__ __forceinline__ float3 load_g(const float* __restrict__ g0, int l, long long V)
{
    if (IN4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(g0) + l);
        return make_float3(q.x, q.y, q.z);
    }
    return make_float3(__ldg(g0 + l), __ldg(g0 + V + l), __ldg(g0 + 2 * V + l));
}

__device__ __forceinline__ bool is_near(float3 u)
{
    return fabsf(u.x) < 1.f && fabsf(u.y) < 1.f && fabsf(u.z) < 1.f;   // false for NaN
}

// the displacement a near source at coordinate q (extent n) contributes
// with: an outward move at a face samples the face (border padding)
__device__ __forceinline__ float border_disp(float u, int q, int n)
{
    return ((q == 0 && u < 0.f) || (q == n - 1 && u > 0.f)) ? 0.f : u;
}

__device__ __forceinline__ void stage(GatherPlane& sp, int sy, int sx, bool near, float3 u, float3 g, int z, int y,
                                      int x, const Vol& v)
{
    if (near) {
        const float uz = border_disp(u.x, z, v.D), uy = border_disp(u.y, y, v.H), ux = border_disp(u.z, x, v.W);
        sp.a[sy][sx] = make_float4(fmaxf(-uz, 0.f), 1.f - fabsf(uz), fmaxf(uz, 0.f), uy);
        sp.b[sy][sx] = make_float4(g.x, g.y, g.z, 1.f - fabsf(uy));
        sp.hx[0][sy][sx] = fmaxf(-ux, 0.f);
        sp.hx[1][sy][sx] = 1.f - fabsf(ux);
        sp.hx[2][sy][sx] = fmaxf(ux, 0.f);
    } else {
        sp.a[sy][sx] = make_float4(0.f, 0.f, 0.f, 0.f);
        sp.b[sy][sx] = make_float4(0.f, 0.f, 0.f, 0.f);
        sp.hx[0][sy][sx] = sp.hx[1][sy][sx] = sp.hx[2][sy][sx] = 0.f;
    }
}

// per target row: the (z, y) channels paired, x alone
struct Acc {
    float2 p[GA_RY];
    float s[GA_RY];
};

// raw displacement (scaled) and gradient of this thread's sources of one plane
struct Raw {
    float3 u[GA_RY], g[GA_RY];
    float3 hu, hg;
};

template <class Src, bool IN4, bool OUT4>
struct Gather {
    Src f;
    float scale, out_scale;
    const float* __restrict__ g0;
    float* __restrict__ gout;
    int* __restrict__ flags;
    Vol v;
    int lane, wy, x0, y0, z0, zend, x, row0, b, hy, hxc, plane;
    GatherPlane& sp;

    __device__ __forceinline__ bool own_ok(int j) const { return x < v.W && row0 + j < v.H; }
    __device__ __forceinline__ bool halo_ok() const
    {
        const int y = y0 - 1 + hy, xx = x0 - 1 + hxc;
        return hy >= 0 && y >= 0 && y < v.H && xx >= 0 && xx < v.W;
    }

    __device__ __forceinline__ void load(int zs, Raw& r) const
    {
        const bool pin = zs >= 0 && zs < v.D;
#pragma unroll
        for (int j = 0; j < GA_RY; ++j) {
            r.u[j] = r.g[j] = make_float3(0.f, 0.f, 0.f);
            if (pin && own_ok(j)) {
                const int l = zs * plane + (row0 + j) * v.W + x;
                const float3 q = f.own(l);
                r.u[j] = make_float3(scale * q.x, scale * q.y, scale * q.z);
                r.g[j] = load_g<IN4>(g0, l, v.V);
            }
        }
        r.hu = r.hg = make_float3(0.f, 0.f, 0.f);
        if (pin && halo_ok()) {
            const int l = zs * plane + (y0 - 1 + hy) * v.W + x0 - 1 + hxc;
            const float3 q = f.own(l);
            r.hu = make_float3(scale * q.x, scale * q.y, scale * q.z);
            r.hg = load_g<IN4>(g0, l, v.V);
        }
    }

    // one source plane zs: am, a0, ap hold the target planes zs - 1, zs, zs + 1
    __device__ __forceinline__ void plane_step(int zs, Acc& am, Acc& a0, Acc& ap, Raw& r) const
    {
        const bool pin = zs >= 0 && zs < v.D;
        bool near_any = false;
        if (pin) {
            const bool own_plane = zs >= z0 && zs < zend;
            __syncthreads();                           // the previous plane has been read
            bool far_any = false;
#pragma unroll
            for (int j = 0; j < GA_RY; ++j) {
                const int y = row0 + j;
                const bool ok = own_ok(j);
                const bool near = ok && is_near(r.u[j]);
                near_any |= near;
                if (own_plane && ok) {
                    far_any |= !near;
                    const Cell c = make_cell_warp(zs, y, x, r.u[j].x, r.u[j].y, r.u[j].z, v);
                    const float3 jt = field_jac_t(f, c, v, r.g[j]);
                    a0.p[j] = fma2(dup2(scale), p2(jt.x, jt.y), add2(a0.p[j], p2(r.g[j].x, r.g[j].y)));
                    a0.s[j] = fmaf(scale, jt.z, a0.s[j] + r.g[j].z);
                }
                stage(sp, 1 + GA_RY * wy + j, 1 + lane, near, r.u[j], r.g[j], zs, y, x, v);
            }
            if (hy >= 0) {
                const bool near = halo_ok() && is_near(r.hu);
                near_any |= near;
                stage(sp, hy, hxc, near, r.hu, r.hg, zs, y0 - 1 + hy, x0 - 1 + hxc, v);
            }
            // one mark per warp: the warp's targets lie in one far-scatter tile
            if (own_plane && __any_sync(0xffffffffu, far_any) && lane == 0 && x0 < v.W && row0 < v.H) {
                const int ntx = (v.W + FT_X - 1) / FT_X, nty = (v.H + FT_Y - 1) / FT_Y, ntz = (v.D + FT_Z - 1) / FT_Z;
                flags[(((size_t)b * ntz + zs / FT_Z) * nty + row0 / FT_Y) * ntx + x0 / FT_X] = 1;
            }
        }
        if (zs + 1 <= zend) load(zs + 1, r);           // in flight while this plane is summed
        if (pin && __syncthreads_or(near_any)) {
            // transpose terms of the staged near sources
#pragma unroll
            for (int dxs = 0; dxs < 3; ++dxs) {        // source column x - 1 + dxs
#pragma unroll
                for (int i = 0; i < GA_RY + 2; ++i) {  // source row row0 - 1 + i
                    const int ry = GA_RY * wy + i, cx = lane + dxs;
                    const float4 A = sp.a[ry][cx];
                    const float4 Bq = sp.b[ry][cx];
                    const float hxw = sp.hx[2 - dxs][ry][cx];
                    const float2 g2 = mul2(p2(Bq.x, Bq.y), dup2(hxw));
                    const float g1 = Bq.z * hxw;
                    const float2 hzm = dup2(A.x), hz0 = dup2(A.y), hzp = dup2(A.z);
#pragma unroll
                    for (int j = 0; j < GA_RY; ++j) {
                        const int dy = j + 1 - i;      // target row - source row
                        if (dy < -1 || dy > 1) continue;
                        const float hyw = dy == 1 ? fmaxf(A.w, 0.f) : (dy == 0 ? Bq.w : fmaxf(-A.w, 0.f));
                        const float2 c2 = mul2(g2, dup2(hyw));
                        const float c1 = g1 * hyw;
                        am.p[j] = fma2(hzm, c2, am.p[j]);
                        am.s[j] = fmaf(A.x, c1, am.s[j]);
                        a0.p[j] = fma2(hz0, c2, a0.p[j]);
                        a0.s[j] = fmaf(A.y, c1, a0.s[j]);
                        ap.p[j] = fma2(hzp, c2, ap.p[j]);
                        ap.s[j] = fmaf(A.z, c1, ap.s[j]);
                    }
                }
            }
        }
        // target plane zs - 1 is complete
        const int zo = zs - 1;
        if (zo >= z0 && zo < zend && x < v.W) {
#pragma unroll
            for (int j = 0; j < GA_RY; ++j) {
                const int y = row0 + j;
                if (y >= v.H) break;
                const size_t l = (size_t)zo * plane + (size_t)y * v.W + x;
                const float2 o2 = mul2(dup2(out_scale), am.p[j]);
                const float o1 = out_scale * am.s[j];
                if (OUT4) {
                    reinterpret_cast<float4*>(gout)[(size_t)b * v.V + l] = make_float4(o2.x, o2.y, o1, 0.f);
                } else {
                    float* o = gout + (size_t)b * 3 * v.V + l;
                    o[0] = o2.x;
                    o[v.V] = o2.y;
                    o[2 * v.V] = o1;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < GA_RY; ++j) {
            am.p[j] = make_float2(0.f, 0.f);
            am.s[j] = 0.f;
        }
    }
};

template <class Src, bool IN4, bool OUT4>
__global__ void __launch_bounds__(GA_THREADS, 4)
exp_gather_kernel(Src src_all, float scale, const float* __restrict__ gin, float* __restrict__ gout,
                  float out_scale, Vol v, int nzt, int* __restrict__ flags)
{
    __shared__ GatherPlane sp;
    const int lane = threadIdx.x, wy = threadIdx.y;
    const int tid = wy * 32 + lane;
    const int zt = blockIdx.z % nzt, b = blockIdx.z / nzt;
    // this thread's halo source of every staged plane (tid < GA_HALO)
    int hy = -1, hxc = -1;
    if (tid < GA_SX) {
        hy = 0; hxc = tid;
    } else if (tid < 2 * GA_SX) {
        hy = GA_SY - 1; hxc = tid - GA_SX;
    } else if (tid < 2 * GA_SX + GA_TY) {
        hy = 1 + tid - 2 * GA_SX; hxc = 0;
    } else if (tid < GA_HALO) {
        hy = 1 + tid - 2 * GA_SX - GA_TY; hxc = GA_SX - 1;
    }
    const int x0 = blockIdx.x * GA_TX, y0 = blockIdx.y * GA_TY, z0 = zt * GA_TZ;
    const Gather<Src, IN4, OUT4> G{src_all.subject(b), scale, out_scale, gin + (size_t)b * (IN4 ? 4 : 3) * v.V,
                                   gout, flags, v, lane, wy, x0, y0, z0, min(z0 + GA_TZ, v.D), x0 + lane,
                                   y0 + GA_RY * wy, b, hy, hxc, v.H * v.W, sp};
    Acc P, Q, R;
#pragma unroll
    for (int j = 0; j < GA_RY; ++j) {
        P.p[j] = Q.p[j] = R.p[j] = make_float2(0.f, 0.f);
        P.s[j] = Q.s[j] = R.s[j] = 0.f;
    }
    Raw raw;
    G.load(z0 - 1, raw);
    // three source planes per trip, so the three sums rotate without copies
    for (int zs = z0 - 1; zs <= G.zend; zs += 3) {
        G.plane_step(zs, P, Q, R, raw);
        if (zs + 1 <= G.zend) G.plane_step(zs + 1, Q, R, P, raw);
        if (zs + 2 <= G.zend) G.plane_step(zs + 2, R, P, Q, raw);
    }
}

template <class Src>
void launch_gather(Src f, float scale, const float* gin, int in4, float* gout, int out4, float out_scale, int* flags,
                   int B, const Vol& v, cudaStream_t s)
{
    const int nzt = div_up(v.D, GA_TZ);
    const dim3 grid(div_up(v.W, GA_TX), div_up(v.H, GA_TY), nzt * B), block(32, GA_WARPS);
    if (in4 && out4)
        exp_gather_kernel<Src, true, true><<<grid, block, 0, s>>>(f, scale, gin, gout, out_scale, v, nzt, flags);
    else if (in4)
        exp_gather_kernel<Src, true, false><<<grid, block, 0, s>>>(f, scale, gin, gout, out_scale, v, nzt, flags);
    else if (out4)
        exp_gather_kernel<Src, false, true><<<grid, block, 0, s>>>(f, scale, gin, gout, out_scale, v, nzt, flags);
    else
        exp_gather_kernel<Src, false, false><<<grid, block, 0, s>>>(f, scale, gin, gout, out_scale, v, nzt, flags);
}

}  // namespace

size_t exp_far_flags(int B, const Vol& v)
{
    return (size_t)B * div_up(v.D, FT_Z) * div_up(v.H, FT_Y) * div_up(v.W, FT_X);
}

cudaError_t exp_adjoint_gather(const float* src, int src_packed, float scale, const float* gin, int gin_interleaved,
                               float* gout, int gout_interleaved, float out_scale, int* flags, int B, const Vol& v,
                               cudaStream_t s)
{
    if ((src_packed && (reinterpret_cast<uintptr_t>(src) & 15)) ||
        (gin_interleaved && (reinterpret_cast<uintptr_t>(gin) & 15)) ||
        (gout_interleaved && (reinterpret_cast<uintptr_t>(gout) & 15)))
        return cudaErrorMisalignedAddress;
    if (src_packed)
        launch_gather(PackedField{reinterpret_cast<const float4*>(src), v.V}, scale, gin, gin_interleaved, gout,
                      gout_interleaved, out_scale, flags, B, v, s);
    else
        launch_gather(PlanarField{src, v.V}, scale, gin, gin_interleaved, gout, gout_interleaved, out_scale, flags, B,
                      v, s);
    return cudaGetLastError();
}

}  // namespace darc_impl
