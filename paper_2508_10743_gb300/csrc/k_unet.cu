// k_unet.cu -- BF16 tensor-core (tcgen05, TMEM) kernels for the learned
// warm start: a dense GEMM core and the implicit-GEMM 3-D convolutions of the
// U-Net (forward, data gradient, weight gradient).
#include "kernels.h"
#include "umma.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace darc_impl {
namespace {

using bf16 = __nv_bfloat16;
constexpr int TC_M = 128;            // rows of a CTA tile (TMEM lanes)
constexpr int TC_KC = 64;            // K elements staged per round (4 MMAs of K = 16)
constexpr long long TC_WAIT = 1LL << 26;

// C[M x N] (fp32, row-major) = A[M x K] (bf16, K contiguous) * B[N x K]^T
// (bf16, K contiguous).  Grid: M / 128 CTAs of 128 threads; N <= 256.
__global__ void __launch_bounds__(128)
gemm_bf16_kernel(const bf16* __restrict__ A, const bf16* __restrict__ B, float* __restrict__ C, int N, int K)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M;
    uint8_t* sA = smem;                                  // 128 x 64 bf16 = 16 KB
    uint8_t* sB = smem + TC_M * TC_KC * 2;               // N x 64 bf16
    const uint32_t lboA = (TC_M / 8) * 128, lboB = (uint32_t)(N / 8) * 128;
    uint32_t ncols = 32;
    while ((int)ncols < N) ncols <<= 1;
    if (warp == 0) umma::tmem_alloc(&tslot, ncols);
    if (tid == 0) {
        umma::mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t idesc = umma::idesc_bf16_f32(TC_M, N);
    bool ok = true;
    uint32_t phase = 0;
    for (int k0 = 0; k0 < K; k0 += TC_KC) {
        const int kc = min(TC_KC, K - k0);               // multiple of 16
        // stage A: row r, 8-element group g  ->  core matrix layout
        for (int e = tid; e < TC_M * (kc / 8); e += 128) {
            const int r = e / (kc / 8), g = e % (kc / 8);
            const uint4 val = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * K + k0 + 8 * g);
            *reinterpret_cast<uint4*>(sA + umma::kmajor_offset(r, 8 * g, lboA)) = val;
        }
        for (int e = tid; e < N * (kc / 8); e += 128) {
            const int r = e / (kc / 8), g = e % (kc / 8);
            const uint4 val = *reinterpret_cast<const uint4*>(B + (size_t)r * K + k0 + 8 * g);
            *reinterpret_cast<uint4*>(sB + umma::kmajor_offset(r, 8 * g, lboB)) = val;
        }
        umma::fence_smem_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            for (int j = 0; j < kc / 16; ++j) {
                const uint64_t da = umma::smem_desc(umma::smem_u32(sA) + 2 * j * lboA, lboA, 128);
                const uint64_t db = umma::smem_desc(umma::smem_u32(sB) + 2 * j * lboB, lboB, 128);
                umma::mma_bf16(tmem, da, db, idesc, (k0 + 16 * j) > 0);
            }
            umma::commit(&mbar);
        }
        ok = umma::mbar_wait(&mbar, phase, TC_WAIT) && ok;
        phase ^= 1;
        umma::fence_after_sync();
        __syncthreads();
    }
    // epilogue: warp w holds rows 32w .. 32w + 31 (TMEM lanes)
    const int row = m0 + 32 * warp + lane;
    for (int c = 0; c < N; c += 8) {
        float v[8];
        umma::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
#pragma unroll
        for (int j = 0; j < 8; ++j) C[(size_t)row * N + c + j] = ok ? v[j] : __int_as_float(0x7fc00000);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}


// ---------------------------------------------------------------------------
// 3x3x3 'same' convolution as an implicit GEMM on the tensor cores.
//   out[v][co] = act( sum_{tap, ci} in[v + off(tap)][ci] * W[co][tap*cin + ci] + bias[co] )
// Activations are channels-last bf16 with a per-voxel stride (multiple of 8)
// so a layer can read or write a channel slice of a wider buffer (skip
// concatenation costs nothing).  Rows of the GEMM are 128 consecutive voxels
// of the batch; K runs over (tap, channel) in groups of 8 channels (16 bytes,
// one gather); N is the padded output channel count (<= 128).  Two shared
// stages alternate so the gathers of one overlap the MMAs of the other.
struct ConvArgs {
    const bf16* in;
    int in_stride, cin;           // channels used: [0, cin), cin % 8 == 0
    const bf16* wt;               // [np][kp] bf16, k = tap * cin + ci, zero padded
    const float* bias;            // [cout] or null
    bf16* out;
    int out_stride, out_off, cout;
    float* out_f32;               // optional planar fp32 output [batch][cout][D*H*W] (instead of out)
    const bf16* gate;             // optional: result *= (gate > 0 ? 1 : slope), gate channels-last
    int gate_stride;
    int act;                      // 1: leaky ReLU
    float slope;
    int D, H, W;
    long long nvox;               // batch * D * H * W
    int kp, np;
};

constexpr int CONV_SMEM_STAGE_A = TC_M * TC_KC * 2;     // 16 KB

__global__ void __launch_bounds__(128)
conv3_fwd_kernel(ConvArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long m0 = (long long)blockIdx.x * TC_M;
    const int stageB = a.np * TC_KC * 2;
    uint8_t* sA[2] = {smem, smem + CONV_SMEM_STAGE_A + stageB};
    uint8_t* sB[2] = {smem + CONV_SMEM_STAGE_A, smem + 2 * CONV_SMEM_STAGE_A + stageB};
    const uint32_t lboA = (TC_M / 8) * 128, lboB = (uint32_t)(a.np / 8) * 128;
    uint32_t ncols = 32;
    while ((int)ncols < a.np) ncols <<= 1;
    if (warp == 0) umma::tmem_alloc(&tslot, ncols);
    if (tid == 0) {
        umma::mbar_init(&mbar[0], 1);
        umma::mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t idesc = umma::idesc_bf16_f32(TC_M, a.np);
    const long long plane = (long long)a.H * a.W, vol = (long long)a.D * plane;
    bool ok = true;
    const int steps = (a.kp + TC_KC - 1) / TC_KC;
    for (int i = 0; i < steps; ++i) {
        const int st = i & 1;
        if (i >= 2) ok = umma::mbar_wait(&mbar[st], ((i - 2) >> 1) & 1, TC_WAIT) && ok;
        const int k0 = i * TC_KC, kc = min(TC_KC, a.kp - k0);
        const int ng = kc / 8;
        // A: implicit im2col gather, one 16-byte group of 8 channels per load
        for (int e = tid; e < TC_M * ng; e += 128) {
            const int r = e / ng, g = e - r * ng;
            const int k = k0 + 8 * g;
            const int tap = k / a.cin, ci = k - tap * a.cin;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            const long long v = m0 + r;
            if (tap < 27 && v < a.nvox) {
                const long long bb = v / vol, rem = v - bb * vol;
                const int z = (int)(rem / plane), y = (int)((rem / a.W) % a.H), x = (int)(rem % a.W);
                const int zz = z + tap / 9 - 1, yy = y + (tap / 3) % 3 - 1, xx = x + tap % 3 - 1;
                if (zz >= 0 && zz < a.D && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
                    const long long nv = bb * vol + ((long long)zz * a.H + yy) * a.W + xx;
                    val = *reinterpret_cast<const uint4*>(a.in + nv * a.in_stride + ci);
                }
            }
            *reinterpret_cast<uint4*>(sA[st] + umma::kmajor_offset(r, 8 * g, lboA)) = val;
        }
        for (int e = tid; e < a.np * ng; e += 128) {
            const int r = e / ng, g = e - r * ng;
            const uint4 val = *reinterpret_cast<const uint4*>(a.wt + (size_t)r * a.kp + k0 + 8 * g);
            *reinterpret_cast<uint4*>(sB[st] + umma::kmajor_offset(r, 8 * g, lboB)) = val;
        }
        umma::fence_smem_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            for (int j = 0; j < kc / 16; ++j) {
                const uint64_t da = umma::smem_desc(umma::smem_u32(sA[st]) + 2 * j * lboA, lboA, 128);
                const uint64_t db = umma::smem_desc(umma::smem_u32(sB[st]) + 2 * j * lboB, lboB, 128);
                umma::mma_bf16(tmem, da, db, idesc, (k0 + 16 * j) > 0);
            }
            umma::commit(&mbar[st]);
        }
    }
    // the last two commits (one per stage) retire in order: wait for both
    for (int i = max(steps - 2, 0); i < steps; ++i) ok = umma::mbar_wait(&mbar[i & 1], (i >> 1) & 1, TC_WAIT) && ok;
    umma::fence_after_sync();
    // epilogue: warp w holds voxels m0 + 32w .. m0 + 32w + 31 (TMEM lanes)
    const long long v = m0 + 32 * warp + lane;
    const bool in_range = v < a.nvox;
    const long long vb = v / vol, vl = v - vb * vol;        // planar fp32 output is [batch][cout][vol]
    for (int c = 0; c < a.np; c += 8) {
        float r8[8];
        umma::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, r8);
        if (!in_range || c >= a.cout) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int co = c + j;
            if (co >= a.cout) break;
            float y = ok ? r8[j] : __int_as_float(0x7fc00000);
            if (a.bias) y += __ldg(a.bias + co);
            if (a.act == 1) y = y > 0.f ? y : a.slope * y;
            if (a.gate) {
                const float gt = __bfloat162float(a.gate[v * a.gate_stride + co]);
                y = gt > 0.f ? y : a.slope * y;
            }
            if (a.out_f32) a.out_f32[((size_t)vb * a.cout + co) * vol + vl] = y;
            else a.out[v * a.out_stride + a.out_off + co] = __float2bfloat16(y);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// Weight gradient of a conv layer as a GEMM over voxels on the tensor cores:
//   dW[co][k] = sum_v gz[v][co] * im2col(in)[v][k],  k = tap * cin + ci.
// Rows (TMEM lanes) are k in tiles of 128, columns co (np <= 128), K runs
// over a CTA's range of voxels.  Both operands are stored voxel-major (8
// channels per 16 bytes), so they are transposed while staging: one 16-byte
// load gives 8 rows of one K column.  Each CTA writes its partial sums;
// conv3_wgrad_reduce adds them in a fixed order.
struct WgradArgs {
    const bf16* in;
    int in_stride, cin;
    const bf16* gz;             // channels-last gradient wrt the pre-activation
    int gz_stride, cout;        // cout % 8 == 0 (padded storage)
    float* partial;             // [splits][kp][np]
    int D, H, W;
    long long nvox, chunk;      // voxels per split (multiple of 64)
    int kp, np;
};

__global__ void __launch_bounds__(128)
conv3_wgrad_kernel(WgradArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.x * TC_M;                       // first k row of this tile
    const long long v0 = (long long)blockIdx.y * a.chunk;
    const long long v1 = min(a.nvox, v0 + a.chunk);
    const int stageB = a.np * TC_KC * 2;
    uint8_t* sA[2] = {smem, smem + CONV_SMEM_STAGE_A + stageB};
    uint8_t* sB[2] = {smem + CONV_SMEM_STAGE_A, smem + 2 * CONV_SMEM_STAGE_A + stageB};
    const uint32_t lboA = (TC_M / 8) * 128, lboB = (uint32_t)(a.np / 8) * 128;
    uint32_t ncols = 32;
    while ((int)ncols < a.np) ncols <<= 1;
    if (warp == 0) umma::tmem_alloc(&tslot, ncols);
    if (tid == 0) {
        umma::mbar_init(&mbar[0], 1);
        umma::mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t idesc = umma::idesc_bf16_f32(TC_M, a.np);
    const long long plane = (long long)a.H * a.W, vol = (long long)a.D * plane;
    bool ok = true;
    const int steps = (int)((v1 - v0 + TC_KC - 1) / TC_KC);
    for (int i = 0; i < steps; ++i) {
        const int st = i & 1;
        if (i >= 2) ok = umma::mbar_wait(&mbar[st], ((i - 2) >> 1) & 1, TC_WAIT) && ok;
        const long long vb = v0 + (long long)i * TC_KC;
        bf16* A16 = reinterpret_cast<bf16*>(sA[st]);
        bf16* B16 = reinterpret_cast<bf16*>(sB[st]);
        // A: 64 voxels x 16 groups of 8 rows (k), transposed into K-major
        for (int e = tid; e < TC_KC * (TC_M / 8); e += 128) {
            const int j = e % TC_KC, mg = e / TC_KC;
            const int k = r0 + 8 * mg;
            const int tap = k / a.cin, ci = k - tap * a.cin;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            const long long v = vb + j;
            if (tap < 27 && k < a.kp && v < v1) {
                const long long bb = v / vol, rem = v - bb * vol;
                const int z = (int)(rem / plane), y = (int)((rem / a.W) % a.H), x = (int)(rem % a.W);
                const int zz = z + tap / 9 - 1, yy = y + (tap / 3) % 3 - 1, xx = x + tap % 3 - 1;
                if (zz >= 0 && zz < a.D && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
                    val = *reinterpret_cast<const uint4*>(a.in + (bb * vol + ((long long)zz * a.H + yy) * a.W + xx) * a.in_stride + ci);
            }
            const bf16* pv = reinterpret_cast<const bf16*>(&val);
#pragma unroll
            for (int q = 0; q < 8; ++q) A16[umma::kmajor_offset(8 * mg + q, j, lboA) >> 1] = pv[q];
        }
        // B: 64 voxels x (np / 8) groups of 8 output channels
        for (int e = tid; e < TC_KC * (a.np / 8); e += 128) {
            const int j = e % TC_KC, cg = e / TC_KC;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            const long long v = vb + j;
            if (v < v1 && 8 * cg < a.cout) val = *reinterpret_cast<const uint4*>(a.gz + v * a.gz_stride + 8 * cg);
            const bf16* pv = reinterpret_cast<const bf16*>(&val);
#pragma unroll
            for (int q = 0; q < 8; ++q) B16[umma::kmajor_offset(8 * cg + q, j, lboB) >> 1] = pv[q];
        }
        umma::fence_smem_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            for (int j = 0; j < TC_KC / 16; ++j) {
                const uint64_t da = umma::smem_desc(umma::smem_u32(sA[st]) + 2 * j * lboA, lboA, 128);
                const uint64_t db = umma::smem_desc(umma::smem_u32(sB[st]) + 2 * j * lboB, lboB, 128);
                umma::mma_bf16(tmem, da, db, idesc, (i > 0) || (j > 0));
            }
            umma::commit(&mbar[st]);
        }
    }
    for (int i = max(steps - 2, 0); i < steps; ++i) ok = umma::mbar_wait(&mbar[i & 1], (i >> 1) & 1, TC_WAIT) && ok;
    umma::fence_after_sync();
    const int row = r0 + 32 * warp + lane;
    float* out = a.partial + ((size_t)blockIdx.y * a.kp + row) * a.np;
    for (int c = 0; c < a.np; c += 8) {
        float r8[8];
        umma::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, r8);
        if (row < a.kp) {
#pragma unroll
            for (int j = 0; j < 8; ++j) out[c + j] = (steps > 0 && ok) ? r8[j] : (ok ? 0.f : __int_as_float(0x7fc00000));
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

// dw[co][k] = sum over splits of partial[s][k][co] (fixed order)
__global__ void conv3_wgrad_reduce_kernel(const float* __restrict__ partial, int splits, int kp, int np,
                                          float* __restrict__ dw)
{
    const long long n = (long long)kp * np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / np), co = (int)(e % np);
        float s = 0.f;
        for (int q = 0; q < splits; ++q) s += partial[(size_t)q * n + e];
        dw[(size_t)co * kp + k] = s;
    }
}

// db[c] = sum_v gz[v][c], c < 8 G (G groups of 8 channels, G | 256).  Each
// block strides over voxels with 16-byte loads and writes one partial row;
// bias_grad_reduce adds the rows in block order (deterministic).
constexpr int BG_BLOCKS = 304;

__global__ void __launch_bounds__(256)
bias_grad_kernel(const bf16* __restrict__ gz, int stride, long long nvox, int G, float* __restrict__ partial)
{
    __shared__ float sh[256][9];
    const int tid = threadIdx.x, slots = 256 / G;
    const int g = tid % G, slot = tid / G;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long v = (long long)blockIdx.x * slots + slot; v < nvox; v += (long long)gridDim.x * slots) {
        const uint4 raw = *reinterpret_cast<const uint4*>(gz + v * stride + 8 * g);
        const bf16* pv = reinterpret_cast<const bf16*>(&raw);
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] += __bfloat162float(pv[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) sh[tid][q] = acc[q];
    __syncthreads();
    if (tid < 8 * G) {
        const int gg = tid / 8, q = tid % 8;
        float s = 0.f;
        for (int k = 0; k < slots; ++k) s += sh[k * G + gg][q];
        partial[(size_t)blockIdx.x * 8 * G + tid] = s;
    }
}

__global__ void bias_grad_reduce_kernel(const float* __restrict__ partial, int nblk, int C, int cout,
                                        float* __restrict__ db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cout) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * C + c];
    db[c] = s;
}

// ---------------------------------------------------------------------------
// 2x average pooling of channels-last bf16 volumes and its adjoint.
// The adjoint adds (g / 8) * lrelu'(x) into gx at each of the 8 children
// (x = the pooled activation, whose pre-activation gradient this is).
__global__ void pool2_kernel(const bf16* __restrict__ x, int xs, bf16* __restrict__ y, int ys, int C, int B, int D,
                             int H, int W)
{
    const int Do = D / 2, Ho = H / 2, Wo = W / 2;
    const long long n = (long long)B * Do * Ho * Wo * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long v = e / C;
        const int xo = (int)(v % Wo), yo = (int)((v / Wo) % Ho), zo = (int)((v / ((long long)Wo * Ho)) % Do);
        const long long b = v / ((long long)Wo * Ho * Do);
        float s = 0.f;
        for (int q = 0; q < 8; ++q) {
            const long long iv = ((b * D + 2 * zo + (q >> 2)) * H + 2 * yo + ((q >> 1) & 1)) * W + 2 * xo + (q & 1);
            s += __bfloat162float(x[iv * xs + c]);
        }
        y[v * ys + c] = __float2bfloat16(0.125f * s);
    }
}

__global__ void pool2_adjoint_kernel(const bf16* __restrict__ gy, int gys, const bf16* __restrict__ x, int xs,
                                     bf16* __restrict__ gx, int gxs, int C, float slope, int B, int D, int H, int W)
{
    const long long n = (long long)B * D * H * W * C;
    const int Ho = H / 2, Wo = W / 2, Do = D / 2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long v = e / C;
        const int xx = (int)(v % W), yy = (int)((v / W) % H), zz = (int)((v / ((long long)W * H)) % D);
        const long long b = v / ((long long)W * H * D);
        const long long ov = ((b * Do + zz / 2) * Ho + yy / 2) * Wo + xx / 2;
        const float g = 0.125f * __bfloat162float(gy[ov * gys + c]);
        const float act = __bfloat162float(x[v * xs + c]);
        const float add = act > 0.f ? g : slope * g;
        gx[v * gxs + c] = __float2bfloat16(__bfloat162float(gx[v * gxs + c]) + add);
    }
}

// nearest 2x upsampling into a channel slice, and its adjoint (sum of 8 children)
__global__ void up2_kernel(const bf16* __restrict__ x, int xs, bf16* __restrict__ y, int ys, int yoff, int C, int B,
                           int D, int H, int W)
{
    const long long n = (long long)B * D * H * W * C;      // D, H, W: output size
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long v = e / C;
        const int xx = (int)(v % W), yy = (int)((v / W) % H), zz = (int)((v / ((long long)W * H)) % D);
        const long long b = v / ((long long)W * H * D);
        const long long iv = ((b * (D / 2) + zz / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2;
        y[v * ys + yoff + c] = x[iv * xs + c];
    }
}

__global__ void up2_adjoint_kernel(const bf16* __restrict__ gy, int gys, int gyoff, bf16* __restrict__ gx, int gxs,
                                   int C, int B, int D, int H, int W)
{
    const int Do = D / 2, Ho = H / 2, Wo = W / 2;           // D, H, W: size of gy
    const long long n = (long long)B * Do * Ho * Wo * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long v = e / C;
        const int xo = (int)(v % Wo), yo = (int)((v / Wo) % Ho), zo = (int)((v / ((long long)Wo * Ho)) % Do);
        const long long b = v / ((long long)Wo * Ho * Do);
        float s = 0.f;
        for (int q = 0; q < 8; ++q) {
            const long long iv = ((b * D + 2 * zo + (q >> 2)) * H + 2 * yo + ((q >> 1) & 1)) * W + 2 * xo + (q & 1);
            s += __bfloat162float(gy[iv * gys + gyoff + c]);
        }
        gx[v * gxs + c] = __float2bfloat16(s);
    }
}

// network input: channel 0 = subject[b], channel 1 = atlas (shared), rest 0
__global__ void pack_input_kernel(const float* __restrict__ subj, const float* __restrict__ atlas, bf16* __restrict__ x,
                                  int xs, long long V, int B)
{
    const long long n = (long long)B * V;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        bf16* o = x + v * xs;
        o[0] = __float2bfloat16(subj[v]);
        o[1] = __float2bfloat16(atlas[v % V]);
        for (int c = 2; c < xs; ++c) o[c] = __float2bfloat16(0.f);
    }
}

// loss = mean over voxels and 3 channels of (pred - target)^2 (block partials),
// pred and target planar [batch][3][V], n = batch * V voxels;
// g (channels-last bf16, stride gs) = dloss/dpred, channels 3.. set to zero
__global__ void velocity_loss_kernel(const float* __restrict__ pred, const float* __restrict__ target, long long n,
                                     long long V, bf16* __restrict__ g, int gs, double* __restrict__ partials, float inv)
{
    __shared__ double sh[32];
    float acc = 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const long long b = v / V, l = v - b * V;
        for (int c = 0; c < 3; ++c) {
            const size_t e = ((size_t)b * 3 + c) * V + l;
            const float d = pred[e] - target[e];
            acc += d * d * inv;
            g[v * gs + c] = __float2bfloat16(2.f * d * inv);
        }
        for (int c = 3; c < gs; ++c) g[v * gs + c] = __float2bfloat16(0.f);
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// forward weights (bf16 [np][kp]) and the flipped, transposed weights of the
// data gradient (bf16 [npd][kpd], k' = tap' * coutp + co, tap' = 26 - tap)
__global__ void weight_prep_kernel(const float* __restrict__ w, int kp, int np, int cin, int cinp_real, int cout,
                                   int coutp, bf16* __restrict__ wb, bf16* __restrict__ wd, int kpd, int npd)
{
    const long long n = (long long)np * kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        wb[e] = __float2bfloat16(w[e]);
    const long long nd = (long long)npd * kpd;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nd; e += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(e / kpd), kd = (int)(e % kpd);
        const int tapd = kd / coutp, co = kd % coutp;
        float val = 0.f;
        if (tapd < 27 && co < cout && ci < cinp_real) val = w[(size_t)co * kp + (26 - tapd) * cin + ci];
        wd[e] = __float2bfloat16(val);
    }
}

// full-resolution velocity from the half-resolution one: trilinear
// interpolation at (x + 1/2)/2 - 1/2 (cell centres), values x 2 (the voxel
// unit halves)
__global__ void upsample_velocity_kernel(const float* __restrict__ vh, int Dh, int Hh, int Wh, float* __restrict__ v,
                                         int D, int H, int W, int B)
{
    const long long Vh = (long long)Dh * Hh * Wh, V = (long long)D * H * W;
    const long long n = (long long)B * 3 * V;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long l = e % V, bc = e / V;
        const int x = (int)(l % W), y = (int)((l / W) % H), z = (int)(l / ((long long)W * H));
        const float pz = fminf(fmaxf((z + 0.5f) * 0.5f - 0.5f, 0.f), (float)(Dh - 1));
        const float py = fminf(fmaxf((y + 0.5f) * 0.5f - 0.5f, 0.f), (float)(Hh - 1));
        const float px = fminf(fmaxf((x + 0.5f) * 0.5f - 0.5f, 0.f), (float)(Wh - 1));
        const int iz = min((int)pz, Dh - 2), iy = min((int)py, Hh - 2), ix = min((int)px, Wh - 2);
        const float tz = pz - iz, ty = py - iy, tx = px - ix;
        const float* f = vh + bc * Vh;
        auto at = [&](int a, int b2, int c) { return f[((long long)a * Hh + b2) * Wh + c]; };
        const float c00 = at(iz, iy, ix) + tx * (at(iz, iy, ix + 1) - at(iz, iy, ix));
        const float c01 = at(iz, iy + 1, ix) + tx * (at(iz, iy + 1, ix + 1) - at(iz, iy + 1, ix));
        const float c10 = at(iz + 1, iy, ix) + tx * (at(iz + 1, iy, ix + 1) - at(iz + 1, iy, ix));
        const float c11 = at(iz + 1, iy + 1, ix) + tx * (at(iz + 1, iy + 1, ix + 1) - at(iz + 1, iy + 1, ix));
        const float c0 = c00 + ty * (c01 - c00), c1 = c10 + ty * (c11 - c10);
        v[e] = 2.f * (c0 + tz * (c1 - c0));
    }
}

// half-resolution image: mean of each 2x2x2 block (fp32, planar)
__global__ void downsample_image_kernel(const float* __restrict__ I, int D, int H, int W, float* __restrict__ Ih, int B)
{
    const int Dh = D / 2, Hh = H / 2, Wh = W / 2;
    const long long Vh = (long long)Dh * Hh * Wh, V = (long long)D * H * W;
    const long long n = (long long)B * Vh;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long l = e % Vh, b = e / Vh;
        const int x = (int)(l % Wh), y = (int)((l / Wh) % Hh), z = (int)(l / ((long long)Wh * Hh));
        float s = 0.f;
        for (int q = 0; q < 8; ++q)
            s += I[b * V + ((long long)(2 * z + (q >> 2)) * H + 2 * y + ((q >> 1) & 1)) * W + 2 * x + (q & 1)];
        Ih[e] = 0.125f * s;
    }
}

int ew_grid(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16)); }

}  // namespace

cudaError_t gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, cudaStream_t s)
{
    const size_t smem = (size_t)TC_M * TC_KC * 2 + (size_t)N * TC_KC * 2;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(TC_M * TC_KC * 2 + 256 * TC_KC * 2));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    gemm_bf16_kernel<<<M / TC_M, 128, smem, s>>>(static_cast<const bf16*>(A), static_cast<const bf16*>(B), C, N, K);
    return cudaGetLastError();
}

cudaError_t conv3_forward(const ConvDesc& d, cudaStream_t s)
{
    ConvArgs a;
    a.in = static_cast<const bf16*>(d.in);
    a.in_stride = d.in_stride;
    a.cin = d.cin;
    a.wt = static_cast<const bf16*>(d.wt);
    a.bias = d.bias;
    a.out = static_cast<bf16*>(d.out);
    a.out_stride = d.out_stride;
    a.out_off = d.out_off;
    a.cout = d.cout;
    a.out_f32 = d.out_f32;
    a.gate = static_cast<const bf16*>(d.gate);
    a.gate_stride = d.gate_stride;
    a.act = d.act;
    a.slope = d.slope;
    a.D = d.D;
    a.H = d.H;
    a.W = d.W;
    a.nvox = (long long)d.batch * d.D * d.H * d.W;
    a.kp = d.kp;
    a.np = d.np;
    const size_t smem = 2 * ((size_t)CONV_SMEM_STAGE_A + (size_t)d.np * TC_KC * 2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             2 * (CONV_SMEM_STAGE_A + 256 * TC_KC * 2));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long blocks = (a.nvox + TC_M - 1) / TC_M;
    conv3_fwd_kernel<<<(unsigned)blocks, 128, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t conv3_wgrad(const void* in, int in_stride, int cin, const void* gz, int gz_stride, int cout, float* partial,
                        int splits, float* dw, int batch, int D, int H, int W, int kp, int np, cudaStream_t s)
{
    WgradArgs a;
    a.in = static_cast<const bf16*>(in);
    a.in_stride = in_stride;
    a.cin = cin;
    a.gz = static_cast<const bf16*>(gz);
    a.gz_stride = gz_stride;
    a.cout = cout;
    a.partial = partial;
    a.D = D;
    a.H = H;
    a.W = W;
    a.nvox = (long long)batch * D * H * W;
    a.chunk = ((a.nvox + splits - 1) / splits + TC_KC - 1) / TC_KC * TC_KC;
    a.kp = kp;
    a.np = np;
    const size_t smem = 2 * ((size_t)CONV_SMEM_STAGE_A + (size_t)np * TC_KC * 2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             2 * (CONV_SMEM_STAGE_A + 128 * TC_KC * 2));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    conv3_wgrad_kernel<<<dim3((kp + TC_M - 1) / TC_M, splits), 128, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    conv3_wgrad_reduce_kernel<<<ew_grid((long long)kp * np), 256, 0, s>>>(partial, splits, kp, np, dw);
    return cudaGetLastError();
}

int bias_grad_work_floats(int cout) { return BG_BLOCKS * ((cout + 7) / 8) * 8; }

cudaError_t bias_grad(const void* gz, int stride, long long nvox, int cout, float* db, float* work, cudaStream_t s)
{
    const int G = (cout + 7) / 8;                 // 1, 2, 4, 8 or 16 (checked by the caller)
    bias_grad_kernel<<<BG_BLOCKS, 256, 0, s>>>(static_cast<const bf16*>(gz), stride, nvox, G, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bias_grad_reduce_kernel<<<(cout + 127) / 128, 128, 0, s>>>(work, BG_BLOCKS, 8 * G, cout, db);
    return cudaGetLastError();
}

cudaError_t pool2(const void* x, int xs, void* y, int ys, int C, int B, int D, int H, int W, cudaStream_t s)
{
    pool2_kernel<<<ew_grid((long long)B * (D / 2) * (H / 2) * (W / 2) * C), 256, 0, s>>>(
        static_cast<const bf16*>(x), xs, static_cast<bf16*>(y), ys, C, B, D, H, W);
    return cudaGetLastError();
}

cudaError_t pool2_adjoint(const void* gy, int gys, const void* x, int xs, void* gx, int gxs, int C, float slope, int B,
                          int D, int H, int W, cudaStream_t s)
{
    pool2_adjoint_kernel<<<ew_grid((long long)B * D * H * W * C), 256, 0, s>>>(
        static_cast<const bf16*>(gy), gys, static_cast<const bf16*>(x), xs, static_cast<bf16*>(gx), gxs, C, slope, B,
        D, H, W);
    return cudaGetLastError();
}

cudaError_t up2(const void* x, int xs, void* y, int ys, int yoff, int C, int B, int D, int H, int W, cudaStream_t s)
{
    up2_kernel<<<ew_grid((long long)B * D * H * W * C), 256, 0, s>>>(static_cast<const bf16*>(x), xs,
                                                                      static_cast<bf16*>(y), ys, yoff, C, B, D, H, W);
    return cudaGetLastError();
}

cudaError_t up2_adjoint(const void* gy, int gys, int gyoff, void* gx, int gxs, int C, int B, int D, int H, int W,
                        cudaStream_t s)
{
    up2_adjoint_kernel<<<ew_grid((long long)B * (D / 2) * (H / 2) * (W / 2) * C), 256, 0, s>>>(
        static_cast<const bf16*>(gy), gys, gyoff, static_cast<bf16*>(gx), gxs, C, B, D, H, W);
    return cudaGetLastError();
}

cudaError_t pack_input(const float* subj, const float* atlas, void* x, int xs, long long V, int B, cudaStream_t s)
{
    pack_input_kernel<<<ew_grid((long long)B * V), 256, 0, s>>>(subj, atlas, static_cast<bf16*>(x), xs, V, B);
    return cudaGetLastError();
}

int velocity_loss_blocks(long long n) { return ew_grid(n); }

cudaError_t velocity_loss(const float* pred, const float* target, long long n, long long V, void* g, int gs,
                          double* partials, cudaStream_t s)
{
    velocity_loss_kernel<<<ew_grid(n), 256, 0, s>>>(pred, target, n, V, static_cast<bf16*>(g), gs, partials,
                                                    (float)(1.0 / (3.0 * (double)n)));
    return cudaGetLastError();
}

cudaError_t weight_prep(const float* w, int kp, int np, int cin, int cin_real, int cout, int coutp, void* wb, void* wd,
                        int kpd, int npd, cudaStream_t s)
{
    weight_prep_kernel<<<ew_grid(std::max((long long)np * kp, (long long)npd * kpd)), 256, 0, s>>>(
        w, kp, np, cin, cin_real, cout, coutp, static_cast<bf16*>(wb), static_cast<bf16*>(wd), kpd, npd);
    return cudaGetLastError();
}

cudaError_t upsample_velocity(const float* vh, int Dh, int Hh, int Wh, float* v, int D, int H, int W, int B,
                              cudaStream_t s)
{
    upsample_velocity_kernel<<<ew_grid((long long)B * 3 * D * H * W), 256, 0, s>>>(vh, Dh, Hh, Wh, v, D, H, W, B);
    return cudaGetLastError();
}

cudaError_t downsample_image(const float* I, int D, int H, int W, float* Ih, int B, cudaStream_t s)
{
    downsample_image_kernel<<<ew_grid((long long)B * (D / 2) * (H / 2) * (W / 2)), 256, 0, s>>>(I, D, H, W, Ih, B);
    return cudaGetLastError();
}

}  // namespace darc_impl
