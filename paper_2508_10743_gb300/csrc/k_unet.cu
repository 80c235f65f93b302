// k_unet.cu -- BF16 tensor-core (tcgen05, TMEM) kernels for the learned
// warm start: a dense GEMM core and the 3-D convolutions of the U-Net
// (forward and data gradient by one kernel, weight gradient by another).
//
// Activations are channels-last bf16 volumes stored with a one-voxel zero
// border ([batch][D+2][H+2][W+2][stride]).  In the flattened padded index a
// 3x3x3 tap is a constant row shift, (dz-1) P + (dy-1) (W+2) + (dx-1) with
// P = (H+2)(W+2), so the convolution of 128 consecutive padded rows reads,
// for each dz, one contiguous window of 128 + 2 (W+2) + 2 rows, and the nine
// (dy, dx) taps are the same window seen from nine start rows.  In the
// no-swizzle K-major layout the rows of a window are 16 bytes apart, so a
// tap is a shared-memory descriptor whose start address moves by 16 bytes a
// row: one staged window feeds nine MMAs.  Border rows of the output are
// computed and discarded; the borders of every buffer stay zero.
#include "kernels.h"
#include "umma.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>

namespace darc_impl {
namespace {

using bf16 = __nv_bfloat16;
constexpr int TC_M = 128;            // rows of a CTA tile (TMEM lanes)
constexpr int TC_KC = 64;            // K elements staged per round (4 MMAs of K = 16)
constexpr long long TC_WAIT = 1LL << 26;
constexpr int CONV_SMEM_MAX = 225 * 1024;      // dynamic; the static mbarriers and TMEM slot take the rest of 227 KB

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 :: "r"(umma::smem_u32(dst_smem)), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// padded row of interior voxel (z, y, x)
__device__ __forceinline__ long long pad_row(const PadVol& g, int z, int y, int x)
{
    return ((long long)(z + 1) * g.Hp + (y + 1)) * g.Wp + (x + 1);
}

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
// 3x3x3 'same' convolution on the tensor cores (forward, and the data
// gradient when run on dL/dz with flipped weights):
//   out[q][co] = act( bias[co] + sum_{tap, ci} in[q + off(tap)][ci] W[co][tap][ci] )
// A CTA owns 128 consecutive padded rows q (TMEM lanes) x np output channels
// (TMEM columns).  Stage (c, dz), c = 16-channel chunk: the dz window of the
// chunk and the chunk's nine (dy, dx) weight tiles.  One thread runs the
// whole main loop: it copies a stage with TMA (the window as 2 channel
// groups x `parts` boxes of 8 channels x BR rows of a 2-D tensor map over
// the padded rows, zero-filled outside the batch; the weight tiles with one
// bulk copy), waits for the stage's bytes on the slot's `full` barrier,
// issues nine M128 x N x K16 MMAs whose A descriptors start (dy (W+2) + dx)
// rows into the window, and commits them to the slot's `empty` barrier,
// which gates the slot's refill.  The other threads wait at a block barrier
// and then for the last commit, and run the epilogue.  Waits are bounded: a
// timeout poisons the output with NaN instead of hanging.
// pipeline slots of the window convolution: 2 = two (more resident blocks:
// a block runs only 3 x cin/16 stages, and the blocks of an SM hide each
// other's latencies better than a deeper pipeline does), 0 = three where
// they fit in 200 KB
#ifndef DARC_CONV_NS
#define DARC_CONV_NS 2
#endif

struct WinArgs {
    const bf16* in;
    int in_stride, nchunk;        // channels [0, 16 nchunk) read
    const bf16* wt;               // packed [nchunk][3][9][2][np][8]
    const float* bias;            // [cout] or null
    bf16* out;
    int out_stride, cout, out_vec;
    float* out_f32;               // planar [batch][cout][D H W] (replaces out)
    const bf16* gate;             // x slope where gate <= 0 (same geometry), or null
    int gate_stride;
    int act;                      // 1: leaky ReLU
    float slope;
    int B;
    PadVol g;
    int np, R, ns, slot_bytes;
    int parts, br;                // R = parts x br window rows per channel group (br <= 256, a multiple of 8)
    int mt;                       // 128-row sub-tiles a block owns (1 or 2), one TMEM accumulator each
    long long tiles_per_batch;    // of mt x 128 rows
};

template <int MT>
__global__ void __launch_bounds__(128)
conv3_win_kernel(const __grid_constant__ CUtensorMap tmap, WinArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t full[3], empty[3];
    __shared__ uint32_t tslot;
    __shared__ int bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const PadVol g = a.g;
    const int b = (int)(blockIdx.x / a.tiles_per_batch);
    const long long q0 = g.P + (long long)(blockIdx.x % a.tiles_per_batch) * TC_M * MT;
    const long long base_b = (long long)b * g.Vp;
    uint32_t ncols = 32;
    while ((int)ncols < a.np) ncols <<= 1;
    if (warp == 0) umma::tmem_alloc(&tslot, ncols * (uint32_t)MT);
    if (tid == 0) {
        for (int k = 0; k < a.ns; ++k) {
            umma::mbar_init(&full[k], 1);
            umma::mbar_init(&empty[k], 1);
        }
        bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tslot;
    const int nst = 3 * a.nchunk;

    if (tid == 0) {
        const uint32_t idesc = umma::idesc_bf16_f32(TC_M, a.np);
        const uint32_t lboA = (uint32_t)a.R * 16u, lboB = (uint32_t)a.np * 16u;
        const uint32_t wbytes = 288u * (uint32_t)a.np, tx = 32u * (uint32_t)a.R + wbytes;
        auto issue = [&](int st, int slot) {
            const int c = st / 3, dz = st - 3 * c;
            uint8_t* As = smem + (size_t)slot * a.slot_bytes;
            // first window row; negative or past the last batch at the ends (zero fill)
            const int r0 = (int)(base_b + q0 + (long long)(dz - 1) * g.P - g.Wp - 1);
            umma::mbar_arrive_expect_tx(&full[slot], tx);
            for (int grp = 0; grp < 2; ++grp)
                for (int p = 0; p < a.parts; ++p)
                    umma::tma_load_2d(As + grp * lboA + (uint32_t)p * a.br * 16u, &tmap, 16 * c + 8 * grp,
                                      r0 + p * a.br, &full[slot]);
            umma::bulk_load(As + 2 * lboA, a.wt + (size_t)(c * 3 + dz) * 18 * a.np * 8, wbytes, &full[slot]);
        };
        bool ok = true;
        for (int p = 0; p < a.ns && p < nst; ++p) issue(p, p);
        for (int i = 0; i < nst; ++i) {
            const int slot = i % a.ns;
            ok = umma::mbar_wait(&full[slot], (uint32_t)((i / a.ns) & 1), TC_WAIT) && ok;
            umma::fence_after_sync();
            const uint32_t As = umma::smem_u32(smem + (size_t)slot * a.slot_bytes);
            const uint32_t Bs = As + 2 * lboA;
            for (int t9 = 0; t9 < 9; ++t9) {
                const int dy = t9 / 3, dx = t9 - 3 * dy;
                const uint64_t db = umma::smem_desc(Bs + (uint32_t)t9 * 2u * lboB, lboB, 128);
                // sub-tile h reads the window 128 h rows further on, into accumulator h
#pragma unroll
                for (int h = 0; h < MT; ++h) {
                    const uint32_t row = (uint32_t)(dy * g.Wp + dx + TC_M * h);
                    const uint64_t da = umma::smem_desc(As + row * 16u, lboA, 128);
                    umma::mma_bf16(tmem + (uint32_t)h * ncols, da, db, idesc, (i > 0) || (t9 > 0));
                }
            }
            umma::commit(&empty[slot]);
            // refill the previous stage's slot once its MMAs (queued before these) retire
            const int k = i - 1;
            if (k >= 0 && k + a.ns < nst) {
                const int sk = k % a.ns;
                ok = umma::mbar_wait(&empty[sk], (uint32_t)((k / a.ns) & 1), TC_WAIT) && ok;
                issue(k + a.ns, sk);
            }
        }
        if (!ok) bad = 1;
    }
    __syncthreads();
    const bool ok = umma::mbar_wait(&empty[(nst - 1) % a.ns], (uint32_t)(((nst - 1) / a.ns) & 1), TC_WAIT) && !bad;
    umma::fence_after_sync();

    // epilogue: warp w holds rows q0 + 128 h + 32 w + lane of sub-tile h
    for (int h = 0; h < MT; ++h) {
    const long long q = q0 + TC_M * h + 32 * warp + lane;
    const int xp = (int)(q % g.Wp), yp = (int)((q / g.Wp) % g.Hp);
    const long long zp = q / g.P;
    const bool valid = zp <= g.D && yp >= 1 && yp <= g.H && xp >= 1 && xp <= g.W;
    const long long orow = base_b + q;
    const long long V = (long long)g.D * g.H * g.W;
    const long long l = ((zp - 1) * g.H + (yp - 1)) * (long long)g.W + (xp - 1);
    for (int c = 0; c < a.np; c += 8) {
        float r8[8];
        umma::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)h * ncols + (uint32_t)c, r8);
        if (!valid || c >= a.cout) continue;
        float y8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int co = c + j;
            float y = ok ? r8[j] : __int_as_float(0x7fc00000);
            if (co < a.cout) {
                if (a.bias) y += __ldg(a.bias + co);
                if (a.act == 1) y = y > 0.f ? y : a.slope * y;
                if (a.gate) {
                    const float gt = __bfloat162float(a.gate[orow * a.gate_stride + co]);
                    y = gt > 0.f ? y : a.slope * y;
                }
            }
            y8[j] = y;
        }
        if (a.out_f32) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (c + j < a.cout) a.out_f32[((size_t)b * a.cout + c + j) * V + l] = y8[j];
        } else if (a.out_vec && c + 8 <= a.cout) {
            uint4 pk;
            __nv_bfloat162* hp = reinterpret_cast<__nv_bfloat162*>(&pk);
#pragma unroll
            for (int j = 0; j < 4; ++j) hp[j] = __floats2bfloat162_rn(y8[2 * j], y8[2 * j + 1]);
            *reinterpret_cast<uint4*>(a.out + orow * a.out_stride + c) = pk;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (c + j < a.cout) a.out[orow * a.out_stride + c + j] = __float2bfloat16(y8[j]);
        }
    }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, ncols * (uint32_t)MT);
}

// packed[(((c 3 + dz) 9 + t9) 2 + grp) nrows + row] [e], tap = 9 dz + t9,
// channel ch = 16 c + 8 grp + e of the convolution's input:
//   forward (flip 0): row = output channel, W[row][tap][ch]
//   data gradient (flip 1): row = input channel of the layer, ch = its output
//   channel, W[ch][26 - tap][row]  (the transpose of the mirrored kernel)
// from fp32 masters w[co][k], k = tap cin + ci; zero outside cout / cin.
__global__ void pack_weights_kernel(const float* __restrict__ w, int kp, int cin, int cout, int nchunk, int nrows,
                                    int flip, bf16* __restrict__ out)
{
    const long long n = (long long)nchunk * 54 * nrows * 8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int e8 = (int)(e % 8);
        long long rest = e / 8;
        const int row = (int)(rest % nrows);
        rest /= nrows;
        const int grp = (int)(rest % 2);
        rest /= 2;
        const int t9 = (int)(rest % 9);
        rest /= 9;
        const int dz = (int)(rest % 3);
        const int c = (int)(rest / 3);
        const int tap = 9 * dz + t9, ch = 16 * c + 8 * grp + e8;
        float val = 0.f;
        if (!flip) {
            if (row < cout && ch < cin) val = w[(size_t)row * kp + tap * cin + ch];
        } else {
            if (ch < cout && row < cin) val = w[(size_t)ch * kp + (26 - tap) * cin + row];
        }
        out[e] = __float2bfloat16(val);
    }
}

// ---------------------------------------------------------------------------
// Weight gradient as a GEMM over the padded rows of the interior planes,
// gathered per (tap, channel) row (used when a call has fewer splits than
// batches; conv3_wgrad_win_kernel below is the fast path):
//   dW[co][k] = sum_q gz[q][co] in[q + off(tap)][ci],  k = tap cin + ci.
// Rows (TMEM lanes) are k in tiles of 128, columns co (np <= 128), K runs
// over a CTA's range of rows.  Border rows contribute zero (gz is zero
// there); their shifted reads can leave the buffer (the first border rows
// of batch 0, the last of the last batch), so those are not made.
// Operands are stored row-major by voxel, so they are transposed while
// staging (one 16-byte load gives 8 k-rows of one K column).  Each CTA
// writes its partial sums; conv3_wgrad_reduce adds them in a fixed order.
struct WgradArgs {
    const bf16* in;
    int in_stride, cin;
    const bf16* gz;             // gradient wrt the pre-activation, same geometry
    int gz_stride, cout;        // cout % 8 == 0 channels read
    float* partial;             // [splits][kp][np]
    PadVol g;
    long long nrows, chunk;     // K extent (batch x D x P) and rows per split (multiple of 64)
    long long rows_total;       // batch x Vp: rows of the buffers
    int kp, np;
};

__global__ void __launch_bounds__(128)
conv3_wgrad_kernel(WgradArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const PadVol g = a.g;
    const int r0 = blockIdx.x * TC_M;                       // first k row of this tile
    const long long v0 = (long long)blockIdx.y * a.chunk;
    const long long v1 = min(a.nrows, v0 + a.chunk);
    const int stageA = TC_M * TC_KC * 2, stageB = a.np * TC_KC * 2;
    uint8_t* sA[2] = {smem, smem + stageA + stageB};
    uint8_t* sB[2] = {smem + stageA, smem + 2 * stageA + stageB};
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
    const long long DP = (long long)g.D * g.P;
    bool ok = true;
    const int steps = (int)((v1 - v0 + TC_KC - 1) / TC_KC);
    for (int i = 0; i < steps; ++i) {
        const int st = i & 1;
        if (i >= 2) ok = umma::mbar_wait(&mbar[st], ((i - 2) >> 1) & 1, TC_WAIT) && ok;
        const long long vb = v0 + (long long)i * TC_KC;
        bf16* A16 = reinterpret_cast<bf16*>(sA[st]);
        bf16* B16 = reinterpret_cast<bf16*>(sB[st]);
        // A: 64 rows x 16 groups of 8 k-rows, transposed into K-major
        for (int e = tid; e < TC_KC * (TC_M / 8); e += 128) {
            const int j = e % TC_KC, mg = e / TC_KC;
            const int k = r0 + 8 * mg;
            const int tap = k / a.cin, ci = k - tap * a.cin;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            const long long v = vb + j;
            if (tap < 27 && k < a.kp && v < v1) {
                const long long row = (v / DP) * g.Vp + g.P + v % DP;
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                const long long src = row + (long long)(dz - 1) * g.P + (long long)(dy - 1) * g.Wp + (dx - 1);
                if (src >= 0 && src < a.rows_total) val = *reinterpret_cast<const uint4*>(a.in + src * a.in_stride + ci);
            }
            const bf16* pv = reinterpret_cast<const bf16*>(&val);
#pragma unroll
            for (int q = 0; q < 8; ++q) A16[umma::kmajor_offset(8 * mg + q, j, lboA) >> 1] = pv[q];
        }
        // B: 64 rows x (np / 8) groups of 8 output channels
        for (int e = tid; e < TC_KC * (a.np / 8); e += 128) {
            const int j = e % TC_KC, cg = e / TC_KC;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            const long long v = vb + j;
            if (v < v1 && 8 * cg < a.cout) {
                const long long row = (v / DP) * g.Vp + g.P + v % DP;
                val = *reinterpret_cast<const uint4*>(a.gz + row * a.gz_stride + 8 * cg);
            }
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

// ---------------------------------------------------------------------------
// Weight gradient on staged windows.  For a fixed (dz, dy) the three dx taps
// read the input at row q + off(dz, dy) + dx - 1, so one window of Kc + 2
// input rows serves all three: a CTA owns (dz, dy), a tile of up to 128
// input channels (TMEM lanes) and a range of rows of one batch (the K
// dimension), and keeps three accumulators of np columns, one per dx.
// Both operands are staged in the no-swizzle MN-major layout -- each
// 16-byte unit holds 8 consecutive channels of one row, the rows of one
// 8-channel group follow each other 16 bytes apart -- which is the
// channels-last storage itself, so nothing is transposed; the dx tap is a
// descriptor whose start moves by dx rows.  In MN-major no-swizzle
// descriptors the leading offset is the distance between 8-row K groups
// (128 bytes here) and the stride offset the distance between 8-channel
// groups (checked on the GPU against the oracle's weight gradient).
#ifndef DARC_WG_KC
#define DARC_WG_KC 64
#endif
#ifndef DARC_WGRAD_NS
#define DARC_WGRAD_NS 0
#endif
constexpr int WG_KC = DARC_WG_KC;         // rows (K) per stage
constexpr int WG_RA = WG_KC + 2;          // input window rows per stage

// (tap pair, channel group) items a CTA stacks where cin <= 64: the 9 cin/8
// items over as few CTAs as 16 lane groups allow, evened out (16 channels:
// 9 + 9 items; 48 channels: 14 + 14 + 14 + 12); 0 above (a pair a CTA)
int wgrad_items(int cin)
{
    if (cin > 64) return 0;
    const int total = 9 * std::max(cin / 8, 1), ctas = (total + 15) / 16;
    return (total + ctas - 1) / ctas;
}

// With few input channels most of the 128 lanes would idle, so a CTA then
// stacks (dz, dy) pairs in the M dimension: the 9 ng items (tap pair 3 dz +
// dy, 8-channel group) are dealt out evenly, `items` consecutive ones a
// CTA (lane row = (item within the CTA, channel within its group)), each
// staged from its pair's own shifted window.  The dx taps shift all of
// them alike.
struct WgradWinArgs {
    const bf16* in;
    int in_stride, cin;                   // cin % 16 == 0
    const bf16* gz;
    int gz_stride, cout;                  // cout % 8 == 0 channels read
    float* partial;                       // [B * sp][kp][np]
    PadVol g;
    int B, sp;                            // splits per batch
    long long chunk;                      // rows per split (multiple of WG_KC)
    int kp, np, ns, slot_bytes;
    int items;                            // (pair, group) items per CTA (cin <= 64), or 0: one pair a CTA
};

__global__ void __launch_bounds__(128)
conv3_wgrad_win_kernel(WgradWinArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mbar[3];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const PadVol g = a.g;
    const int c0 = blockIdx.y * TC_M, nci = min(TC_M, a.cin - c0), ng = nci / 8;
    const int per = a.items ? a.items : ng;
    const int item0 = blockIdx.x * per, used = min(per, 9 * ng - item0);   // 8-lane groups in use (<= 16)
    const int b = blockIdx.z / a.sp, spi = blockIdx.z - b * a.sp;
    const long long DP = (long long)g.D * g.P;
    const long long r0 = (long long)spi * a.chunk, r1 = min(DP, r0 + a.chunk);
    const long long base = (long long)b * g.Vp + g.P;            // padded row of interior row 0 of batch b
    const long long rows_total = (long long)a.B * g.Vp;
    const int steps = r1 > r0 ? (int)((r1 - r0 + WG_KC - 1) / WG_KC) : 0;
    const uint32_t strideA = (uint32_t)WG_RA * 16u, strideB = (uint32_t)WG_KC * 16u;
    const int bytesA = 16 * WG_RA * 16;                           // 16 channel groups (M = 128)
    uint32_t ncols = 32;
    while ((int)ncols < 3 * a.np) ncols <<= 1;
    // lane groups the tile does not use stay zero in every slot
    for (int e = tid; e < a.ns * (16 - used) * WG_RA; e += 128) {
        const int slot = e / ((16 - used) * WG_RA), rest = e - slot * (16 - used) * WG_RA;
        const int gi = used + rest / WG_RA, r = rest % WG_RA;
        *reinterpret_cast<uint4*>(smem + (size_t)slot * a.slot_bytes + gi * strideA + r * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) umma::tmem_alloc(&tslot, ncols);
    if (tid == 0) {
        for (int k = 0; k < a.ns; ++k) umma::mbar_init(&mbar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t idesc = umma::idesc_bf16_f32_mn(TC_M, a.np);

    // this thread's A copies of every stage (fixed over the stages but for
    // the stage's first row): shared-memory offset, row offset of its
    // window row from the stage's first row, channel offset
    constexpr int WG_AMAX = (16 * WG_RA + 127) / 128;
    int a_sm[WG_AMAX], a_row[WG_AMAX], a_ch[WG_AMAX];
    const int na = (used * WG_RA - tid + 127) / 128;
#pragma unroll
    for (int i = 0; i < WG_AMAX; ++i) {
        const int e = tid + 128 * i;
        const int grp = e / WG_RA, r = e - grp * WG_RA;
        const int item = item0 + grp, pr = item / ng, gi = item - pr * ng;   // tap pair 3 dz + dy, group
        a_sm[i] = grp * (int)strideA + r * 16;
        a_row[i] = (pr / 3 - 1) * (int)g.P + (pr % 3 - 1) * g.Wp - 1 + r;   // window row r (dx = 0 at r = 0)
        a_ch[i] = c0 + 8 * gi;
    }
    auto load = [&](int st, int slot) {
        uint8_t* As = smem + (size_t)slot * a.slot_bytes;
        uint8_t* Bs = As + bytesA;
        const long long k0 = r0 + (long long)st * WG_KC;
#pragma unroll
        for (int i = 0; i < WG_AMAX; ++i) {
            if (i >= na) break;
            const long long q = base + k0 + a_row[i];
            const bool ok = q >= 0 && q < rows_total;
            const bf16* src = ok ? a.in + q * a.in_stride + a_ch[i] : a.in;
            cp_async16(As + a_sm[i], src, ok ? 16 : 0);
        }
        for (int e = tid; e < (a.np / 8) * WG_KC; e += 128) {
            const int go = e / WG_KC, r = e - go * WG_KC;
            const bool ok = k0 + r < r1 && 8 * go < a.cout;
            const bf16* src = ok ? a.gz + (base + k0 + r) * a.gz_stride + 8 * go : a.gz;
            cp_async16(Bs + go * strideB + r * 16, src, ok ? 16 : 0);
        }
    };

    for (int p = 0; p < a.ns - 1; ++p) {
        if (p < steps) load(p, p);
        cp_async_commit();
    }
    bool ok = true;
    for (int i = 0; i < steps; ++i) {
        const int j = i + a.ns - 1;
        if (j < steps) {
            const int sj = j % a.ns;
            if (j >= a.ns) ok = umma::mbar_wait(&mbar[sj], (uint32_t)(((j - a.ns) / a.ns) & 1), TC_WAIT) && ok;
            load(j, sj);
        }
        cp_async_commit();
        if (a.ns == 3) cp_async_wait<2>();
        else cp_async_wait<1>();
        umma::fence_smem_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            const uint32_t As = umma::smem_u32(smem + (size_t)(i % a.ns) * a.slot_bytes);
            const uint32_t Bs = As + bytesA;
            for (int dx = 0; dx < 3; ++dx)
                for (int kq = 0; kq < WG_KC / 16; ++kq) {
                    const uint32_t sa = As + (uint32_t)(dx + 16 * kq) * 16u, sb = Bs + (uint32_t)(16 * kq) * 16u;
                    const uint64_t da = umma::smem_desc(sa, 128, strideA);
                    const uint64_t db = umma::smem_desc(sb, 128, strideB);
                    umma::mma_bf16(tmem + (uint32_t)(dx * a.np), da, db, idesc, (i > 0) || (kq > 0));
                }
            umma::commit(&mbar[i % a.ns]);
        }
    }
    if (steps > 0) ok = umma::mbar_wait(&mbar[(steps - 1) % a.ns], (uint32_t)(((steps - 1) / a.ns) & 1), TC_WAIT) && ok;
    umma::fence_after_sync();
    // epilogue: lane m = 32 w + lane is channel m % 8 of the CTA's item m / 8;
    // columns dx * np + co
    const int m = 32 * warp + lane, item = item0 + m / 8, pr = item / ng;
    const int ci = c0 + 8 * (item - pr * ng) + m % 8;
    for (int dx = 0; dx < 3; ++dx) {
        const int tap = 3 * pr + dx;                             // 9 dz + 3 dy + dx
        float* out = a.partial + ((size_t)blockIdx.z * a.kp + (size_t)tap * a.cin + ci) * a.np;
        for (int c = 0; c < a.np; c += 8) {
            float r8[8];
            umma::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(dx * a.np + c), r8);
            if (m < 8 * used) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    out[c + q] = (steps > 0 && ok) ? r8[q] : (ok ? 0.f : __int_as_float(0x7fc00000));
            }
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

// one warp per channel: lane j adds rows j, j + 32, ..., then a fixed
// shuffle tree (deterministic)
__global__ void bias_grad_reduce_kernel(const float* __restrict__ partial, int nblk, int C, int cout,
                                        float* __restrict__ db)
{
    const int c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= cout) return;
    float s = 0.f;
    for (int b = lane; b < nblk; b += 32) s += partial[(size_t)b * C + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[c] = s;
}

// ---------------------------------------------------------------------------
// 2x average pooling of padded channels-last volumes and its adjoint (fine
// grid gf, coarse grid gc = gf / 2).  The adjoint adds (g / 8) lrelu'(x) into
// gx at each of the 8 children (x = the pooled activation, whose
// pre-activation gradient this is).  A thread takes 8 channels of one voxel
// (16-byte loads and stores: channel counts, strides and channel offsets are
// multiples of 8); blockIdx.y walks the (batch, plane) pairs of the grid
// the thread's voxel is on, so the index arithmetic stays in 32 bits.
__device__ __forceinline__ void bf8_to_f(const uint4& q, float f[8])
{
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 t = __bfloat1622float2(h[j]);
        f[2 * j] = t.x;
        f[2 * j + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 f_to_bf8(const float f[8])
{
    uint4 q;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
    return q;
}

// the voxel (b, z, y, x) and channel group c8 of this thread on grid g, or false
__device__ __forceinline__ bool vox8(const PadVol& g, int G, int bz, int& b, int& z, int& y, int& x, int& c8)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= g.H * g.W * G) return false;
    c8 = 8 * (e % G);
    const int t = e / G;
    x = t % g.W;
    y = t / g.W;
    b = bz / g.D;
    z = bz - b * g.D;
    return true;
}

__global__ void pool2_kernel(const bf16* __restrict__ x, int xs, bf16* __restrict__ y, int ys, int C, int B,
                             PadVol gf, PadVol gc)
{
    const int G = C / 8;
    for (int bz = blockIdx.y; bz < B * gc.D; bz += gridDim.y) {
        int b, zo, yo, xo, c8;
        if (!vox8(gc, G, bz, b, zo, yo, xo, c8)) return;
        float s[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long long iv = (long long)b * gf.Vp + pad_row(gf, 2 * zo + (q >> 2), 2 * yo + ((q >> 1) & 1),
                                                                 2 * xo + (q & 1));
            float f[8];
            bf8_to_f(*reinterpret_cast<const uint4*>(x + iv * xs + c8), f);
#pragma unroll
            for (int j = 0; j < 8; ++j) s[j] += f[j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] *= 0.125f;
        *reinterpret_cast<uint4*>(y + ((long long)b * gc.Vp + pad_row(gc, zo, yo, xo)) * ys + c8) = f_to_bf8(s);
    }
}

__global__ void pool2_adjoint_kernel(const bf16* __restrict__ gy, int gys, const bf16* __restrict__ x, int xs,
                                     bf16* __restrict__ gx, int gxs, int C, float slope, int B, PadVol gf, PadVol gc)
{
    const int G = C / 8;
    for (int bz = blockIdx.y; bz < B * gf.D; bz += gridDim.y) {
        int b, zz, yy, xx, c8;
        if (!vox8(gf, G, bz, b, zz, yy, xx, c8)) return;
        const long long ov = (long long)b * gc.Vp + pad_row(gc, zz / 2, yy / 2, xx / 2);
        const long long iv = (long long)b * gf.Vp + pad_row(gf, zz, yy, xx);
        float gv[8], act[8], cur[8];
        bf8_to_f(*reinterpret_cast<const uint4*>(gy + ov * gys + c8), gv);
        bf8_to_f(*reinterpret_cast<const uint4*>(x + iv * xs + c8), act);
        uint4* dst = reinterpret_cast<uint4*>(gx + iv * gxs + c8);
        bf8_to_f(*dst, cur);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float g8 = 0.125f * gv[j];
            cur[j] += act[j] > 0.f ? g8 : slope * g8;
        }
        *dst = f_to_bf8(cur);
    }
}

// nearest 2x upsampling into a channel slice, and its adjoint (sum of 8 children)
__global__ void up2_kernel(const bf16* __restrict__ x, int xs, bf16* __restrict__ y, int ys, int C, int B, PadVol gf,
                           PadVol gc)
{
    const int G = C / 8;
    for (int bz = blockIdx.y; bz < B * gf.D; bz += gridDim.y) {
        int b, zz, yy, xx, c8;
        if (!vox8(gf, G, bz, b, zz, yy, xx, c8)) return;
        *reinterpret_cast<uint4*>(y + ((long long)b * gf.Vp + pad_row(gf, zz, yy, xx)) * ys + c8) =
            *reinterpret_cast<const uint4*>(x + ((long long)b * gc.Vp + pad_row(gc, zz / 2, yy / 2, xx / 2)) * xs + c8);
    }
}

__global__ void up2_adjoint_kernel(const bf16* __restrict__ gy, int gys, bf16* __restrict__ gx, int gxs, int C, int B,
                                   PadVol gf, PadVol gc)
{
    const int G = C / 8;
    for (int bz = blockIdx.y; bz < B * gc.D; bz += gridDim.y) {
        int b, zo, yo, xo, c8;
        if (!vox8(gc, G, bz, b, zo, yo, xo, c8)) return;
        float s[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long long iv = (long long)b * gf.Vp + pad_row(gf, 2 * zo + (q >> 2), 2 * yo + ((q >> 1) & 1),
                                                                 2 * xo + (q & 1));
            float f[8];
            bf8_to_f(*reinterpret_cast<const uint4*>(gy + iv * gys + c8), f);
#pragma unroll
            for (int j = 0; j < 8; ++j) s[j] += f[j];
        }
        *reinterpret_cast<uint4*>(gx + ((long long)b * gc.Vp + pad_row(gc, zo, yo, xo)) * gxs + c8) = f_to_bf8(s);
    }
}

// network input (16 channels): 0 = subject[b], 1 = atlas (shared), rest 0
__global__ void pack_input_kernel(const float* __restrict__ subj, const float* __restrict__ atlas, bf16* __restrict__ x,
                                  PadVol g, int B)
{
    const long long V = (long long)g.D * g.H * g.W, n = (long long)B * V;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const long long b = v / V, l = v - b * V;
        const int xx = (int)(l % g.W), yy = (int)((l / g.W) % g.H), zz = (int)(l / ((long long)g.W * g.H));
        uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = make_uint4(0u, 0u, 0u, 0u);
        reinterpret_cast<__nv_bfloat162*>(&lo)[0] = __floats2bfloat162_rn(subj[v], atlas[l]);
        uint4* o = reinterpret_cast<uint4*>(x + (b * g.Vp + pad_row(g, zz, yy, xx)) * 16);
        o[0] = lo;
        o[1] = hi;
    }
}

// loss = mean over voxels and 3 channels of (pred - target)^2 (block partials),
// pred and target planar [batch][3][V]; g (padded channels-last bf16, stride
// gs) = dloss/dpred, channels 3.. set to zero
__global__ void velocity_loss_kernel(const float* __restrict__ pred, const float* __restrict__ target, int B, PadVol g,
                                     bf16* __restrict__ gout, int gs, double* __restrict__ partials, float inv)
{
    __shared__ double sh[32];
    const long long V = (long long)g.D * g.H * g.W, n = (long long)B * V;
    float acc = 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const long long b = v / V, l = v - b * V;
        const int xx = (int)(l % g.W), yy = (int)((l / g.W) % g.H), zz = (int)(l / ((long long)g.W * g.H));
        uint4* o = reinterpret_cast<uint4*>(gout + (b * g.Vp + pad_row(g, zz, yy, xx)) * gs);
        float gv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < 3; ++c) {
            const size_t e = ((size_t)b * 3 + c) * V + l;
            const float d = pred[e] - target[e];
            acc += d * d * inv;
            gv[c] = 2.f * d * inv;
        }
        o[0] = f_to_bf8(gv);
        for (int c = 8; c < gs; c += 8) o[c / 8] = make_uint4(0u, 0u, 0u, 0u);
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
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

}  // namespace

static int ew_grid(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16)); }

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


PadVol make_pad(int D, int H, int W)
{
    PadVol g;
    g.D = D;
    g.H = H;
    g.W = W;
    g.Wp = W + 2;
    g.Hp = H + 2;
    g.P = (long long)g.Hp * g.Wp;
    g.Vp = (long long)(D + 2) * g.P;
    return g;
}

// window rows a stage needs, split into parts of br <= 256 rows (a TMA box
// dimension), br a multiple of 8 (128-byte aligned boxes)
static void conv_window_split(int W, int mt, int& parts, int& br)
{
    const int need = TC_M * mt + 2 * (W + 2) + 2;
    parts = (need + 255) / 256;
    br = ((need + parts - 1) / parts + 7) / 8 * 8;
}

// 128-row sub-tiles a block owns: two (one window for 256 rows: 1.9 staged
// rows an output row instead of 2.9 at W = 112) where their two
// accumulators leave TMEM for the resident blocks (np <= 64) and the grid
// still has many blocks an SM (large volumes); else one
static int conv_mt_max(int np) { return np <= 64 ? 2 : 1; }
static int conv_mt(int np, long long rows) { return conv_mt_max(np) == 2 && rows / (2 * TC_M) >= 24 * 152 ? 2 : 1; }

int conv_window_rows(int W, int mt)
{
    int parts, br;
    conv_window_split(W, mt, parts, br);
    return parts * br;
}

static int conv_slot_bytes(int W, int np, int mt) { return (32 * conv_window_rows(W, mt) + 288 * np + 127) / 128 * 128; }

int conv_slot_bytes(int W, int np) { return conv_slot_bytes(W, np, conv_mt_max(np)); }

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}
}  // namespace

bool conv_fits(int W, int np) { return 2 * conv_slot_bytes(W, np) <= CONV_SMEM_MAX; }

cudaError_t conv3_forward(const ConvDesc& d, cudaStream_t s)
{
    WinArgs a;
    a.in = static_cast<const bf16*>(d.in);
    a.in_stride = d.in_stride;
    a.nchunk = d.cin / 16;
    a.wt = static_cast<const bf16*>(d.wt);
    a.bias = d.bias;
    a.out = static_cast<bf16*>(d.out);
    a.out_stride = d.out_stride;
    a.cout = d.cout;
    a.out_vec = (d.out_stride % 8 == 0) && ((reinterpret_cast<uintptr_t>(d.out) & 15) == 0);
    a.out_f32 = d.out_f32;
    a.gate = static_cast<const bf16*>(d.gate);
    a.gate_stride = d.gate_stride;
    a.act = d.act;
    a.slope = d.slope;
    a.B = d.batch;
    a.g = make_pad(d.D, d.H, d.W);
    a.np = d.np;
    a.mt = conv_mt(d.np, (long long)d.batch * d.D * a.g.P);
    conv_window_split(d.W, a.mt, a.parts, a.br);
    a.R = a.parts * a.br;
    a.slot_bytes = conv_slot_bytes(d.W, d.np, a.mt);
    a.ns = (DARC_CONV_NS == 2 || 3 * a.slot_bytes > 200 * 1024) ? 2 : 3;
    a.tiles_per_batch = ((long long)d.D * a.g.P + TC_M * a.mt - 1) / (TC_M * a.mt);
    if (!conv_fits(d.W, d.np)) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3_win_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             CONV_SMEM_MAX);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv3_win_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM_MAX);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // the input as rows x channels [0, cin): boxes of 8 channels x br rows
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    // TMA row coordinates are 32-bit
    if ((long long)d.batch * a.g.Vp + 2 * a.g.P >= (1LL << 31)) return cudaErrorInvalidValue;
    if (!encode || d.in_stride % 8 || (reinterpret_cast<uintptr_t>(d.in) & 15) ||
        (reinterpret_cast<uintptr_t>(d.wt) & 15))
        return cudaErrorInvalidValue;
    CUtensorMap tmap;
    const cuuint64_t gdim[2] = {(cuuint64_t)d.cin, (cuuint64_t)((long long)d.batch * a.g.Vp)};
    const cuuint64_t gstride[1] = {(cuuint64_t)d.in_stride * sizeof(bf16)};
    const cuuint32_t box[2] = {8u, (cuuint32_t)a.br}, estride[2] = {1u, 1u};
    if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(d.in), gdim, gstride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const long long blocks = (long long)d.batch * a.tiles_per_batch;
    if (a.mt == 2)
        conv3_win_kernel<2><<<(unsigned)blocks, 128, (size_t)a.ns * a.slot_bytes, s>>>(tmap, a);
    else
        conv3_win_kernel<1><<<(unsigned)blocks, 128, (size_t)a.ns * a.slot_bytes, s>>>(tmap, a);
    return cudaGetLastError();
}

size_t packed_weight_elems(int conv_cin, int nrows) { return (size_t)(conv_cin / 16) * 54 * nrows * 8; }

cudaError_t pack_weights(const float* w, int kp, int cin, int cout, int conv_cin, int nrows, int flip, void* out,
                         cudaStream_t s)
{
    const long long n = (long long)packed_weight_elems(conv_cin, nrows);
    pack_weights_kernel<<<ew_grid(n), 256, 0, s>>>(w, kp, cin, cout, conv_cin / 16, nrows, flip,
                                                    static_cast<bf16*>(out));
    return cudaGetLastError();
}

cudaError_t conv3_wgrad_gather(const void* in, int in_stride, int cin, const void* gz, int gz_stride, int cout,
                               float* partial, int splits, float* dw, int batch, int D, int H, int W, int kp, int np,
                               cudaStream_t s)
{
    WgradArgs a;
    a.in = static_cast<const bf16*>(in);
    a.in_stride = in_stride;
    a.cin = cin;
    a.gz = static_cast<const bf16*>(gz);
    a.gz_stride = gz_stride;
    a.cout = cout;
    a.partial = partial;
    a.g = make_pad(D, H, W);
    a.nrows = (long long)batch * D * a.g.P;
    a.rows_total = (long long)batch * a.g.Vp;
    a.chunk = ((a.nrows + splits - 1) / splits + TC_KC - 1) / TC_KC * TC_KC;
    a.kp = kp;
    a.np = np;
    const size_t smem = 2 * ((size_t)TC_M * TC_KC * 2 + (size_t)np * TC_KC * 2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             2 * (TC_M * TC_KC * 2 + 128 * TC_KC * 2));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    conv3_wgrad_kernel<<<dim3((kp + TC_M - 1) / TC_M, splits), 128, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    conv3_wgrad_reduce_kernel<<<ew_grid((long long)kp * np), 256, 0, s>>>(partial, splits, kp, np, dw);
    return cudaGetLastError();
}

// the window kernel: splits are taken per batch (a K range never crosses a
// batch), at most `splits` in all
cudaError_t conv3_wgrad_win(const void* in, int in_stride, int cin, const void* gz, int gz_stride, int cout,
                            float* partial, int splits, float* dw, int batch, int D, int H, int W, int kp, int np,
                            cudaStream_t s)
{
    WgradWinArgs a;
    a.in = static_cast<const bf16*>(in);
    a.in_stride = in_stride;
    a.cin = cin;
    a.gz = static_cast<const bf16*>(gz);
    a.gz_stride = gz_stride;
    a.cout = cout;
    a.partial = partial;
    a.g = make_pad(D, H, W);
    a.B = batch;
    a.sp = std::max(1, splits / batch);
    const long long DP = (long long)D * a.g.P;
    a.chunk = ((DP + a.sp - 1) / a.sp + WG_KC - 1) / WG_KC * WG_KC;
    a.kp = kp;
    a.np = np;
    a.slot_bytes = (16 * WG_RA * 16 + np * WG_KC * 2 + 127) / 128 * 128;
    a.ns = (DARC_WGRAD_NS == 2 || 3 * a.slot_bytes > 200 * 1024) ? 2 : 3;
    a.items = wgrad_items(cin);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3_wgrad_win_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             CONV_SMEM_MAX);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid(a.items ? (9 * (cin / 8) + a.items - 1) / a.items : 9, (cin + TC_M - 1) / TC_M, a.sp * batch);
    conv3_wgrad_win_kernel<<<grid, 128, (size_t)a.ns * a.slot_bytes, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    conv3_wgrad_reduce_kernel<<<ew_grid((long long)kp * np), 256, 0, s>>>(partial, a.sp * batch, kp, np, dw);
    return cudaGetLastError();
}

int wgrad_ctas_per_split(int cin)
{
    const int items = wgrad_items(cin);
    return items ? (9 * (cin / 8) + items - 1) / items : 9 * ((cin + TC_M - 1) / TC_M);
}

int wgrad_resident_ctas(int np)
{
    // blocks of the weight-gradient window kernel resident at once on the
    // device: a split-K grid of at most this many runs in one wave
    static int sms = 0, smem_sm = 0, smem_rsv = 0, regs = 0, smem_static = 0;
    if (!sms) {
        int dev = 0, n = 0;
        cudaFuncAttributes fa{};
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, conv3_wgrad_win_kernel) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            return 4 * 152;
        }
        regs = fa.numRegs;
        smem_static = (int)fa.sharedSizeBytes;
        sms = n;
    }
    const int slot = (16 * WG_RA * 16 + np * WG_KC * 2 + 127) / 128 * 128;
    const int ns = (DARC_WGRAD_NS == 2 || 3 * slot > 200 * 1024) ? 2 : 3;
    const int per_smem = smem_sm / (ns * slot + smem_static + smem_rsv);
    const int per_regs = 65536 / (((regs + 7) & ~7) * 128);
    return std::max(1, std::min({per_smem, per_regs, 16})) * sms;
}

cudaError_t conv3_wgrad(const void* in, int in_stride, int cin, const void* gz, int gz_stride, int cout, float* partial,
                        int splits, float* dw, int batch, int D, int H, int W, int kp, int np, cudaStream_t s)
{
    // the window kernel needs one split per batch at least (its partial sums
    // are laid out per batch split)
    if (splits >= batch && cin % 16 == 0 && np <= 128)
        return conv3_wgrad_win(in, in_stride, cin, gz, gz_stride, cout, partial, splits, dw, batch, D, H, W, kp, np, s);
    return conv3_wgrad_gather(in, in_stride, cin, gz, gz_stride, cout, partial, splits, dw, batch, D, H, W, kp, np, s);
}

int bias_grad_work_floats(int cout) { return BG_BLOCKS * ((cout + 7) / 8) * 8; }

cudaError_t bias_grad(const void* gz, int stride, long long nvox, int cout, float* db, float* work, cudaStream_t s)
{
    const int G = (cout + 7) / 8;                 // 1, 2, 4, 8 or 16 (checked by the caller)
    bias_grad_kernel<<<BG_BLOCKS, 256, 0, s>>>(static_cast<const bf16*>(gz), stride, nvox, G, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bias_grad_reduce_kernel<<<(cout + 3) / 4, 128, 0, s>>>(work, BG_BLOCKS, 8 * G, cout, db);
    return cudaGetLastError();
}

namespace {
// grid of the 8-channel resampling kernels on a grid g: x over the (y, x,
// channel group) threads of a plane, y over (batch, plane) pairs
dim3 vox8_grid(const PadVol& g, int C, int B)
{
    const int per_plane = g.H * g.W * (C / 8);
    return dim3((unsigned)((per_plane + 255) / 256), (unsigned)std::min(B * g.D, 65535));
}
bool vox8_ok(const void* a, int as, const void* b, int bs, int C)
{
    return C % 8 == 0 && as % 8 == 0 && bs % 8 == 0 && !((uintptr_t)a & 15) && !((uintptr_t)b & 15);
}
}  // namespace

cudaError_t pool2(const void* x, int xs, void* y, int ys, int C, int B, int D, int H, int W, cudaStream_t s)
{
    if (!vox8_ok(x, xs, y, ys, C)) return cudaErrorInvalidValue;
    const PadVol gf = make_pad(D, H, W), gc = make_pad(D / 2, H / 2, W / 2);
    pool2_kernel<<<vox8_grid(gc, C, B), 256, 0, s>>>(static_cast<const bf16*>(x), xs, static_cast<bf16*>(y), ys, C, B,
                                                      gf, gc);
    return cudaGetLastError();
}

cudaError_t pool2_adjoint(const void* gy, int gys, const void* x, int xs, void* gx, int gxs, int C, float slope, int B,
                          int D, int H, int W, cudaStream_t s)
{
    if (!vox8_ok(gy, gys, x, xs, C) || !vox8_ok(gx, gxs, gx, gxs, C)) return cudaErrorInvalidValue;
    const PadVol gf = make_pad(D, H, W), gc = make_pad(D / 2, H / 2, W / 2);
    pool2_adjoint_kernel<<<vox8_grid(gf, C, B), 256, 0, s>>>(static_cast<const bf16*>(gy), gys,
                                                              static_cast<const bf16*>(x), xs, static_cast<bf16*>(gx),
                                                              gxs, C, slope, B, gf, gc);
    return cudaGetLastError();
}

cudaError_t up2(const void* x, int xs, void* y, int ys, int C, int B, int D, int H, int W, cudaStream_t s)
{
    if (!vox8_ok(x, xs, y, ys, C)) return cudaErrorInvalidValue;
    const PadVol gf = make_pad(D, H, W), gc = make_pad(D / 2, H / 2, W / 2);
    up2_kernel<<<vox8_grid(gf, C, B), 256, 0, s>>>(static_cast<const bf16*>(x), xs, static_cast<bf16*>(y), ys, C, B, gf,
                                                    gc);
    return cudaGetLastError();
}

cudaError_t up2_adjoint(const void* gy, int gys, void* gx, int gxs, int C, int B, int D, int H, int W, cudaStream_t s)
{
    if (!vox8_ok(gy, gys, gx, gxs, C)) return cudaErrorInvalidValue;
    const PadVol gf = make_pad(D, H, W), gc = make_pad(D / 2, H / 2, W / 2);
    up2_adjoint_kernel<<<vox8_grid(gc, C, B), 256, 0, s>>>(static_cast<const bf16*>(gy), gys, static_cast<bf16*>(gx),
                                                            gxs, C, B, gf, gc);
    return cudaGetLastError();
}

cudaError_t pack_input(const float* subj, const float* atlas, void* x, int B, int D, int H, int W, cudaStream_t s)
{
    pack_input_kernel<<<ew_grid((long long)B * D * H * W), 256, 0, s>>>(subj, atlas, static_cast<bf16*>(x),
                                                                        make_pad(D, H, W), B);
    return cudaGetLastError();
}

int velocity_loss_blocks(long long n) { return ew_grid(n); }

cudaError_t velocity_loss(const float* pred, const float* target, int B, int D, int H, int W, void* g, int gs,
                          double* partials, cudaStream_t s)
{
    if (gs % 8 || ((uintptr_t)g & 15)) return cudaErrorInvalidValue;
    const long long n = (long long)B * D * H * W;
    velocity_loss_kernel<<<ew_grid(n), 256, 0, s>>>(pred, target, B, make_pad(D, H, W), static_cast<bf16*>(g), gs,
                                                    partials, (float)(1.0 / (3.0 * (double)n)));
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
