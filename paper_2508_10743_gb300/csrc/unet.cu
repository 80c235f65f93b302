// unet.cu -- the learned warm start: a 3-D U-Net (4 levels, 16-32-64-128
// channels, BF16 weights and activations, FP32 accumulation on the tensor
// cores) that maps a (subject, atlas) pair at half resolution to a
// 3-channel velocity field, trained on velocities the plain method produced.
// This is an addition to the method; the paper has no counterpart.
//
// Layout: activations channels-last bf16 with a one-voxel zero border,
// [batch][D+2][H+2][W+2][stride] (borders are never written, so they stay
// zero); a skip connection is a channel slice of the decoder's concatenation
// buffer, so concatenation costs nothing.  Down-sampling: 2x average pooling;
// up-sampling: nearest 2x.  Every conv is 3x3x3 'same' + bias + leaky ReLU
// (slope 0.2), except the 3-channel head.
#include "../../include/darc.h"
#include "kernels.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

using namespace darc_impl;

namespace {

constexpr float kSlope = 0.2f;

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Layer {
    int cin, cinp, cout, kp, np, level, act;        // cinp, np: rounded up to 16; kp = 27 cinp
    float *w = nullptr, *b = nullptr, *mw = nullptr, *sw = nullptr, *mb = nullptr, *sb = nullptr;
    float *dw = nullptr, *db = nullptr;
    void *wb = nullptr, *wd = nullptr;     // bf16 packed forward / data-gradient weights
};

struct Buf {
    void* p = nullptr;                     // bf16 channels-last
    int stride = 0;
};

}  // namespace

struct darc_unet {
    int D, H, W, maxb, step = 0;
    std::vector<Layer> L;
    std::vector<void*> allocs;
    // activations and their gradients, per level
    Buf x0, a0, cat0, d0a, d0b, gh, ga0, gcat0, gd0a, gd0b;
    Buf p0, a1, cat1, d1a, d1b, gp0, ga1, gcat1, gd1a, gd1b;
    Buf p1, a2, cat2, d2a, d2b, gp1, ga2, gcat2, gd2a, gd2b;
    Buf p2, a3, b3, gp2, ga3, gb3;
    float *pred = nullptr, *partial = nullptr;
    double* lpart = nullptr;
    float* loss_dev = nullptr;
    size_t partial_floats = 0;
    int dims[4][3];
};

namespace {


int ufail(int code, const std::string& m) { return darc_impl::report_error(code, m); }

#define UCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return ufail(DARC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
int ualloc(darc_unet* u, T** p, size_t n)
{
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return ufail(DARC_ERR_OOM, "cudaMalloc failed");
    }
    if (cudaMemset(q, 0, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return ufail(DARC_ERR_CUDA, "cudaMemset failed");
    }
    u->allocs.push_back(q);
    *p = (T*)q;
    return DARC_OK;
}

int balloc(darc_unet* u, Buf& b, long long rows, int stride)
{
    b.stride = stride;
    return ualloc(u, reinterpret_cast<uint16_t**>(&b.p), (size_t)rows * stride);
}

void* ch(const Buf& b, int off) { return static_cast<uint16_t*>(b.p) + off; }

// SplitMix64 + Box-Muller: seeded He-normal initialisation on the host
struct Rng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return std::sqrt(-2.0 * std::log(uniform())) * std::cos(6.283185307179586 * uniform()); }
};

const int kSpec[15][4] = {
    // cin, cout, level, act
    {2, 16, 0, 1},  {16, 16, 0, 1}, {16, 32, 1, 1},  {32, 32, 1, 1}, {32, 64, 2, 1},
    {64, 64, 2, 1}, {64, 128, 3, 1}, {128, 128, 3, 1}, {192, 64, 2, 1}, {64, 64, 2, 1},
    {96, 32, 1, 1}, {32, 32, 1, 1}, {48, 16, 0, 1},  {16, 16, 0, 1}, {16, 3, 0, 0},
};

int prep_weights(darc_unet* u, Layer& l, cudaStream_t s)
{
    UCK(pack_weights(l.w, l.kp, l.cinp, l.cout, l.cinp, l.np, 0, l.wb, s));
    UCK(pack_weights(l.w, l.kp, l.cinp, l.cout, l.np, l.cinp, 1, l.wd, s));
    return DARC_OK;
}

int conv(darc_unet* u, const Layer& l, const Buf& in, int in_off, const Buf& out, int out_off, int B, cudaStream_t s,
         float* out_f32 = nullptr)
{
    const int* d = u->dims[l.level];
    ConvDesc c{};
    c.in = ch(in, in_off);
    c.in_stride = in.stride;
    c.cin = l.cinp;
    c.wt = l.wb;
    c.bias = l.b;
    c.out = out_f32 ? nullptr : ch(out, out_off);
    c.out_stride = out.stride;
    c.cout = l.cout;
    c.out_f32 = out_f32;
    c.act = l.act;
    c.slope = kSlope;
    c.batch = B;
    c.D = d[0];
    c.H = d[1];
    c.W = d[2];
    c.np = l.np;
    UCK(conv3_forward(c, s));
    return DARC_OK;
}

// gradient wrt the layer input: conv of gz with the flipped weights; gate =
// the layer input when it is itself a leaky-ReLU output (null otherwise)
int dgrad(darc_unet* u, const Layer& l, const Buf& gz, int gz_off, const Buf& gin, int gin_off, const Buf* gate,
          int gate_off, int B, cudaStream_t s)
{
    const int* d = u->dims[l.level];
    ConvDesc c{};
    c.in = ch(gz, gz_off);
    c.in_stride = gz.stride;
    c.cin = l.np;
    c.wt = l.wd;
    c.bias = nullptr;
    c.out = ch(gin, gin_off);
    c.out_stride = gin.stride;
    c.cout = l.cinp;
    c.gate = gate ? ch(*gate, gate_off) : nullptr;
    c.gate_stride = gate ? gate->stride : 0;
    c.act = 0;
    c.slope = kSlope;
    c.batch = B;
    c.D = d[0];
    c.H = d[1];
    c.W = d[2];
    c.np = l.cinp;
    UCK(conv3_forward(c, s));
    return DARC_OK;
}

int wgrad(darc_unet* u, Layer& l, const Buf& in, int in_off, const Buf& gz, int gz_off, int B, cudaStream_t s)
{
    const int* d = u->dims[l.level];
    const PadVol g = make_pad(d[0], d[1], d[2]);
    const long long nrows = (long long)B * d[0] * g.P;
    const int tiles = wgrad_ctas_per_split(l.cinp);
    int splits = (int)std::max<long long>(1, std::min<long long>(std::min<long long>(wgrad_resident_ctas(l.np) / tiles, nrows / 1024), 256));
    while ((size_t)splits * l.kp * l.np > u->partial_floats && splits > 1) splits /= 2;
    UCK(conv3_wgrad(ch(in, in_off), in.stride, l.cinp, ch(gz, gz_off), gz.stride, l.np, u->partial, splits, l.dw,
                    B, d[0], d[1], d[2], l.kp, l.np, s));
    // partials are free again once the split reduction has run (same stream)
    UCK(bias_grad(ch(gz, gz_off), gz.stride, (long long)B * g.Vp, l.cout, l.db, u->partial, s));
    return DARC_OK;
}

int forward(darc_unet* u, const float* subj, const float* atlas, int B, cudaStream_t s)
{
    auto& L = u->L;
    const int* d0 = u->dims[0];
    const int* d1 = u->dims[1];
    const int* d2 = u->dims[2];
    int rc;
    UCK(pack_input(subj, atlas, u->x0.p, B, d0[0], d0[1], d0[2], s));
#define RUN(x) do { rc = (x); if (rc) return rc; } while (0)
    RUN(conv(u, L[0], u->x0, 0, u->a0, 0, B, s));
    RUN(conv(u, L[1], u->a0, 0, u->cat0, 32, B, s));
    UCK(pool2(ch(u->cat0, 32), 48, u->p0.p, 16, 16, B, d0[0], d0[1], d0[2], s));
    RUN(conv(u, L[2], u->p0, 0, u->a1, 0, B, s));
    RUN(conv(u, L[3], u->a1, 0, u->cat1, 64, B, s));
    UCK(pool2(ch(u->cat1, 64), 96, u->p1.p, 32, 32, B, d1[0], d1[1], d1[2], s));
    RUN(conv(u, L[4], u->p1, 0, u->a2, 0, B, s));
    RUN(conv(u, L[5], u->a2, 0, u->cat2, 128, B, s));
    UCK(pool2(ch(u->cat2, 128), 192, u->p2.p, 64, 64, B, d2[0], d2[1], d2[2], s));
    RUN(conv(u, L[6], u->p2, 0, u->a3, 0, B, s));
    RUN(conv(u, L[7], u->a3, 0, u->b3, 0, B, s));
    UCK(up2(u->b3.p, 128, u->cat2.p, 192, 128, B, d2[0], d2[1], d2[2], s));
    RUN(conv(u, L[8], u->cat2, 0, u->d2a, 0, B, s));
    RUN(conv(u, L[9], u->d2a, 0, u->d2b, 0, B, s));
    UCK(up2(u->d2b.p, 64, u->cat1.p, 96, 64, B, d1[0], d1[1], d1[2], s));
    RUN(conv(u, L[10], u->cat1, 0, u->d1a, 0, B, s));
    RUN(conv(u, L[11], u->d1a, 0, u->d1b, 0, B, s));
    UCK(up2(u->d1b.p, 32, u->cat0.p, 48, 32, B, d0[0], d0[1], d0[2], s));
    RUN(conv(u, L[12], u->cat0, 0, u->d0a, 0, B, s));
    RUN(conv(u, L[13], u->d0a, 0, u->d0b, 0, B, s));
    RUN(conv(u, L[14], u->d0b, 0, u->d0b, 0, B, s, u->pred));
#undef RUN
    return DARC_OK;
}

int backward(darc_unet* u, int B, cudaStream_t s)
{
    auto& L = u->L;
    const int* d0 = u->dims[0];
    const int* d1 = u->dims[1];
    const int* d2 = u->dims[2];
    int rc;
#define RUN(x) do { rc = (x); if (rc) return rc; } while (0)
    // head (no activation): gradient wrt its output is in gh
    RUN(wgrad(u, L[14], u->d0b, 0, u->gh, 0, B, s));
    RUN(dgrad(u, L[14], u->gh, 0, u->gd0b, 0, &u->d0b, 0, B, s));
    RUN(wgrad(u, L[13], u->d0a, 0, u->gd0b, 0, B, s));
    RUN(dgrad(u, L[13], u->gd0b, 0, u->gd0a, 0, &u->d0a, 0, B, s));
    RUN(wgrad(u, L[12], u->cat0, 0, u->gd0a, 0, B, s));
    RUN(dgrad(u, L[12], u->gd0a, 0, u->gcat0, 0, &u->cat0, 0, B, s));
    UCK(up2_adjoint(u->gcat0.p, 48, u->gd1b.p, 32, 32, B, d0[0], d0[1], d0[2], s));
    RUN(wgrad(u, L[11], u->d1a, 0, u->gd1b, 0, B, s));
    RUN(dgrad(u, L[11], u->gd1b, 0, u->gd1a, 0, &u->d1a, 0, B, s));
    RUN(wgrad(u, L[10], u->cat1, 0, u->gd1a, 0, B, s));
    RUN(dgrad(u, L[10], u->gd1a, 0, u->gcat1, 0, &u->cat1, 0, B, s));
    UCK(up2_adjoint(u->gcat1.p, 96, u->gd2b.p, 64, 64, B, d1[0], d1[1], d1[2], s));
    RUN(wgrad(u, L[9], u->d2a, 0, u->gd2b, 0, B, s));
    RUN(dgrad(u, L[9], u->gd2b, 0, u->gd2a, 0, &u->d2a, 0, B, s));
    RUN(wgrad(u, L[8], u->cat2, 0, u->gd2a, 0, B, s));
    RUN(dgrad(u, L[8], u->gd2a, 0, u->gcat2, 0, &u->cat2, 0, B, s));
    UCK(up2_adjoint(u->gcat2.p, 192, u->gb3.p, 128, 128, B, d2[0], d2[1], d2[2], s));
    RUN(wgrad(u, L[7], u->a3, 0, u->gb3, 0, B, s));
    RUN(dgrad(u, L[7], u->gb3, 0, u->ga3, 0, &u->a3, 0, B, s));
    RUN(wgrad(u, L[6], u->p2, 0, u->ga3, 0, B, s));
    RUN(dgrad(u, L[6], u->ga3, 0, u->gp2, 0, nullptr, 0, B, s));
    UCK(pool2_adjoint(u->gp2.p, 64, ch(u->cat2, 128), 192, ch(u->gcat2, 128), 192, 64, kSlope, B, d2[0], d2[1], d2[2], s));
    RUN(wgrad(u, L[5], u->a2, 0, u->gcat2, 128, B, s));
    RUN(dgrad(u, L[5], u->gcat2, 128, u->ga2, 0, &u->a2, 0, B, s));
    RUN(wgrad(u, L[4], u->p1, 0, u->ga2, 0, B, s));
    RUN(dgrad(u, L[4], u->ga2, 0, u->gp1, 0, nullptr, 0, B, s));
    UCK(pool2_adjoint(u->gp1.p, 32, ch(u->cat1, 64), 96, ch(u->gcat1, 64), 96, 32, kSlope, B, d1[0], d1[1], d1[2], s));
    RUN(wgrad(u, L[3], u->a1, 0, u->gcat1, 64, B, s));
    RUN(dgrad(u, L[3], u->gcat1, 64, u->ga1, 0, &u->a1, 0, B, s));
    RUN(wgrad(u, L[2], u->p0, 0, u->ga1, 0, B, s));
    RUN(dgrad(u, L[2], u->ga1, 0, u->gp0, 0, nullptr, 0, B, s));
    UCK(pool2_adjoint(u->gp0.p, 16, ch(u->cat0, 32), 48, ch(u->gcat0, 32), 48, 16, kSlope, B, d0[0], d0[1], d0[2], s));
    RUN(wgrad(u, L[1], u->a0, 0, u->gcat0, 32, B, s));
    RUN(dgrad(u, L[1], u->gcat0, 32, u->ga0, 0, &u->a0, 0, B, s));
    RUN(wgrad(u, L[0], u->x0, 0, u->ga0, 0, B, s));
#undef RUN
    return DARC_OK;
}

int check_unet_dims(int D, int H, int W)
{
    if (D < 16 || H < 16 || W < 16 || D % 8 || H % 8 || W % 8)
        return ufail(DARC_ERR_SHAPE, "U-Net volume must be >= 16 and a multiple of 8 along every axis");
    if (!conv_fits(W, 256)) return ufail(DARC_ERR_SHAPE, "U-Net volume too wide for the convolution's window");
    return DARC_OK;
}

}  // namespace

extern "C" {

int darc_unet_create(darc_unet** out, int D, int H, int W, int max_batch, unsigned long long seed)
{
    if (!out || max_batch < 1) return ufail(DARC_ERR_ARG, "bad argument");
    *out = nullptr;
    int rc = check_unet_dims(D, H, W);
    if (rc) return rc;
    darc_unet* u = new darc_unet();
    u->D = D;
    u->H = H;
    u->W = W;
    u->maxb = max_batch;
    for (int lv = 0; lv < 4; ++lv) {
        u->dims[lv][0] = D >> lv;
        u->dims[lv][1] = H >> lv;
        u->dims[lv][2] = W >> lv;
    }
    auto fail_out = [&](int code) {
        darc_unet_destroy(u);
        return code;
    };
    Rng rng{seed * 0x2545F4914F6CDD1DULL + 17};
    for (int i = 0; i < 15; ++i) {
        Layer l;
        l.cin = kSpec[i][0];
        l.cinp = round_up(l.cin, 16);
        l.cout = kSpec[i][1];
        l.level = kSpec[i][2];
        l.act = kSpec[i][3];
        l.kp = 27 * l.cinp;
        l.np = round_up(l.cout, 16);
        const size_t nw = (size_t)l.np * l.kp;
        if ((rc = ualloc(u, &l.w, nw)) || (rc = ualloc(u, &l.mw, nw)) || (rc = ualloc(u, &l.sw, nw)) ||
            (rc = ualloc(u, &l.dw, nw)) || (rc = ualloc(u, &l.b, l.cout)) || (rc = ualloc(u, &l.mb, l.cout)) ||
            (rc = ualloc(u, &l.sb, l.cout)) || (rc = ualloc(u, &l.db, l.cout)) ||
            (rc = ualloc(u, reinterpret_cast<uint16_t**>(&l.wb), packed_weight_elems(l.cinp, l.np))) ||
            (rc = ualloc(u, reinterpret_cast<uint16_t**>(&l.wd), packed_weight_elems(l.np, l.cinp))))
            return fail_out(rc);
        // He-normal for leaky ReLU; the head starts small so the first
        // proposals stay close to zero velocity
        std::vector<float> hw(nw, 0.f);
        const double std = std::sqrt(2.0 / (1.0 + kSlope * kSlope) / (27.0 * l.cin)) * (l.act ? 1.0 : 0.1);
        for (int co = 0; co < l.cout; ++co)
            for (int tap = 0; tap < 27; ++tap)
                for (int ci = 0; ci < l.cin; ++ci) hw[(size_t)co * l.kp + tap * l.cinp + ci] = (float)(std * rng.normal());
        if (cudaMemcpy(l.w, hw.data(), nw * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail_out(ufail(DARC_ERR_CUDA, "weight upload failed"));
        u->L.push_back(l);
    }
    const int B = max_batch;
    const long long V0 = (long long)D * H * W;
    const long long P0 = make_pad(D, H, W).Vp, P1 = make_pad(D / 2, H / 2, W / 2).Vp,
                    P2 = make_pad(D / 4, H / 4, W / 4).Vp, P3 = make_pad(D / 8, H / 8, W / 8).Vp;
    struct { Buf* b; long long v; int c; } bufs[] = {
        {&u->x0, P0, 16}, {&u->a0, P0, 16}, {&u->cat0, P0, 48}, {&u->d0a, P0, 16}, {&u->d0b, P0, 16},
        {&u->gh, P0, 16}, {&u->ga0, P0, 16}, {&u->gcat0, P0, 48}, {&u->gd0a, P0, 16}, {&u->gd0b, P0, 16},
        {&u->p0, P1, 16}, {&u->a1, P1, 32}, {&u->cat1, P1, 96}, {&u->d1a, P1, 32}, {&u->d1b, P1, 32},
        {&u->gp0, P1, 16}, {&u->ga1, P1, 32}, {&u->gcat1, P1, 96}, {&u->gd1a, P1, 32}, {&u->gd1b, P1, 32},
        {&u->p1, P2, 32}, {&u->a2, P2, 64}, {&u->cat2, P2, 192}, {&u->d2a, P2, 64}, {&u->d2b, P2, 64},
        {&u->gp1, P2, 32}, {&u->ga2, P2, 64}, {&u->gcat2, P2, 192}, {&u->gd2a, P2, 64}, {&u->gd2b, P2, 64},
        {&u->p2, P3, 64}, {&u->a3, P3, 128}, {&u->b3, P3, 128}, {&u->gp2, P3, 64}, {&u->ga3, P3, 128},
        {&u->gb3, P3, 128},
    };
    for (auto& e : bufs)
        if ((rc = balloc(u, *e.b, e.v * B, e.c))) return fail_out(rc);
    u->partial_floats = (size_t)64 << 20;       // 256 MB of split-K partial sums
    if ((rc = ualloc(u, &u->pred, (size_t)3 * V0 * B)) || (rc = ualloc(u, &u->partial, u->partial_floats)) ||
        (rc = ualloc(u, &u->lpart, (size_t)velocity_loss_blocks(V0 * B))) || (rc = ualloc(u, &u->loss_dev, 1)))
        return fail_out(rc);
    for (auto& l : u->L)
        if ((rc = prep_weights(u, l, 0))) return fail_out(rc);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail_out(ufail(DARC_ERR_CUDA, "initialisation failed"));
    *out = u;
    return DARC_OK;
}

void darc_unet_destroy(darc_unet* u)
{
    if (!u) return;
    cudaDeviceSynchronize();
    for (void* p : u->allocs) cudaFree(p);
    delete u;
}

int darc_unet_forward(darc_unet* u, const float* subj_dev, const float* atlas_dev, int B, float* v_dev, void* stream)
{
    if (!u || !subj_dev || !atlas_dev || !v_dev) return ufail(DARC_ERR_ARG, "null argument");
    if (B < 1 || B > u->maxb) return ufail(DARC_ERR_ARG, "batch outside 1..max_batch");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = forward(u, subj_dev, atlas_dev, B, s);
    if (rc) return rc;
    UCK(cudaMemcpyAsync(v_dev, u->pred, sizeof(float) * 3 * (size_t)B * u->D * u->H * u->W, cudaMemcpyDeviceToDevice, s));
    return DARC_OK;
}

int darc_unet_train_step(darc_unet* u, const float* subj_dev, const float* atlas_dev, const float* target_dev, int B,
                         float lr, float* loss_host, void* stream)
{
    if (!u || !subj_dev || !atlas_dev || !target_dev) return ufail(DARC_ERR_ARG, "null argument");
    if (B < 1 || B > u->maxb || !(lr > 0.f)) return ufail(DARC_ERR_ARG, "bad batch or learning rate");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = forward(u, subj_dev, atlas_dev, B, s);
    if (rc) return rc;
    const long long n = (long long)B * u->D * u->H * u->W;
    UCK(velocity_loss(u->pred, target_dev, B, u->D, u->H, u->W, u->gh.p, 16, u->lpart, s));
    UCK(reduce_partials(u->lpart, velocity_loss_blocks(n), 1, 1.0, u->loss_dev, 1, 1, s));
    rc = backward(u, B, s);
    if (rc) return rc;
    u->step += 1;
    const double c1 = 1.0 - std::pow(0.9, u->step), c2 = 1.0 - std::pow(0.999, u->step);
    for (auto& l : u->L) {
        UCK(adam_flat(l.w, l.mw, l.sw, l.dw, (size_t)l.np * l.kp, (float)(lr / c1), (float)(1.0 / std::sqrt(c2)), 0.9f,
                      0.999f, 1e-8f, s));
        UCK(adam_flat(l.b, l.mb, l.sb, l.db, (size_t)l.cout, (float)(lr / c1), (float)(1.0 / std::sqrt(c2)), 0.9f,
                      0.999f, 1e-8f, s));
        if ((rc = prep_weights(u, l, s))) return rc;
    }
    if (loss_host) {
        UCK(cudaStreamSynchronize(s));
        UCK(cudaMemcpy(loss_host, u->loss_dev, sizeof(float), cudaMemcpyDeviceToHost));
    }
    return DARC_OK;
}

int darc_unet_gradients(darc_unet* u, const float* subj_dev, const float* atlas_dev, const float* target_dev, int B,
                        float* loss_host, void* stream)
{
    if (!u || !subj_dev || !atlas_dev || !target_dev) return ufail(DARC_ERR_ARG, "null argument");
    if (B < 1 || B > u->maxb) return ufail(DARC_ERR_ARG, "batch outside 1..max_batch");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = forward(u, subj_dev, atlas_dev, B, s);
    if (rc) return rc;
    const long long n = (long long)B * u->D * u->H * u->W;
    UCK(velocity_loss(u->pred, target_dev, B, u->D, u->H, u->W, u->gh.p, 16, u->lpart, s));
    UCK(reduce_partials(u->lpart, velocity_loss_blocks(n), 1, 1.0, u->loss_dev, 1, 1, s));
    rc = backward(u, B, s);
    if (rc) return rc;
    if (loss_host) {
        UCK(cudaStreamSynchronize(s));
        UCK(cudaMemcpy(loss_host, u->loss_dev, sizeof(float), cudaMemcpyDeviceToHost));
    }
    return DARC_OK;
}

int darc_unet_layer_info(darc_unet* u, int layer, int* cin, int* cout, int* kp, int* np)
{
    if (!u || layer < 0 || layer >= (int)u->L.size()) return ufail(DARC_ERR_ARG, "bad layer");
    const Layer& l = u->L[layer];
    if (cin) *cin = l.cinp;
    if (cout) *cout = l.cout;
    if (kp) *kp = l.kp;
    if (np) *np = l.np;
    return DARC_OK;
}

int darc_unet_layer_params(darc_unet* u, int layer, float* w_dev, float* b_dev, float* dw_dev, float* db_dev, int set)
{
    if (!u || layer < 0 || layer >= (int)u->L.size()) return ufail(DARC_ERR_ARG, "bad layer");
    Layer& l = u->L[layer];
    const size_t nw = (size_t)l.np * l.kp;
    if (set) {
        if (w_dev) UCK(cudaMemcpy(l.w, w_dev, nw * sizeof(float), cudaMemcpyDeviceToDevice));
        if (b_dev) UCK(cudaMemcpy(l.b, b_dev, l.cout * sizeof(float), cudaMemcpyDeviceToDevice));
        int rc = prep_weights(u, l, 0);
        if (rc) return rc;
        UCK(cudaDeviceSynchronize());
        return DARC_OK;
    }
    UCK(cudaDeviceSynchronize());
    if (w_dev) UCK(cudaMemcpy(w_dev, l.w, nw * sizeof(float), cudaMemcpyDeviceToDevice));
    if (b_dev) UCK(cudaMemcpy(b_dev, l.b, l.cout * sizeof(float), cudaMemcpyDeviceToDevice));
    if (dw_dev) UCK(cudaMemcpy(dw_dev, l.dw, nw * sizeof(float), cudaMemcpyDeviceToDevice));
    if (db_dev) UCK(cudaMemcpy(db_dev, l.db, l.cout * sizeof(float), cudaMemcpyDeviceToDevice));
    return DARC_OK;
}

int darc_unet_save(darc_unet* u, const char* path)
{
    if (!u || !path) return ufail(DARC_ERR_ARG, "null argument");
    UCK(cudaDeviceSynchronize());
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return ufail(DARC_ERR_IO, std::string("cannot open ") + path);
    const char magic[8] = {'D', 'A', 'R', 'C', 'U', 'N', 'T', '1'};
    bool ok = std::fwrite(magic, 1, 8, fp) == 8 && std::fwrite(&u->step, sizeof(int), 1, fp) == 1;
    for (auto& l : u->L) {
        const size_t nw = (size_t)l.np * l.kp;
        std::vector<float> h(nw);
        for (float* arr : {l.w, l.mw, l.sw}) {
            ok = ok && cudaMemcpy(h.data(), arr, nw * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess &&
                 std::fwrite(h.data(), sizeof(float), nw, fp) == nw;
        }
        for (float* arr : {l.b, l.mb, l.sb}) {
            ok = ok && cudaMemcpy(h.data(), arr, l.cout * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess &&
                 std::fwrite(h.data(), sizeof(float), l.cout, fp) == (size_t)l.cout;
        }
    }
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? DARC_OK : ufail(DARC_ERR_IO, "writing the U-Net failed");
}

int darc_unet_load(darc_unet* u, const char* path)
{
    if (!u || !path) return ufail(DARC_ERR_ARG, "null argument");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return ufail(DARC_ERR_IO, std::string("cannot open ") + path);
    char magic[8];
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "DARCUNT1", 8) == 0 &&
              std::fread(&u->step, sizeof(int), 1, fp) == 1;
    for (auto& l : u->L) {
        const size_t nw = (size_t)l.np * l.kp;
        std::vector<float> h(nw);
        for (float* arr : {l.w, l.mw, l.sw})
            ok = ok && std::fread(h.data(), sizeof(float), nw, fp) == nw &&
                 cudaMemcpy(arr, h.data(), nw * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
        for (float* arr : {l.b, l.mb, l.sb})
            ok = ok && std::fread(h.data(), sizeof(float), l.cout, fp) == (size_t)l.cout &&
                 cudaMemcpy(arr, h.data(), l.cout * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
        if (ok) ok = prep_weights(u, l, 0) == DARC_OK;
    }
    std::fclose(fp);
    return ok ? DARC_OK : ufail(DARC_ERR_IO, "reading the U-Net failed");
}

int darc_resample_half(const float* I_dev, int B, int D, int H, int W, float* out_dev, void* stream)
{
    if (!I_dev || !out_dev || B < 1 || D < 2 || H < 2 || W < 2 || D % 2 || H % 2 || W % 2)
        return ufail(DARC_ERR_ARG, "bad argument");
    UCK(downsample_image(I_dev, D, H, W, out_dev, B, (cudaStream_t)stream));
    return DARC_OK;
}

int darc_upsample_velocity(const float* vh_dev, int B, int Dh, int Hh, int Wh, float* v_dev, void* stream)
{
    if (!vh_dev || !v_dev || B < 1 || Dh < 2 || Hh < 2 || Wh < 2) return ufail(DARC_ERR_ARG, "bad argument");
    UCK(upsample_velocity(vh_dev, Dh, Hh, Wh, v_dev, 2 * Dh, 2 * Hh, 2 * Wh, B, (cudaStream_t)stream));
    return DARC_OK;
}

size_t darc_conv3d_packed_bytes(int conv_cin, int nrows)
{
    if (conv_cin < 16 || conv_cin % 16 || nrows < 16 || nrows % 16) return 0;
    return packed_weight_elems(conv_cin, nrows) * 2;
}

int darc_conv3d_pack_weights(const float* w_dev, int kp, int cin, int cout, int flip, void* packed_dev, void* stream)
{
    if (!w_dev || !packed_dev) return ufail(DARC_ERR_ARG, "null argument");
    if (cin < 16 || cin % 16 || cout < 1 || cout > 256 || kp < 27 * cin || (flip != 0 && flip != 1))
        return ufail(DARC_ERR_SHAPE, "conv3d_pack_weights: cin % 16 == 0, 1 <= cout <= 256, kp >= 27 cin");
    if ((uintptr_t)packed_dev & 15) return ufail(DARC_ERR_ARG, "packed weights must be 16-byte aligned");
    const int coutp = round_up(cout, 16);
    UCK(pack_weights(w_dev, kp, cin, cout, flip ? coutp : cin, flip ? cin : coutp, flip, packed_dev,
                     (cudaStream_t)stream));
    return DARC_OK;
}

int darc_conv3d(const void* in_dev, int in_stride, int cin, const void* wt_dev, const float* bias_dev, void* out_dev,
                int out_stride, int cout, float* out_f32_dev, const void* gate_dev, int gate_stride, int act,
                float slope, int batch, int D, int H, int W, int np, void* stream)
{
    if (!in_dev || !wt_dev || (!out_dev && !out_f32_dev)) return ufail(DARC_ERR_ARG, "null argument");
    if (cin < 16 || cin % 16 || in_stride < cin || in_stride % 8 || np < 16 || np > 256 || np % 16 || cout < 1 ||
        cout > np || (!out_f32_dev && out_stride < cout) || batch < 1 || D < 1 || H < 1 || W < 1 ||
        (gate_dev && gate_stride < cout))
        return ufail(DARC_ERR_SHAPE, "conv3d: cin % 16 == 0, in_stride % 8 == 0, np % 16 == 0 <= 256, cout <= np");
    if (!conv_fits(W, np)) return ufail(DARC_ERR_SHAPE, "conv3d: W too large for the shared-memory window");
    if (((uintptr_t)in_dev & 15) || ((uintptr_t)wt_dev & 15)) return ufail(DARC_ERR_ARG, "operands must be 16-byte aligned");
    ConvDesc c{};
    c.in = in_dev;
    c.in_stride = in_stride;
    c.cin = cin;
    c.wt = wt_dev;
    c.bias = bias_dev;
    c.out = out_dev;
    c.out_stride = out_stride;
    c.cout = cout;
    c.out_f32 = out_f32_dev;
    c.gate = gate_dev;
    c.gate_stride = gate_stride;
    c.act = act;
    c.slope = slope;
    c.batch = batch;
    c.D = D;
    c.H = H;
    c.W = W;
    c.np = np;
    UCK(conv3_forward(c, (cudaStream_t)stream));
    return DARC_OK;
}

int darc_conv3d_wgrad(const void* in_dev, int in_stride, int cin, const void* gz_dev, int gz_stride, int cout,
                      float* dw_dev, float* db_dev, int batch, int D, int H, int W, int np, void* work_dev,
                      size_t work_bytes, void* stream)
{
    if (!in_dev || !gz_dev || !dw_dev || !work_dev) return ufail(DARC_ERR_ARG, "null argument");
    if (cin < 16 || cin % 16 || in_stride % 8 || cout % 8 || gz_stride % 8 || gz_stride < cout || np % 16 ||
        np < 16 || np > 128 || cout > np || batch < 1 || D < 1 || H < 1 || W < 1)
        return ufail(DARC_ERR_SHAPE, "conv3d_wgrad: cin % 16 == 0, cout and strides multiples of 8, np <= 128");
    if (db_dev && 256 % (cout / 8)) return ufail(DARC_ERR_SHAPE, "conv3d_wgrad: cout / 8 must divide 256");
    if (((uintptr_t)in_dev & 15) || ((uintptr_t)gz_dev & 15)) return ufail(DARC_ERR_ARG, "operands must be 16-byte aligned");
    const int kp = 27 * cin;
    const PadVol g = make_pad(D, H, W);
    const long long nrows = (long long)batch * D * g.P;
    int splits = (int)std::max<long long>(
        batch, std::min<long long>(std::min<long long>(256, nrows / 1024), wgrad_resident_ctas(np) /
                                                                                wgrad_ctas_per_split(cin)));
    while (splits > 1 && (size_t)splits * kp * np * sizeof(float) > work_bytes) splits /= 2;
    if ((size_t)splits * kp * np * sizeof(float) > work_bytes ||
        (db_dev && (size_t)bias_grad_work_floats(cout) * sizeof(float) > work_bytes))
        return ufail(DARC_ERR_ARG, "workspace too small");
    UCK(conv3_wgrad(in_dev, in_stride, cin, gz_dev, gz_stride, cout, (float*)work_dev, splits, dw_dev, batch, D, H, W,
                    kp, np, (cudaStream_t)stream));
    // the bias partials reuse the workspace once the split-K reduction has consumed it (same stream)
    if (db_dev)
        UCK(bias_grad(gz_dev, gz_stride, (long long)batch * g.Vp, cout, db_dev, (float*)work_dev, (cudaStream_t)stream));
    return DARC_OK;
}

}  // extern "C"
