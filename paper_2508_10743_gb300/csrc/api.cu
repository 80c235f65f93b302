// api.cu -- the C ABI of libdarc.so (include/darc.h).
//
// The cohort runs Algorithm 1 of arXiv 2508.10743 on the GPU: subject steps
// (Eq. 3, lines 1..n) batched over subjects (they are uncoupled given the
// atlas, Sec. "Coordinate descent method"), the centrality activation
// (Eq. 3, line n+1) and the atlas re-estimate (Eq. 3, last line; closed
// form for MSE, mini-batch Adam for local NCC).  Each subject step is
// recorded once as a CUDA graph per (first, count) chunk and replayed.
#include "../../include/darc.h"
#include "kernels.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

using namespace darc_impl;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(DARC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

int check_dims(int B, int D, int H, int W)
{
    if (B < 1) return fail(DARC_ERR_ARG, "batch must be >= 1");
    if (D < 2 || H < 2 || W < 2) return fail(DARC_ERR_SHAPE, "every dimension must be >= 2");
    if ((long long)D * H * W > (1LL << 31)) return fail(DARC_ERR_SHAPE, "volume too large");
    if ((long long)div_up(D, VT_Z) * B > 65535) return fail(DARC_ERR_SHAPE, "batch x depth too large for one launch");
    return DARC_OK;
}

int check_window(int w, int D, int H, int W)
{
    if (w < 3 || w > 17 || (w % 2) == 0) return fail(DARC_ERR_SHAPE, "NCC window must be odd, 3..17");
    if (w > D || w > H || w > W) return fail(DARC_ERR_SHAPE, "NCC window larger than the volume");
    return DARC_OK;
}

// point-wise metrics (closed-form atlas) and patch-wise metrics (box
// windows, atlas by mini-batch Adam)
bool pointwise(int d) { return d == DARC_MSE || d == DARC_L1; }
bool patchwise(int d) { return d == DARC_LNCC || d == DARC_SSIM; }
int patch_metric(int d) { return d == DARC_SSIM ? 1 : 0; }

int check_config(const darc_config* c, int D, int H, int W)
{
    if (c && c->adjoint != DARC_ADJOINT_SCATTER && c->adjoint != DARC_ADJOINT_GATHER)
        return fail(DARC_ERR_ARG, "adjoint must be DARC_ADJOINT_SCATTER or DARC_ADJOINT_GATHER");
    if (!c) return fail(DARC_ERR_ARG, "null config");
    if (!pointwise(c->dissim) && !patchwise(c->dissim)) return fail(DARC_ERR_ARG, "unknown dissimilarity");
    if (patchwise(c->dissim)) {
        int rc = check_window(c->ncc_window, D, H, W);
        if (rc) return rc;
    }
    if (c->n_squarings < 1 || c->n_squarings > 20) return fail(DARC_ERR_ARG, "n_squarings must be 1..20");
    if (!(c->lr > 0.f) || !(c->beta1 >= 0.f && c->beta1 < 1.f) || !(c->beta2 >= 0.f && c->beta2 < 1.f) ||
        !(c->adam_eps > 0.f) || !(c->ncc_eps >= 0.f) || !(c->lambda >= 0.f))
        return fail(DARC_ERR_ARG, "bad optimiser or loss constant");
    if (c->inner_steps < 1 || c->atlas_epochs < 0 || c->atlas_batch < 1 || c->subject_batch < 0)
        return fail(DARC_ERR_ARG, "bad step / batch count");
    if (c->center_mode != 0) return fail(DARC_ERR_ARG, "only center_mode 0 (velocities) is built");
    if (c->checkpoint_stride < 0) return fail(DARC_ERR_ARG, "checkpoint_stride must be >= 0");
    return DARC_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// sub-allocation of a caller workspace
struct Carve {
    char* base;
    size_t off = 0;
    explicit Carve(void* p) : base((char*)p) {}
    template <typename T>
    T* take(size_t count)
    {
        T* p = base ? (T*)(base + off) : nullptr;
        off += align256(count * sizeof(T));
        return p;
    }
};

int nblk_max(const Vol& v) { return std::max(voxel_blocks(v), box_blocks_max(v)); }

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the k-th output of the
// stream seeded s0 is mix(s0 + k * golden gamma).  Mini-batch order of the
// atlas SGD: Fisher-Yates from the last position down, j = draw mod (i+1),
// s0 = seed * 1000003 + sweep * 1009 + epoch.
uint64_t splitmix64_at(uint64_t s0, uint64_t k)
{
    uint64_t z = s0 + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void minibatch_order(uint64_t seed, int sweep, int epoch, int n, int* perm)
{
    const uint64_t s0 = seed * 1000003ULL + (uint64_t)sweep * 1009ULL + (uint64_t)epoch;
    for (int i = 0; i < n; ++i) perm[i] = i;
    uint64_t k = 0;
    for (int i = n - 1; i >= 1; --i) {
        ++k;
        const int j = (int)(splitmix64_at(s0, k) % (uint64_t)(i + 1));
        std::swap(perm[i], perm[j]);
    }
}

// Exp forward of `cnt` fields into u (T slots of cnt*3V); returns u_T
// Which squaring fields the adjoint keeps.  Stride s (2 <= s < T): u_t is
// stored for (t + 1) % s == 0 and for the last step; every other field sits
// in one of s - 1 scratch slots (slot t % s) and is recomputed, one segment
// of s steps at a time, from the checkpoint below it.  Stride 0, 1 or >= T
// keeps all T.  Fields are t = 0..T-1 = the outputs of the T squarings.
struct CkPlan {
    int T, s, nck;
    CkPlan(int T_, int stride) : T(T_), s((stride <= 1 || stride >= T_) ? 0 : stride)
    {
        nck = s ? T / s + (T % s != 0) : T;
    }
    int fields() const { return s ? nck + s - 1 : T; }
    bool kept(int t) const { return !s || (t + 1) % s == 0 || t == T - 1; }
    int slot(int t) const
    {
        if (!s) return t;
        if ((t + 1) % s == 0) return (t + 1) / s - 1;
        if (t == T - 1) return nck - 1;
        return nck + t % s;
    }
    // segment of the last field the forward leaves in scratch (-1: none)
    int scratch_segment() const
    {
        if (!s) return -1;
        for (int t = T - 1; t >= 0; --t)
            if (!kept(t)) return t / s;
        return -1;
    }
};

// Forward squarings into the plan's slots; sq(src, scale, dst) launches one.
template <typename Sq>
cudaError_t exp_forward_plan(const CkPlan& pl, const float* v, float* u, size_t fb, float s0, Sq sq)
{
    for (int t = 0; t < pl.T; ++t) {
        const float* src = t ? u + (size_t)pl.slot(t - 1) * fb : v;
        cudaError_t e = sq(src, t ? 1.f : s0, u + (size_t)pl.slot(t) * fb);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Adjoint steps t = T-1 .. 0 in segment order, recomputing a segment's
// scratch fields when they are not the ones the forward left there;
// adj(t, src, scale) runs the adjoint of step t.
template <typename Sq, typename Adj>
cudaError_t exp_backward_plan(const CkPlan& pl, const float* v, float* u, size_t fb, float s0, Sq sq, Adj adj)
{
    const int s = pl.s ? pl.s : pl.T;
    int have = pl.scratch_segment();
    for (int j = (pl.T - 1) / s; j >= 0; --j) {
        const int a = j * s, e = std::min(a + s, pl.T) - 1;
        if (pl.s && e > a && j != have) {
            for (int t = a; t < e; ++t) {
                const float* src = t ? u + (size_t)pl.slot(t - 1) * fb : v;
                cudaError_t err = sq(src, t ? 1.f : s0, u + (size_t)pl.slot(t) * fb);
                if (err != cudaSuccess) return err;
            }
            have = j;
        }
        for (int t = e; t >= a; --t) {
            cudaError_t err = adj(t, t ? u + (size_t)pl.slot(t - 1) * fb : v, t ? 1.f : s0);
            if (err != cudaSuccess) return err;
        }
    }
    return cudaSuccess;
}

cudaError_t exp_forward_all(const float* v, float* u, int cnt, const Vol& vol, int T, float sign,
                            cudaStream_t s)
{
    const float s0 = sign * std::ldexp(1.0f, -T);
    const float* src = v;
    float scale = s0;
    for (int t = 0; t < T; ++t) {
        float* dst = u + (size_t)t * cnt * 3 * vol.V;
        cudaError_t e = exp_square(src, scale, dst, cnt, vol, s);
        if (e != cudaSuccess) return e;
        src = dst;
        scale = 1.f;
    }
    return cudaSuccess;
}

// Exp forward keeping two slots only (atlas / labels); returns the slot of u_T
cudaError_t exp_forward_pingpong(const float* v, float* u2, int cnt, const Vol& vol, int T,
                                 float sign, cudaStream_t s, float** uT)
{
    const float s0 = sign * std::ldexp(1.0f, -T);
    const float* src = v;
    float scale = s0;
    float* dst = nullptr;
    for (int t = 0; t < T; ++t) {
        dst = u2 + (size_t)(t % 2) * cnt * 3 * vol.V;
        cudaError_t e = exp_square(src, scale, dst, cnt, vol, s);
        if (e != cudaSuccess) return e;
        src = dst;
        scale = 1.f;
    }
    *uT = dst;
    return cudaSuccess;
}

// Layout of the adjoint chain's gradient after step t: the last two
// squarings (the largest displacements, so most far sources) write
// interleaved float4 gradients for the far scatter's 16-byte atomics; the
// others and the result (t = 0) are planar, 12 bytes a voxel instead of 16.
bool adj_out4(int t, int T) { return t > 0 && t >= T - 2; }

// One adjoint step: the gather writes gout, the far scatter adds onto it.
cudaError_t exp_adjoint_step(const float* src, int src_packed, float scale, const float* gin, int in4, float* gout,
                             int out4, float out_scale, int* flags, int B, const Vol& v, cudaStream_t s)
{
    cudaError_t e = exp_adjoint_gather(src, src_packed, scale, gin, in4, gout, out4, out_scale, flags, B, v, s);
    if (e != cudaSuccess) return e;
    return exp_adjoint_far(src, src_packed, scale, gin, in4, gout, out4, out_scale, flags, B, v, s);
}

// Adjoint of Exp: gin = gT (planar); steps alternate between two
// [cnt][V] float4-sized buffers gbuf, the last one writes gv [cnt][3][V]
// (which may be gT: then a one-squaring chain goes through gbuf).  u holds
// u_1..u_T (planar, cnt fields per slot); flags: exp_far_flags ints.
cudaError_t exp_backward_all(const float* v, const float* u, const float* gT, float* gv, float4* gbuf, int* flags,
                             int cnt, const Vol& vol, int T, float sign, cudaStream_t s)
{
    const float s0 = sign * std::ldexp(1.0f, -T);
    const size_t fb = (size_t)cnt * 3 * vol.V;
    float* g4[2] = {reinterpret_cast<float*>(gbuf), reinterpret_cast<float*>(gbuf + (size_t)cnt * vol.V)};
    const float* gin = gT;
    int in4 = 0;
    for (int t = T - 1; t >= 0; --t) {
        const float* src = (t == 0) ? v : u + (size_t)(t - 1) * fb;
        const float scale = (t == 0) ? s0 : 1.f;
        const int out4 = adj_out4(t, T);
        float* gout = (t == 0 && (gv != gT || T > 1)) ? gv : g4[(T - 1 - t) % 2];
        cudaError_t e = exp_adjoint_step(src, 0, scale, gin, in4, gout, out4, scale, flags, cnt, vol, s);
        if (e != cudaSuccess) return e;
        gin = gout;
        in4 = out4;
    }
    if (gin != gv) return cudaMemcpyAsync(gv, gin, sizeof(float) * fb, cudaMemcpyDeviceToDevice, s);
    return cudaSuccess;
}

}  // namespace

// ===========================================================================
// cohort
// ===========================================================================
struct darc_cohort {
    darc_config cfg;
    int n = 0;
    Vol vol;
    const float* images = nullptr;
    cudaStream_t user = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_perm = nullptr;   // last upload of perm_host (host rewrites it after this)
    int bmax = 0;
    int sweep = 0;
    std::vector<void*> allocs;
    // state
    float *v = nullptr, *m = nullptr, *s = nullptr;
    int* k = nullptr;
    float2* bias = nullptr;
    int* flags = nullptr;
    int* nonfinite = nullptr;
    float* loss = nullptr;       // [n][2]
    float* A = nullptr;
    float* astats = nullptr;     // [2][V]
    // scratch
    float *u_all = nullptr, *gT = nullptr, *gbuf = nullptr, *Wimg = nullptr, *coef = nullptr;
    int* eflags = nullptr;       // far-source tile marks of the Exp adjoint (exp_far_flags)
    double *pL = nullptr, *pR = nullptr, *acc = nullptr, *cpart = nullptr, *cmetrics = nullptr;
    float *Wcache = nullptr, *Am = nullptr, *As = nullptr, *gA = nullptr, *aloss = nullptr;
    float *jstats = nullptr, *gsh = nullptr;   // [n][2][V] window stats of W_i; [V] shared gradient
    float* boxbuf = nullptr;                   // [max(bmax, atlas batch)][3][V] 2-D window sums
    int *perm_dev = nullptr, *iota_dev = nullptr;
    int* perm_host = nullptr;    // pinned [K3][n]
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    std::map<std::pair<int, int>, long long> graph_kernels;     // kernels per replay of each graph
    double* dpart = nullptr;                   // diffeomorphism report: block partials (allocated on first use)
    float* dstats = nullptr;                   //   and per-subject results
    float* pca_mean = nullptr;                 // PCA shape model (allocated on first use): mean velocity [3V],
    double* pca_gram = nullptr;                //   Gram partials and matrix, sampling coefficients
    float* pca_coef = nullptr;
    std::vector<double> pca_mu, pca_e;         //   Gram eigenvalues (descending), eigenvectors [n][n] by row
    std::map<std::pair<int, int>, int> seen;
    // sharded atlas SGD state
    int sgd_k = 0;
    bool sgd_open = false;
    float* gcomb = nullptr;                    // [V] combined mini-batch gradient
    // measurement
    bool profiling = false;
    long long launches = 0;
    struct Mark {
        int id;
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> spare;
};

namespace {

template <typename T>
int cohort_alloc(darc_cohort* c, T** p, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(DARC_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    *p = (T*)q;
    return DARC_OK;
}

void cohort_free(darc_cohort* c)
{
    if (!c) return;
    for (auto& mk : c->marks) { cudaEventDestroy(mk.a); cudaEventDestroy(mk.b); }
    for (auto e : c->spare) cudaEventDestroy(e);
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
    for (void* p : c->allocs) cudaFree(p);
    if (c->perm_host) cudaFreeHost(c->perm_host);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->ev_perm) cudaEventDestroy(c->ev_perm);
    if (c->st) cudaStreamDestroy(c->st);
    delete c;
}

cudaEvent_t take_event(darc_cohort* c)
{
    if (!c->spare.empty()) {
        cudaEvent_t e = c->spare.back();
        c->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// RAII bracket of one kernel-family launch (active only while profiling)
struct Prof {
    darc_cohort* c;
    cudaStream_t s;
    int id;
    double bytes;
    cudaEvent_t a = nullptr;
    Prof(darc_cohort* c_, cudaStream_t s_, int id_, double bytes_) : c(c_), s(s_), id(id_), bytes(bytes_)
    {
        if (c->profiling) {
            a = take_event(c);
            cudaEventRecord(a, s);
        }
    }
    ~Prof()
    {
        if (a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, s);
            c->marks.push_back({id, a, b, bytes});
        }
    }
};

int begin(darc_cohort* c)
{
    CK(cudaEventRecord(c->ev_in, c->user));
    CK(cudaStreamWaitEvent(c->st, c->ev_in, 0));
    return DARC_OK;
}

int end(darc_cohort* c)
{
    CK(cudaEventRecord(c->ev_out, c->st));
    CK(cudaStreamWaitEvent(c->user, c->ev_out, 0));
    return DARC_OK;
}

// the kernels of one subject step for subjects f..f+cnt-1 (Algorithm 1 body)
cudaError_t enqueue_step(darc_cohort* c, int f, int cnt, cudaStream_t s)
{
    const Vol& vol = c->vol;
    const int T = c->cfg.n_squarings;
    // u_1..u_T are packed, one float4 (z, y, x, 0) a voxel: a trilinear gather
    // of a corner's three channels is one 16-byte load; v stays planar
    const size_t fb = (size_t)cnt * 4 * vol.V;
    const double nv = (double)cnt * (double)vol.V;     // voxels of the chunk
    const float* vb = c->v + (size_t)f * 3 * vol.V;
    const float* Ib = c->images + (size_t)f * vol.V;
    cudaError_t e = cudaSuccess;
    const float s0 = std::ldexp(1.0f, -T);
    const CkPlan plan(T, c->cfg.checkpoint_stride);
    // adjoint outputs: one [cnt][V] float4-sized buffer per squaring (gbuf
    // slot t for step t).  The gather adjoint writes every voxel; the
    // scatter adjoint adds into a slot that its forward squaring cleared.
    const bool gather = c->cfg.adjoint == DARC_ADJOINT_GATHER;
    float4* const g4 = reinterpret_cast<float4*>(c->gbuf);
    auto gslot = [&](int t) { return g4 + (size_t)t * cnt * vol.V; };
    auto sq = [&](const float* src, float scale, float* dst) {
        Prof p(c, s, DARC_K_EXP_SQUARE, 24.0 * nv);
        c->launches += 1;
        return exp_square_packed(src, src != vb, scale, reinterpret_cast<float4*>(dst), cnt, vol, s);
    };
    int tf = 0;
    auto sq_clear = [&](const float* src, float scale, float* dst) {
        Prof p(c, s, DARC_K_EXP_SQUARE, 24.0 * nv);
        c->launches += 1;
        return exp_square_packed(src, src != vb, scale, reinterpret_cast<float4*>(dst), cnt, vol, s, gslot(tf++));
    };
    e = gather ? exp_forward_plan(plan, vb, c->u_all, fb, s0, sq) : exp_forward_plan(plan, vb, c->u_all, fb, s0, sq_clear);
    if (e != cudaSuccess) return e;
    const float* uT = c->u_all + (size_t)plan.slot(T - 1) * fb;
    const double *pLp, *pRp;
    int nL, nR, sL, sR;
    if (pointwise(c->cfg.dissim)) {
        Prof p(c, s, DARC_K_MSE_WARP_REG, 32.0 * nv);
        e = mse_warp_reg(Ib, vol.V, c->A, uT, c->cfg.lambda, c->gT, c->pL, cnt, vol, c->cfg.dissim == DARC_L1, s, 1);
        pLp = c->pL; pRp = c->pL + 1; nL = nR = voxel_blocks(vol); sL = sR = 2;
        c->launches += 1;
    } else {
        const int r = c->cfg.ncc_window / 2;
        {
            Prof p(c, s, DARC_K_WARP, 20.0 * nv);
            e = warp_packed(Ib, vol.V, reinterpret_cast<const float4*>(uT), c->Wimg, cnt, vol, s);
        }
        if (e == cudaSuccess) {
            Prof p(c, s, DARC_K_LNCC_FWD, 28.0 * nv);
            e = lncc_forward(c->Wimg, nullptr, c->A, c->astats, r, c->cfg.ncc_eps, 0, patch_metric(c->cfg.dissim),
                             c->coef, c->pL, cnt, vol, c->boxbuf, s);
        }
        if (e == cudaSuccess) {
            Prof p(c, s, DARC_K_LNCC_BWD_WARP_REG, 48.0 * nv);
            e = lncc_backward_warp_reg(c->Wimg, c->A, c->coef, r, Ib, vol.V, uT, c->cfg.lambda, c->gT,
                                       c->pR, cnt, vol, c->boxbuf, s, 1);
        }
        pLp = c->pL; pRp = c->pR; nL = nR = box_blocks(vol, cnt); sL = sR = 1;
        c->launches += 5;           // warp, two box passes of two kernels each
    }
    if (e != cudaSuccess) return e;
    e = finish_step(pLp, nL, sL, pRp, nR, sR, c->loss + 2 * f, c->flags + f, c->k + f, c->bias + f,
                    c->nonfinite, c->cfg.lr, c->cfg.beta1, c->cfg.beta2, cnt, s);
    if (e != cudaSuccess) return e;
    // the adjoint chain: gT (planar) is its input; step t writes gbuf slot t
    // (interleaved or planar, adj_out4), the last one (planar) feeds Adam
    const float* gv = nullptr;
    int gv4 = 0;
    {
        const float* gin = c->gT;
        int in4 = 0;
        auto adj = [&](int t, const float* src, float scale) {
            float* gout = reinterpret_cast<float*>(gslot(t));
            cudaError_t err;
            if (!gather) {
                // interleaved gradients, one 16-byte atomic per scattered corner
                Prof p(c, s, DARC_K_EXP_ADJOINT, 36.0 * nv);
                c->launches += 1;
                err = exp_square_adjoint4(src, t != 0, scale, gin, in4, gslot(t), scale, cnt, vol, s);
                gin = gout;
                in4 = 1;
                gv = gout;
                gv4 = 1;
                return err;
            }
            const int out4 = adj_out4(t, T);
            {
                Prof p(c, s, DARC_K_EXP_ADJOINT, 36.0 * nv);
                err = exp_adjoint_gather(src, t != 0, scale, gin, in4, gout, out4, scale, c->eflags, cnt, vol, s);
            }
            if (err == cudaSuccess) {
                Prof p(c, s, DARC_K_EXP_FAR, 0.0);
                err = exp_adjoint_far(src, t != 0, scale, gin, in4, gout, out4, scale, c->eflags, cnt, vol, s);
            }
            c->launches += 2;
            gin = gout;
            in4 = out4;
            gv = gout;
            gv4 = out4;
            return err;
        };
        e = exp_backward_plan(plan, vb, c->u_all, fb, s0, sq, adj);
    }
    if (e != cudaSuccess) return e;
    Prof p(c, s, DARC_K_ADAM, 84.0 * nv);
    c->launches += 2;
    float* vf = c->v + (size_t)f * 3 * vol.V;
    float* mf = c->m + (size_t)f * 3 * vol.V;
    float* sf = c->s + (size_t)f * 3 * vol.V;
    if (gv4)
        return adam_fields_g4(vf, mf, sf, reinterpret_cast<const float4*>(gv), c->bias + f, c->flags + f,
                              c->cfg.beta1, c->cfg.beta2, c->cfg.adam_eps, cnt, vol.V, s);
    return adam_fields(vf, mf, sf, gv, 1.f, c->bias + f, c->flags + f, c->cfg.beta1, c->cfg.beta2, c->cfg.adam_eps,
                       cnt, 3 * vol.V, s);
}

int run_steps(darc_cohort* c, int first, int count, int steps)
{
    for (int f = first; f < first + count; f += c->bmax) {
        const int cnt = std::min(c->bmax, first + count - f);
        const auto key = std::make_pair(f, cnt);
        int done = 0;
        if (c->profiling) {
            for (int st = 0; st < steps; ++st) CK(enqueue_step(c, f, cnt, c->st));
            continue;
        }
        if (!c->seen.count(key)) {
            // first use of this chunk: launch directly (sets kernel attributes outside capture)
            CK(enqueue_step(c, f, cnt, c->st));
            c->seen[key] = 1;
            done = 1;
        }
        if (done >= steps) continue;
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ex = nullptr;
            CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
            const long long before = c->launches;
            cudaError_t e = enqueue_step(c, f, cnt, c->st);
            c->graph_kernels[key] = c->launches - before;   // kernels one replay launches
            c->launches = before;                           // recording launches nothing
            cudaError_t e2 = cudaStreamEndCapture(c->st, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return fail(DARC_ERR_CUDA, std::string("graph capture failed: ") +
                                               cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            CK(e);
            it = c->graphs.emplace(key, ex).first;
        }
        const long long per_step = c->graph_kernels[key];
        for (int s = done; s < steps; ++s) {
            CK(cudaGraphLaunch(it->second, c->st));
            c->launches += per_step;
        }
    }
    return DARC_OK;
}

int update_atlas_body(darc_cohort* c);

int update_atlas_impl(darc_cohort* c)
{
    const Vol& vol = c->vol;
    const int T = c->cfg.n_squarings, n = c->n, K3 = c->cfg.atlas_epochs;
    // algorithmic bytes: centrality 24n + 12 per voxel; warped cohort (24T + 20) n;
    // L1 median: the cached cohort read once, the atlas written; patch-wise:
    // the cohort's window statistics 12n, then per mini-batch of nb subjects
    // either the fused passes (Adam state 24, the two shared coefficients
    // written and read 16, per subject 24: J twice, its statistics, its
    // coefficient written and read; per sub-batch after the first 28: A read,
    // the shared coefficients read and written again, the running gradient
    // written and read) or the unfused chain (statistics 12, Adam 24, per
    // subject 28 + 20)
    double bytes = (24.0 * n + 12.0) + (24.0 * T + 20.0) * n;
    if (c->cfg.dissim == DARC_L1) bytes += 4.0 * n + 4.0;
    const long long chunks = (n + c->bmax - 1) / c->bmax;
    long long launches = 2 + chunks * (T + 1) + 1;
    if (patchwise(c->cfg.dissim)) {
        // per mini-batch: fused 2 per sub-batch + 1 + 2 per sub-batch kernels,
        // unfused 2 + 2 + 1 + 4 + 1
        bytes += 12.0 * n;
        launches += 2 * chunks + 1;
        for (int b0 = 0; b0 < n; b0 += c->cfg.atlas_batch) {
            const int nb = std::min(c->cfg.atlas_batch, n - b0);
            const bool fused = nb <= ATLAS_FUSED_MAX;
            const int K = atlas_sub_batches(nb);
            bytes += K3 * (fused ? 40.0 + 24.0 * nb + 28.0 * (K - 1) : 36.0 + 48.0 * nb);
            launches += (long long)K3 * (fused ? 4 * K + 1 : 10);
        }
    }
    Prof p(c, c->st, DARC_K_ATLAS, bytes * (double)vol.V);
    c->launches += launches;
    return update_atlas_body(c);
}

int update_atlas_body(darc_cohort* c)
{
    const Vol& vol = c->vol;
    const int T = c->cfg.n_squarings, n = c->n;
    cudaStream_t s = c->st;
    CK(centrality(c->v, n, vol, c->cpart, c->cmetrics, s));
    if (c->cfg.dissim == DARC_MSE) {
        CK(cudaMemsetAsync(c->acc, 0, sizeof(double) * vol.V, s));
        for (int f = 0; f < n; f += c->bmax) {
            const int cnt = std::min(c->bmax, n - f);
            float* uT = nullptr;
            CK(exp_forward_pingpong(c->v + (size_t)f * 3 * vol.V, c->u_all, cnt, vol, T, 1.f, s, &uT));
            CK(warp_accumulate(c->images, c->iota_dev + f, uT, c->acc, cnt, vol, s));
        }
        CK(finalize_mean(c->acc, 1.0 / n, c->A, vol, s));
        return DARC_OK;
    }
    // L1 and patch-wise: cache W_i = I_i o Exp(hat v_i)
    for (int f = 0; f < n; f += c->bmax) {
        const int cnt = std::min(c->bmax, n - f);
        float* uT = nullptr;
        CK(exp_forward_pingpong(c->v + (size_t)f * 3 * vol.V, c->u_all, cnt, vol, T, 1.f, s, &uT));
        CK(warp(c->images + (size_t)f * vol.V, vol.V, uT, c->Wcache + (size_t)f * vol.V, cnt, vol, s));
    }
    if (c->cfg.dissim == DARC_L1) {
        // closed form: the voxel-wise median of the warped cohort
        CK(median(c->Wcache, n, vol.V, c->A, s));
        return DARC_OK;
    }
    // patch-wise: K3 epochs of mini-batch Adam on A
    const int K3 = c->cfg.atlas_epochs, B = c->cfg.atlas_batch, r = c->cfg.ncc_window / 2;
    if (K3 > 0) {
        // Box(W_i), Box(W_i^2) do not depend on A: once per atlas update
        for (int f = 0; f < n; f += c->bmax) {
            const int cnt = std::min(c->bmax, n - f);
            CK(image_stats(c->Wcache + (size_t)f * vol.V, c->jstats + (size_t)f * 2 * vol.V, cnt, r, vol,
                           c->boxbuf, s));
        }
        CK(cudaEventSynchronize(c->ev_perm));   // the previous upload has left perm_host
        for (int ep = 0; ep < K3; ++ep) minibatch_order(c->cfg.seed, c->sweep, ep, n, c->perm_host + (size_t)ep * n);
        CK(cudaMemcpyAsync(c->perm_dev, c->perm_host, sizeof(int) * (size_t)K3 * n, cudaMemcpyHostToDevice, s));
        CK(cudaEventRecord(c->ev_perm, s));
        CK(cudaMemsetAsync(c->Am, 0, sizeof(float) * vol.V, s));
        CK(cudaMemsetAsync(c->As, 0, sizeof(float) * vol.V, s));
        int kk = 0;
        for (int ep = 0; ep < K3; ++ep) {
            for (int b0 = 0; b0 < n; b0 += B) {
                const int nb = std::min(B, n - b0);
                if (nb <= ATLAS_FUSED_MAX) {
                    // per sub-batch two box passes: the metrics with Box(A), Box(A^2);
                    // the adjoint, the last with the Adam step (subject rows from the
                    // host's order)
                    const int* sh = c->perm_host + (size_t)ep * n + b0;
                    const float* Jr[ATLAS_FUSED_MAX];
                    const float* jr[ATLAS_FUSED_MAX];
                    for (int b = 0; b < nb; ++b) {
                        Jr[b] = c->Wcache + (size_t)sh[b] * vol.V;
                        jr[b] = c->jstats + (size_t)sh[b] * 2 * vol.V;
                    }
                    CK(atlas_sgd_fused_forward(Jr, jr, nb, c->A, r, c->cfg.ncc_eps, patch_metric(c->cfg.dissim),
                                               c->coef, c->pL, vol, c->boxbuf, s));
                    CK(reduce_partials(c->pL, box_blocks(vol, 1), 1, 1.0, c->aloss + (size_t)ep * n + b0, 1, nb, s));
                    ++kk;
                    const double c1 = 1.0 - std::pow((double)c->cfg.beta1, kk);
                    const double c2 = 1.0 - std::pow((double)c->cfg.beta2, kk);
                    CK(atlas_sgd_fused_adam(Jr, nb, c->coef, r, c->A, c->Am, c->As,
                                            (float)(-1.0 / ((double)vol.V * nb)), (float)(c->cfg.lr / c1),
                                            (float)(1.0 / std::sqrt(c2)), c->cfg.beta1, c->cfg.beta2,
                                            c->cfg.adam_eps, c->gsh, vol, c->boxbuf, s));
                    continue;
                }
                const int* subj = c->perm_dev + (size_t)ep * n + b0;
                CK(atlas_stats(c->A, c->astats, r, vol, c->boxbuf, s));
                CK(atlas_sgd_forward(c->Wcache, c->jstats, subj, c->A, c->astats, r, c->cfg.ncc_eps,
                                     patch_metric(c->cfg.dissim), c->coef,
                                     c->pL, nb, vol, c->boxbuf, s));
                CK(reduce_partials(c->pL, box_blocks(vol, nb), 1, 1.0, c->aloss + (size_t)ep * n + b0, 1, nb, s));
                CK(atlas_sgd_backward(c->Wcache, subj, c->A, c->coef, r, c->gsh, c->gA, nb, vol, c->boxbuf, s));
                ++kk;
                const double c1 = 1.0 - std::pow((double)c->cfg.beta1, kk);
                const double c2 = 1.0 - std::pow((double)c->cfg.beta2, kk);
                // mean over the batch of dL_i/dA = -1/V [gshared + sum_b gsubj_b] / nb
                CK(atlas_adam(c->A, c->Am, c->As, c->gsh, c->gA, nb, (float)(-1.0 / ((double)vol.V * nb)),
                              (float)(c->cfg.lr / c1), (float)(1.0 / std::sqrt(c2)), c->cfg.beta1,
                              c->cfg.beta2, c->cfg.adam_eps, vol, s));
            }
        }
    }
    CK(atlas_stats(c->A, c->astats, r, vol, c->boxbuf, s));
    return DARC_OK;
}

// Eigenpairs of a symmetric n x n matrix by cyclic Jacobi rotations (Jacobi
// 1846; Golub & Van Loan, Matrix Computations, Sec. 8.5): each rotation
// zeroes one off-diagonal pair; sweeps run until the off-diagonal mass is
// below 1e-30 of the total.  On return mu[k] (descending) and e[k][i] (row k
// an eigenvector), each eigenvector signed so that its entry of largest
// magnitude (the first such) is positive.
void sym_eigen(std::vector<double> a, int n, std::vector<double>& mu, std::vector<double>& e)
{
    std::vector<double> V((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto A = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
    double total = 0.0;
    for (double x : a) total += x * x;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (i != j) off += A(i, j) * A(i, j);
        if (off <= 1e-30 * total || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (A(p, q) == 0.0) continue;
                const double theta = (A(q, q) - A(p, p)) / (2.0 * A(p, q));
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {          // columns p, q
                    const double akp = A(k, p), akq = A(k, q);
                    A(k, p) = cs * akp - sn * akq;
                    A(k, q) = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {          // rows p, q
                    const double apk = A(p, k), aqk = A(q, k);
                    A(p, k) = cs * apk - sn * aqk;
                    A(q, k) = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {          // eigenvectors are the columns of V
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = cs * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return A(x, x) > A(y, y); });
    mu.assign(n, 0.0);
    e.assign((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k) {
        const int col = order[k];
        mu[k] = A(col, col);
        int big = 0;
        for (int i = 1; i < n; ++i)
            if (std::fabs(V[(size_t)i * n + col]) > std::fabs(V[(size_t)big * n + col])) big = i;
        const double sg = V[(size_t)big * n + col] < 0 ? -1.0 : 1.0;
        for (int i = 0; i < n; ++i) e[(size_t)k * n + i] = sg * V[(size_t)i * n + col];
    }
}

int fill_atlas_stats(darc_cohort* c, darc_sweep_stats* stats)
{
    double m[2] = {0, 0};
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemcpy(m, c->cmetrics, sizeof(m), cudaMemcpyDeviceToHost));
    stats->centrality_before = m[0];
    stats->centrality_after = m[1];
    stats->atlas_loss = 0.0;
    if (patchwise(c->cfg.dissim) && c->cfg.atlas_epochs > 0) {
        std::vector<float> al(c->n);
        CK(cudaMemcpy(al.data(), c->aloss + (size_t)(c->cfg.atlas_epochs - 1) * c->n, sizeof(float) * c->n,
                      cudaMemcpyDeviceToHost));
        double t = 0;
        for (float x : al) t += x;
        stats->atlas_loss = t / c->n;
    }
    return DARC_OK;
}

}  // namespace

namespace darc_impl {
int report_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace darc_impl

extern "C" {

void darc_default_config(darc_config* c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->dissim = DARC_LNCC;
    c->ncc_window = 9;
    c->n_squarings = 7;
    c->lambda = 1.0f;
    c->lr = 1e-2f;
    c->beta1 = 0.9f;
    c->beta2 = 0.999f;
    c->adam_eps = 1e-8f;
    c->ncc_eps = 1e-5f;
    c->inner_steps = 10;
    c->atlas_epochs = 20;
    c->atlas_batch = 4;
}

const char* darc_last_error(void) { return g_err.c_str(); }

const char* darc_version(void) { return "darc-gb300 0.1 (sm_103a)"; }

int darc_init_cohort(darc_cohort** out, const darc_config* cfg, int n, int D, int H, int W,
                     const float* images_dev, void* stream)
{
    if (!out || !images_dev) return fail(DARC_ERR_ARG, "null argument");
    *out = nullptr;
    int rc = check_dims(1, D, H, W);
    if (rc) return rc;
    if (n < 1) return fail(DARC_ERR_ARG, "n must be >= 1");
    rc = check_config(cfg, D, H, W);
    if (rc) return rc;
    darc_cohort* c = new darc_cohort();
    c->cfg = *cfg;
    c->n = n;
    c->vol = make_vol(D, H, W);
    c->images = images_dev;
    c->user = (cudaStream_t)stream;
    c->bmax = (cfg->subject_batch > 0) ? std::min(cfg->subject_batch, n) : n;
    rc = check_dims(c->bmax, D, H, W);
    if (!rc && cfg->dissim == DARC_L1 && median_threads(n) == 0)
        rc = fail(DARC_ERR_ARG, "the L1 (median) atlas supports at most 1600 subjects per cohort");
    if (rc) { delete c; return rc; }
    const Vol& v = c->vol;
    const int T = cfg->n_squarings;
    const size_t F = 3 * (size_t)v.V;
    const int bsub = std::max(c->bmax, cfg->atlas_batch);
    const int nb = nblk_max(v);
#define ALLOC(ptr, cnt)                      \
    do {                                     \
        int r_ = cohort_alloc(c, &(ptr), (cnt)); \
        if (r_) { cohort_free(c); return r_; } \
    } while (0)
    if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_perm, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cohort_free(c);
        return fail(DARC_ERR_CUDA, "stream/event creation failed");
    }
    ALLOC(c->v, F * n);
    ALLOC(c->m, F * n);
    ALLOC(c->s, F * n);
    ALLOC(c->k, n);
    ALLOC(c->bias, n);
    ALLOC(c->flags, n);
    ALLOC(c->nonfinite, 1);
    ALLOC(c->loss, 2 * (size_t)n);
    ALLOC(c->A, v.V);
    // packed squaring fields of the subject step (4V floats each); also two
    // planar slots for the atlas's Exp
    ALLOC(c->u_all, 4 * (size_t)v.V * c->bmax * std::max(CkPlan(T, cfg->checkpoint_stride).fields(), 2));
    ALLOC(c->gT, F * c->bmax);
    // one interleaved float4 gradient set per squaring (at least two planar
    // field slots for the inverse-map scratch of the diffeomorphism report)
    ALLOC(c->gbuf, 4 * (size_t)v.V * c->bmax * std::max(T, 2));
    ALLOC(c->eflags, exp_far_flags(c->bmax, v));
    ALLOC(c->pL, 2 * (size_t)nb * bsub);
    ALLOC(c->pR, (size_t)nb * bsub);
    ALLOC(c->acc, v.V);
    ALLOC(c->cpart, 2 * (size_t)centrality_blocks(v));
    ALLOC(c->cmetrics, 2);
    ALLOC(c->iota_dev, n);
    if (cfg->dissim == DARC_L1) ALLOC(c->Wcache, (size_t)v.V * n);
    if (patchwise(cfg->dissim)) {
        ALLOC(c->astats, 2 * v.V);
        ALLOC(c->boxbuf, 3 * (size_t)v.V * bsub);
        ALLOC(c->Wimg, (size_t)v.V * c->bmax);
        ALLOC(c->coef, 3 * (size_t)v.V * bsub);
        ALLOC(c->Wcache, (size_t)v.V * n);
        ALLOC(c->Am, v.V);
        ALLOC(c->As, v.V);
        ALLOC(c->gA, (size_t)v.V * cfg->atlas_batch);
        ALLOC(c->gsh, (size_t)v.V);
        ALLOC(c->gcomb, (size_t)v.V);
        ALLOC(c->jstats, 2 * (size_t)v.V * n);
        ALLOC(c->aloss, (size_t)std::max(cfg->atlas_epochs, 1) * n);
        ALLOC(c->perm_dev, (size_t)std::max(cfg->atlas_epochs, 1) * n);
        if (cudaMallocHost(&c->perm_host, sizeof(int) * (size_t)std::max(cfg->atlas_epochs, 1) * n) != cudaSuccess) {
            cudaGetLastError();
            c->perm_host = nullptr;
            cohort_free(c);
            return fail(DARC_ERR_OOM, "pinned allocation failed");
        }
    }
#undef ALLOC
    cudaStream_t s = c->st;
    std::vector<int> iota(n);
    for (int i = 0; i < n; ++i) iota[i] = i;
    const bool ok =
        cudaEventRecord(c->ev_in, c->user) == cudaSuccess && cudaStreamWaitEvent(s, c->ev_in, 0) == cudaSuccess &&
        cudaMemcpyAsync(c->iota_dev, iota.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s) == cudaSuccess &&
        cudaMemsetAsync(c->v, 0, sizeof(float) * F * n, s) == cudaSuccess &&
        cudaMemsetAsync(c->m, 0, sizeof(float) * F * n, s) == cudaSuccess &&
        cudaMemsetAsync(c->s, 0, sizeof(float) * F * n, s) == cudaSuccess &&
        cudaMemsetAsync(c->k, 0, sizeof(int) * n, s) == cudaSuccess &&
        cudaMemsetAsync(c->flags, 0, sizeof(int) * n, s) == cudaSuccess &&
        cudaMemsetAsync(c->eflags, 0, sizeof(int) * exp_far_flags(c->bmax, v), s) == cudaSuccess &&
        cudaMemsetAsync(c->nonfinite, 0, sizeof(int), s) == cudaSuccess &&
        cudaMemsetAsync(c->loss, 0, sizeof(float) * 2 * n, s) == cudaSuccess &&
        cudaMemsetAsync(c->cmetrics, 0, sizeof(double) * 2, s) == cudaSuccess &&
        image_mean_accumulate(images_dev, n, c->acc, v, s) == cudaSuccess &&
        finalize_mean(c->acc, 1.0 / n, c->A, v, s) == cudaSuccess &&
        (!patchwise(cfg->dissim) || atlas_stats(c->A, c->astats, cfg->ncc_window / 2, v, c->boxbuf, s) == cudaSuccess) &&
        cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) {
        cudaError_t e = cudaGetLastError();
        cohort_free(c);
        return fail(DARC_ERR_CUDA, std::string("cohort initialisation failed: ") + cudaGetErrorString(e));
    }
    *out = c;
    return DARC_OK;
}

int darc_subject_step(darc_cohort* c, int first, int count, int steps, float* loss_host)
{
    if (!c) return fail(DARC_ERR_ARG, "null cohort");
    if (first < 0 || count < 1 || first + count > c->n || steps < 0)
        return fail(DARC_ERR_ARG, "subject range or step count out of bounds");
    if (steps == 0) return DARC_OK;
    int rc = begin(c);
    if (rc) return rc;
    rc = run_steps(c, first, count, steps);
    if (rc) return rc;
    rc = end(c);
    if (rc) return rc;
    if (loss_host) {
        std::vector<float> l(2 * (size_t)count);
        std::vector<int> fl(count);
        CK(cudaStreamSynchronize(c->st));
        CK(cudaMemcpy(l.data(), c->loss + 2 * (size_t)first, sizeof(float) * 2 * count, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(fl.data(), c->flags + first, sizeof(int) * count, cudaMemcpyDeviceToHost));
        int bad = 0;
        for (int i = 0; i < count; ++i) {
            loss_host[i] = l[2 * i] + c->cfg.lambda * l[2 * i + 1];
            bad += fl[i] != 0;
        }
        if (bad) return fail(DARC_ERR_NONFINITE, std::to_string(bad) + " subject(s) had a non-finite loss");
    }
    return DARC_OK;
}

int darc_update_atlas(darc_cohort* c, darc_sweep_stats* stats)
{
    if (!c) return fail(DARC_ERR_ARG, "null cohort");
    int rc = begin(c);
    if (rc) return rc;
    rc = update_atlas_impl(c);
    if (rc) return rc;
    rc = end(c);
    if (rc) return rc;
    if (stats) return fill_atlas_stats(c, stats);
    return DARC_OK;
}

int darc_sweep(darc_cohort* c, darc_sweep_stats* stats)
{
    if (!c) return fail(DARC_ERR_ARG, "null cohort");
    int rc = begin(c);
    if (rc) return rc;
    const size_t F = 3 * (size_t)c->vol.V * c->n;
    if (c->cfg.reset_each_sweep) {
        CK(cudaMemsetAsync(c->v, 0, sizeof(float) * F, c->st));
        CK(cudaMemsetAsync(c->m, 0, sizeof(float) * F, c->st));
        CK(cudaMemsetAsync(c->s, 0, sizeof(float) * F, c->st));
        CK(cudaMemsetAsync(c->k, 0, sizeof(int) * c->n, c->st));
    }
    rc = run_steps(c, 0, c->n, c->cfg.inner_steps);
    if (rc) return rc;
    rc = update_atlas_impl(c);
    if (rc) return rc;
    rc = end(c);
    if (rc) return rc;
    c->sweep += 1;
    int nonfinite = 0;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        rc = fill_atlas_stats(c, stats);
        if (rc) return rc;
        std::vector<float> l(2 * (size_t)c->n);
        CK(cudaMemcpy(l.data(), c->loss, sizeof(float) * 2 * c->n, cudaMemcpyDeviceToHost));
        double L = 0, R = 0;
        for (int i = 0; i < c->n; ++i) { L += l[2 * i]; R += l[2 * i + 1]; }
        stats->loss_data = L / c->n;
        stats->loss_reg = R / c->n;
        CK(cudaMemcpy(&nonfinite, c->nonfinite, sizeof(int), cudaMemcpyDeviceToHost));
        CK(cudaMemset(c->nonfinite, 0, sizeof(int)));
        stats->nonfinite_subjects = nonfinite;
        if (nonfinite) return fail(DARC_ERR_NONFINITE, std::to_string(nonfinite) + " subject step(s) had a non-finite loss");
    }
    return DARC_OK;
}

int darc_sweep_losses(darc_cohort* c, float* out_dev)
{
    if (!c || !out_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = begin(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(out_dev, c->loss, sizeof(float) * 2 * (size_t)c->n, cudaMemcpyDeviceToDevice, c->st));
    return end(c);
}

int darc_propagate_labels(darc_cohort* c, const uint8_t* labels_dev, uint8_t* out_dev, int first, int count)
{
    if (!c || !labels_dev || !out_dev) return fail(DARC_ERR_ARG, "null argument");
    if (first < 0 || count < 1 || first + count > c->n) return fail(DARC_ERR_ARG, "subject range out of bounds");
    int rc = begin(c);
    if (rc) return rc;
    const Vol& vol = c->vol;
    for (int f = first; f < first + count; f += c->bmax) {
        const int cnt = std::min(c->bmax, first + count - f);
        float* uT = nullptr;
        CK(exp_forward_pingpong(c->v + (size_t)f * 3 * vol.V, c->u_all, cnt, vol, c->cfg.n_squarings, -1.f, c->st, &uT));
        CK(label_gather(labels_dev, uT, out_dev + (size_t)(f - first) * vol.V, cnt, vol, c->st));
    }
    return end(c);
}

int darc_diffeo_report(darc_cohort* c, int first, int count, float* stats_host)
{
    if (!c || !stats_host) return fail(DARC_ERR_ARG, "null argument");
    if (first < 0 || count < 1 || first + count > c->n) return fail(DARC_ERR_ARG, "subject range out of bounds");
    const Vol& vol = c->vol;
    if (!c->dpart) {
        void* p = nullptr;
        if (cudaMalloc(&p, sizeof(double) * 4 * (size_t)voxel_blocks(vol) * c->bmax) != cudaSuccess) {
            cudaGetLastError();
            return fail(DARC_ERR_OOM, "cudaMalloc failed");
        }
        c->allocs.push_back(p);
        c->dpart = (double*)p;
        if (cudaMalloc(&p, sizeof(float) * 4 * (size_t)c->bmax) != cudaSuccess) {
            cudaGetLastError();
            return fail(DARC_ERR_OOM, "cudaMalloc failed");
        }
        c->allocs.push_back(p);
        c->dstats = (float*)p;
    }
    int rc = begin(c);
    if (rc) return rc;
    const int T = c->cfg.n_squarings;
    for (int f = first; f < first + count; f += c->bmax) {
        const int cnt = std::min(c->bmax, first + count - f);
        const float* vb = c->v + (size_t)f * 3 * vol.V;
        float *up = nullptr, *um = nullptr;
        CK(exp_forward_pingpong(vb, c->u_all, cnt, vol, T, 1.f, c->st, &up));
        CK(exp_forward_pingpong(vb, c->gbuf, cnt, vol, T, -1.f, c->st, &um));
        CK(compose(up, um, c->gT, cnt, vol, c->st));
        CK(diffeo_stats(up, c->gT, c->dpart, c->dstats, cnt, vol, c->st));
        CK(cudaMemcpyAsync(stats_host + 4 * (size_t)(f - first), c->dstats, sizeof(float) * 4 * cnt,
                           cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    return end(c);
}

int darc_shape_pca(darc_cohort* c, double* eigvals_host, double* weights_host)
{
    if (!c || !eigvals_host) return fail(DARC_ERR_ARG, "null argument");
    const int n = c->n;
    if (n < 2) return fail(DARC_ERR_ARG, "PCA needs at least two subjects");
    const long long M = 3 * c->vol.V;
    if (!c->pca_mean) {
        void* p = nullptr;
        const size_t bytes[3] = {sizeof(float) * (size_t)M,
                                 sizeof(double) * ((size_t)gram_splits(n) + 1) * n * n,
                                 sizeof(float) * 8 * (size_t)n};
        void** dst[3] = {(void**)&c->pca_mean, (void**)&c->pca_gram, (void**)&c->pca_coef};
        for (int k = 0; k < 3; ++k) {
            if (cudaMalloc(&p, bytes[k]) != cudaSuccess) {
                cudaGetLastError();
                return fail(DARC_ERR_OOM, "cudaMalloc failed");
            }
            c->allocs.push_back(p);
            *dst[k] = p;
        }
    }
    int rc = begin(c);
    if (rc) return rc;
    double* G = c->pca_gram + (size_t)gram_splits(n) * n * n;
    CK(field_mean(c->v, n, M, c->pca_mean, c->st));
    CK(gram(c->v, c->pca_mean, n, M, c->pca_gram, G, c->st));
    std::vector<double> Gh((size_t)n * n);
    CK(cudaMemcpyAsync(Gh.data(), G, sizeof(double) * n * n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    sym_eigen(Gh, n, c->pca_mu, c->pca_e);
    for (int k = 0; k < n; ++k) eigvals_host[k] = std::max(c->pca_mu[k], 0.0) / (double)(n - 1);
    if (weights_host) std::memcpy(weights_host, c->pca_e.data(), sizeof(double) * n * n);
    return end(c);
}

int darc_sym_eigen(const double* a_host, int n, double* mu_host, double* e_host)
{
    if (!a_host || !mu_host || !e_host) return fail(DARC_ERR_ARG, "null argument");
    if (n < 1 || n > 4096) return fail(DARC_ERR_ARG, "n must be 1..4096");
    std::vector<double> mu, e;
    sym_eigen(std::vector<double>(a_host, a_host + (size_t)n * n), n, mu, e);
    std::memcpy(mu_host, mu.data(), sizeof(double) * n);
    std::memcpy(e_host, e.data(), sizeof(double) * (size_t)n * n);
    return DARC_OK;
}

int darc_shape_sample(darc_cohort* c, const double* z_host, int m, int p, float* v_out_dev)
{
    if (!c || !z_host || !v_out_dev) return fail(DARC_ERR_ARG, "null argument");
    const int n = c->n;
    if (c->pca_mu.empty()) return fail(DARC_ERR_ARG, "call darc_shape_pca first");
    if (m < 1 || p < 0 || p > n - 1) return fail(DARC_ERR_ARG, "need m >= 1 and 0 <= p <= n - 1");
    const long long M = 3 * c->vol.V;
    int rc = begin(c);
    if (rc) return rc;
    // v_new = mean + sum_j sqrt(lambda_j) z_j U_j with U_j = Xc^T e_j / sqrt(mu_j) and
    // lambda_j = mu_j / (n - 1): the weight of subject i is sum_j e_j[i] z_j / sqrt(n - 1)
    std::vector<float> coef(8 * (size_t)n);
    for (int k0 = 0; k0 < m; k0 += 8) {
        const int mk = std::min(8, m - k0);
        for (int k = 0; k < mk; ++k)
            for (int i = 0; i < n; ++i) {
                double w = 0.0;
                for (int j = 0; j < p; ++j)
                    if (c->pca_mu[j] > 0.0) w += c->pca_e[(size_t)j * n + i] * z_host[(size_t)(k0 + k) * p + j];
                coef[(size_t)k * n + i] = (float)(w / std::sqrt((double)(n - 1)));
            }
        CK(cudaMemcpyAsync(c->pca_coef, coef.data(), sizeof(float) * mk * n, cudaMemcpyHostToDevice, c->st));
        CK(combine_fields(c->v, c->pca_mean, n, M, c->pca_coef, mk, v_out_dev + (size_t)k0 * M, c->st));
        CK(cudaStreamSynchronize(c->st));                 // coef is reused by the next group
    }
    return end(c);
}

int darc_get_atlas(darc_cohort* c, float* out_dev)
{
    if (!c || !out_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = begin(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(out_dev, c->A, sizeof(float) * c->vol.V, cudaMemcpyDeviceToDevice, c->st));
    return end(c);
}

int darc_set_atlas(darc_cohort* c, const float* atlas_dev)
{
    if (!c || !atlas_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = begin(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->A, atlas_dev, sizeof(float) * c->vol.V, cudaMemcpyDeviceToDevice, c->st));
    if (patchwise(c->cfg.dissim)) CK(atlas_stats(c->A, c->astats, c->cfg.ncc_window / 2, c->vol, c->boxbuf, c->st));
    return end(c);
}

int darc_get_velocity(darc_cohort* c, int i, float* out_dev)
{
    if (!c || !out_dev || i < 0 || i >= c->n) return fail(DARC_ERR_ARG, "bad argument");
    int rc = begin(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(out_dev, c->v + (size_t)i * 3 * c->vol.V, sizeof(float) * 3 * c->vol.V,
                       cudaMemcpyDeviceToDevice, c->st));
    return end(c);
}

int darc_set_velocity(darc_cohort* c, int i, const float* v_dev)
{
    if (!c || !v_dev || i < 0 || i >= c->n) return fail(DARC_ERR_ARG, "bad argument");
    int rc = begin(c);
    if (rc) return rc;
    const size_t F = 3 * (size_t)c->vol.V;
    CK(cudaMemcpyAsync(c->v + i * F, v_dev, sizeof(float) * F, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemsetAsync(c->m + i * F, 0, sizeof(float) * F, c->st));
    CK(cudaMemsetAsync(c->s + i * F, 0, sizeof(float) * F, c->st));
    CK(cudaMemsetAsync(c->k + i, 0, sizeof(int), c->st));
    return end(c);
}

int darc_get_adam_state(darc_cohort* c, int i, float* m_dev, float* s_dev, int* step_host)
{
    if (!c || i < 0 || i >= c->n) return fail(DARC_ERR_ARG, "bad argument");
    int rc = begin(c);
    if (rc) return rc;
    const size_t F = 3 * (size_t)c->vol.V;
    if (m_dev) CK(cudaMemcpyAsync(m_dev, c->m + i * F, sizeof(float) * F, cudaMemcpyDeviceToDevice, c->st));
    if (s_dev) CK(cudaMemcpyAsync(s_dev, c->s + i * F, sizeof(float) * F, cudaMemcpyDeviceToDevice, c->st));
    rc = end(c);
    if (rc) return rc;
    if (step_host) {
        CK(cudaStreamSynchronize(c->st));
        CK(cudaMemcpy(step_host, c->k + i, sizeof(int), cudaMemcpyDeviceToHost));
    }
    return DARC_OK;
}

int darc_cohort_info(darc_cohort* c, int* n, int* D, int* H, int* W, darc_config* cfg)
{
    if (!c) return fail(DARC_ERR_ARG, "null cohort");
    if (n) *n = c->n;
    if (D) *D = c->vol.D;
    if (H) *H = c->vol.H;
    if (W) *W = c->vol.W;
    if (cfg) *cfg = c->cfg;
    return DARC_OK;
}

// checkpoint format: magic, version, config, n, D, H, W, sweep, k[n], A[V],
// v, m, s [n][3][V] (all little-endian host copies)
static const char kMagic[8] = {'D', 'A', 'R', 'C', 'C', 'K', 'P', '1'};

int darc_save(darc_cohort* c, const char* path)
{
    if (!c || !path) return fail(DARC_ERR_ARG, "null argument");
    CK(cudaStreamSynchronize(c->user));
    CK(cudaStreamSynchronize(c->st));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(DARC_ERR_IO, std::string("cannot open ") + path);
    const size_t V = (size_t)c->vol.V, F = 3 * V;
    std::vector<int> k(c->n);
    std::vector<float> buf(std::max(F, V));
    bool ok = cudaMemcpy(k.data(), c->k, sizeof(int) * c->n, cudaMemcpyDeviceToHost) == cudaSuccess;
    const int hdr[5] = {c->n, c->vol.D, c->vol.H, c->vol.W, c->sweep};
    ok = ok && std::fwrite(kMagic, 1, 8, fp) == 8 && std::fwrite(&c->cfg, sizeof(darc_config), 1, fp) == 1 &&
         std::fwrite(hdr, sizeof(int), 5, fp) == 5 && std::fwrite(k.data(), sizeof(int), c->n, fp) == (size_t)c->n;
    ok = ok && cudaMemcpy(buf.data(), c->A, sizeof(float) * V, cudaMemcpyDeviceToHost) == cudaSuccess &&
         std::fwrite(buf.data(), sizeof(float), V, fp) == V;
    for (float* arr : {c->v, c->m, c->s})
        for (int i = 0; ok && i < c->n; ++i)
            ok = cudaMemcpy(buf.data(), arr + i * F, sizeof(float) * F, cudaMemcpyDeviceToHost) == cudaSuccess &&
                 std::fwrite(buf.data(), sizeof(float), F, fp) == F;
    if (std::fclose(fp) != 0) ok = false;
    if (!ok) {
        cudaGetLastError();
        return fail(DARC_ERR_IO, std::string("writing ") + path + " failed");
    }
    return DARC_OK;
}

int darc_load(darc_cohort** out, const char* path, const float* images_dev, void* stream)
{
    if (!out || !path || !images_dev) return fail(DARC_ERR_ARG, "null argument");
    *out = nullptr;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(DARC_ERR_IO, std::string("cannot open ") + path);
    char magic[8];
    darc_config cfg;
    int hdr[5];
    if (std::fread(magic, 1, 8, fp) != 8 || std::memcmp(magic, kMagic, 8) != 0 ||
        std::fread(&cfg, sizeof(cfg), 1, fp) != 1 || std::fread(hdr, sizeof(int), 5, fp) != 5) {
        std::fclose(fp);
        return fail(DARC_ERR_IO, "not a darc checkpoint");
    }
    darc_cohort* c = nullptr;
    int rc = darc_init_cohort(&c, &cfg, hdr[0], hdr[1], hdr[2], hdr[3], images_dev, stream);
    if (rc) { std::fclose(fp); return rc; }
    c->sweep = hdr[4];
    const size_t V = (size_t)c->vol.V, F = 3 * V;
    std::vector<int> k(c->n);
    std::vector<float> buf(std::max(F, V));
    bool ok = std::fread(k.data(), sizeof(int), c->n, fp) == (size_t)c->n &&
              cudaMemcpy(c->k, k.data(), sizeof(int) * c->n, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && std::fread(buf.data(), sizeof(float), V, fp) == V &&
         cudaMemcpy(c->A, buf.data(), sizeof(float) * V, cudaMemcpyHostToDevice) == cudaSuccess;
    for (float* arr : {c->v, c->m, c->s})
        for (int i = 0; ok && i < c->n; ++i)
            ok = std::fread(buf.data(), sizeof(float), F, fp) == F &&
                 cudaMemcpy(arr + i * F, buf.data(), sizeof(float) * F, cudaMemcpyHostToDevice) == cudaSuccess;
    std::fclose(fp);
    if (ok && patchwise(cfg.dissim))
        ok = atlas_stats(c->A, c->astats, cfg.ncc_window / 2, c->vol, c->boxbuf, c->st) == cudaSuccess &&
             cudaStreamSynchronize(c->st) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cohort_free(c);
        return fail(DARC_ERR_IO, std::string("reading ") + path + " failed");
    }
    *out = c;
    return DARC_OK;
}

void darc_destroy(darc_cohort* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);
    cohort_free(c);
}

// ---- sharded cohorts: halves of the exchange steps ----

int darc_velocity_sum(darc_cohort* c, float* sum_dev)
{
    if (!c || !sum_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = begin(c);
    if (rc) return rc;
    CK(field_sum(c->v, c->n, sum_dev, c->vol, c->st));
    c->launches += 1;
    return end(c);
}

int darc_centrality_apply(darc_cohort* c, const float* sum_dev, long long n_total)
{
    if (!c || !sum_dev || n_total < 1) return fail(DARC_ERR_ARG, "bad argument");
    int rc = begin(c);
    if (rc) return rc;
    CK(field_subtract(c->v, c->n, sum_dev, (float)(1.0 / (double)n_total), c->vol, c->st));
    c->launches += 1;
    return end(c);
}

int darc_atlas_partial(darc_cohort* c, double* acc_dev)
{
    if (!c || !acc_dev) return fail(DARC_ERR_ARG, "null argument");
    if (c->cfg.dissim != DARC_MSE) return fail(DARC_ERR_ARG, "a summed atlas is the MSE atlas update");
    int rc = begin(c);
    if (rc) return rc;
    const Vol& vol = c->vol;
    CK(cudaMemsetAsync(acc_dev, 0, sizeof(double) * vol.V, c->st));
    for (int f = 0; f < c->n; f += c->bmax) {
        const int cnt = std::min(c->bmax, c->n - f);
        float* uT = nullptr;
        CK(exp_forward_pingpong(c->v + (size_t)f * 3 * vol.V, c->u_all, cnt, vol, c->cfg.n_squarings, 1.f, c->st, &uT));
        CK(warp_accumulate(c->images, c->iota_dev + f, uT, acc_dev, cnt, vol, c->st));
        c->launches += c->cfg.n_squarings + 1;
    }
    return end(c);
}

int darc_atlas_set_sum(darc_cohort* c, const double* acc_dev, long long n_total)
{
    if (!c || !acc_dev || n_total < 1) return fail(DARC_ERR_ARG, "bad argument");
    if (c->cfg.dissim != DARC_MSE) return fail(DARC_ERR_ARG, "a summed atlas is the MSE atlas update");
    int rc = begin(c);
    if (rc) return rc;
    CK(finalize_mean(acc_dev, 1.0 / (double)n_total, c->A, c->vol, c->st));
    if (patchwise(c->cfg.dissim)) CK(atlas_stats(c->A, c->astats, c->cfg.ncc_window / 2, c->vol, c->boxbuf, c->st));
    return end(c);
}

int darc_atlas_batches(darc_cohort* c)
{
    if (!c) return fail(DARC_ERR_ARG, "null cohort");
    return (c->n + c->cfg.atlas_batch - 1) / c->cfg.atlas_batch;
}

int darc_atlas_sgd_begin(darc_cohort* c, int sweep, unsigned long long rank_seed)
{
    if (!c) return fail(DARC_ERR_ARG, "null cohort");
    if (!patchwise(c->cfg.dissim)) return fail(DARC_ERR_ARG, "atlas SGD is the patch-wise (NCC, SSIM) atlas update");
    int rc = begin(c);
    if (rc) return rc;
    const Vol& vol = c->vol;
    const int n = c->n, K3 = std::max(c->cfg.atlas_epochs, 1), r = c->cfg.ncc_window / 2;
    cudaStream_t s = c->st;
    for (int f = 0; f < n; f += c->bmax) {
        const int cnt = std::min(c->bmax, n - f);
        float* uT = nullptr;
        CK(exp_forward_pingpong(c->v + (size_t)f * 3 * vol.V, c->u_all, cnt, vol, c->cfg.n_squarings, 1.f, s, &uT));
        CK(warp(c->images + (size_t)f * vol.V, vol.V, uT, c->Wcache + (size_t)f * vol.V, cnt, vol, s));
        CK(image_stats(c->Wcache + (size_t)f * vol.V, c->jstats + (size_t)f * 2 * vol.V, cnt, r, vol, c->boxbuf, s));
        c->launches += c->cfg.n_squarings + 3;
    }
    CK(cudaEventSynchronize(c->ev_perm));
    for (int ep = 0; ep < K3; ++ep)
        minibatch_order(c->cfg.seed + rank_seed, sweep, ep, n, c->perm_host + (size_t)ep * n);
    CK(cudaMemcpyAsync(c->perm_dev, c->perm_host, sizeof(int) * (size_t)K3 * n, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(c->ev_perm, s));
    CK(cudaMemsetAsync(c->Am, 0, sizeof(float) * vol.V, s));
    CK(cudaMemsetAsync(c->As, 0, sizeof(float) * vol.V, s));
    c->sgd_k = 0;
    c->sgd_open = true;
    return end(c);
}

int darc_atlas_sgd_grad(darc_cohort* c, int epoch, int batch, float* g_dev, float* loss_dev)
{
    if (!c || !g_dev || !loss_dev) return fail(DARC_ERR_ARG, "null argument");
    if (!c->sgd_open) return fail(DARC_ERR_ARG, "darc_atlas_sgd_begin was not called");
    const int B = c->cfg.atlas_batch, nbatch = (c->n + B - 1) / B;
    if (epoch < 0 || epoch >= std::max(c->cfg.atlas_epochs, 1) || batch < 0 || batch >= nbatch)
        return fail(DARC_ERR_ARG, "epoch or mini-batch outside the schedule");
    int rc = begin(c);
    if (rc) return rc;
    const Vol& vol = c->vol;
    const int r = c->cfg.ncc_window / 2, b0 = batch * B, nb = std::min(B, c->n - b0);
    const int* subj = c->perm_dev + (size_t)epoch * c->n + b0;
    cudaStream_t s = c->st;
    if (nb <= ATLAS_FUSED_MAX) {
        // the single-GPU step's box passes (per sub-batch the metrics with
        // Box(A), Box(A^2) and the adjoint), the last writing g instead of
        // stepping A
        const int* sh = c->perm_host + (size_t)epoch * c->n + b0;
        const float* Jr[ATLAS_FUSED_MAX];
        const float* jr[ATLAS_FUSED_MAX];
        for (int b = 0; b < nb; ++b) {
            Jr[b] = c->Wcache + (size_t)sh[b] * vol.V;
            jr[b] = c->jstats + (size_t)sh[b] * 2 * vol.V;
        }
        CK(atlas_sgd_fused_forward(Jr, jr, nb, c->A, r, c->cfg.ncc_eps, patch_metric(c->cfg.dissim), c->coef, c->pL,
                                   vol, c->boxbuf, s));
        CK(reduce_partials(c->pL, nb * box_blocks(vol, 1), 1, 1.0, loss_dev, 1, 1, s));
        CK(atlas_sgd_fused_grad(Jr, nb, c->coef, r, c->A, (float)(-1.0 / (double)vol.V), g_dev, c->gsh, vol,
                                c->boxbuf, s));
        c->launches += 4 * atlas_sub_batches(nb) + 1;
        return end(c);
    }
    CK(atlas_stats(c->A, c->astats, r, vol, c->boxbuf, s));
    CK(atlas_sgd_forward(c->Wcache, c->jstats, subj, c->A, c->astats, r, c->cfg.ncc_eps, patch_metric(c->cfg.dissim),
                         c->coef, c->pL, nb, vol,
                         c->boxbuf, s));
    CK(reduce_partials(c->pL, nb * box_blocks(vol, nb), 1, 1.0, loss_dev, 1, 1, s));
    CK(atlas_sgd_backward(c->Wcache, subj, c->A, c->coef, r, c->gsh, c->gA, nb, vol, c->boxbuf, s));
    CK(combine_grad(c->gsh, c->gA, nb, (float)(-1.0 / (double)vol.V), g_dev, vol, s));
    c->launches += 10;
    return end(c);
}

int darc_atlas_sgd_apply(darc_cohort* c, const float* g_dev, int global_batch)
{
    if (!c || !g_dev || global_batch < 1) return fail(DARC_ERR_ARG, "bad argument");
    if (!c->sgd_open) return fail(DARC_ERR_ARG, "darc_atlas_sgd_begin was not called");
    int rc = begin(c);
    if (rc) return rc;
    c->sgd_k += 1;
    const double c1 = 1.0 - std::pow((double)c->cfg.beta1, c->sgd_k);
    const double c2 = 1.0 - std::pow((double)c->cfg.beta2, c->sgd_k);
    CK(atlas_adam(c->A, c->Am, c->As, g_dev, nullptr, 0, (float)(1.0 / global_batch), (float)(c->cfg.lr / c1),
                  (float)(1.0 / std::sqrt(c2)), c->cfg.beta1, c->cfg.beta2, c->cfg.adam_eps, c->vol, c->st));
    c->launches += 1;
    return end(c);
}

int darc_atlas_sgd_end(darc_cohort* c)
{
    if (!c) return fail(DARC_ERR_ARG, "null cohort");
    int rc = begin(c);
    if (rc) return rc;
    c->sgd_open = false;
    if (patchwise(c->cfg.dissim)) CK(atlas_stats(c->A, c->astats, c->cfg.ncc_window / 2, c->vol, c->boxbuf, c->st));
    return end(c);
}

int darc_gemm_bf16(const void* A_dev, const void* B_dev, float* C_dev, int M, int N, int K, void* stream)
{
    if (!A_dev || !B_dev || !C_dev) return fail(DARC_ERR_ARG, "null argument");
    if (M < 128 || M % 128 || N < 16 || N > 256 || N % 16 || K < 16 || K % 16)
        return fail(DARC_ERR_SHAPE, "gemm needs M % 128 == 0, N % 16 == 0 in [16, 256], K % 16 == 0");
    if (((uintptr_t)A_dev & 15) || ((uintptr_t)B_dev & 15)) return fail(DARC_ERR_ARG, "operands must be 16-byte aligned");
    CK(gemm_bf16(A_dev, B_dev, C_dev, M, N, K, (cudaStream_t)stream));
    return DARC_OK;
}

int darc_set_profiling(darc_cohort* c, int on)
{
    if (!c) return fail(DARC_ERR_ARG, "null cohort");
    c->profiling = on != 0;
    return DARC_OK;
}

int darc_profile_read(darc_cohort* c, int kernel_id, double* total_ms, long long* launches, double* bytes)
{
    if (!c || kernel_id < 0 || kernel_id >= DARC_K_COUNT) return fail(DARC_ERR_ARG, "bad argument");
    CK(cudaStreamSynchronize(c->st));
    double ms = 0.0, by = 0.0;
    long long cnt = 0;
    std::vector<darc_cohort::Mark> keep;
    for (auto& mk : c->marks) {
        if (mk.id != kernel_id) {
            keep.push_back(mk);
            continue;
        }
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, mk.a, mk.b));
        ms += t;
        by += mk.bytes;
        ++cnt;
        c->spare.push_back(mk.a);
        c->spare.push_back(mk.b);
    }
    c->marks.swap(keep);
    if (total_ms) *total_ms = ms;
    if (launches) *launches = cnt;
    if (bytes) *bytes = by;
    return DARC_OK;
}

long long darc_launch_count(darc_cohort* c) { return c ? c->launches : 0; }

// ===========================================================================
// operator API
// ===========================================================================

int darc_exp_forward(const float* v_dev, float* u_dev, int B, int D, int H, int W, int T, float sign,
                     void* stream)
{
    if (!v_dev || !u_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    if (T < 1 || T > 20) return fail(DARC_ERR_ARG, "T must be 1..20");
    CK(exp_forward_all(v_dev, u_dev, B, make_vol(D, H, W), T, sign, (cudaStream_t)stream));
    return DARC_OK;
}

size_t darc_exp_backward_workspace(int B, int D, int H, int W)
{
    return 2 * align256(sizeof(float4) * (size_t)B * D * H * W) +
           align256(sizeof(int) * exp_far_flags(B, make_vol(D, H, W)));
}

int darc_exp_backward(const float* v_dev, const float* u_dev, const float* gT_dev, float* gv_dev, void* work_dev,
                      int B, int D, int H, int W, int T, float sign, void* stream)
{
    if (!v_dev || !u_dev || !gT_dev || !gv_dev || !work_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    if (T < 1 || T > 20) return fail(DARC_ERR_ARG, "T must be 1..20");
    const Vol v = make_vol(D, H, W);
    Carve cv(work_dev);
    float4* gbuf = reinterpret_cast<float4*>(cv.take<float>(2 * 4 * (size_t)B * v.V));
    int* flags = cv.take<int>(exp_far_flags(B, v));
    // the marks only steer which tiles the far scatter visits; clearing them
    // keeps the first step from visiting every tile of a reused workspace
    CK(cudaMemsetAsync(flags, 0, sizeof(int) * exp_far_flags(B, v), (cudaStream_t)stream));
    CK(exp_backward_all(v_dev, u_dev, gT_dev, gv_dev, gbuf, flags, B, v, T, sign, (cudaStream_t)stream));
    return DARC_OK;
}

int darc_warp(const float* I_dev, int I_batch_stride_zero, const float* u_dev, float* out_dev, int B, int D, int H,
              int W, void* stream)
{
    if (!I_dev || !u_dev || !out_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    const Vol v = make_vol(D, H, W);
    CK(warp(I_dev, I_batch_stride_zero ? 0 : v.V, u_dev, out_dev, B, v, (cudaStream_t)stream));
    return DARC_OK;
}

int darc_warp_backward(const float* I_dev, int I_batch_stride_zero, const float* u_dev, const float* gW_dev,
                       float* gu_dev, int B, int D, int H, int W, void* stream)
{
    if (!I_dev || !u_dev || !gW_dev || !gu_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    const Vol v = make_vol(D, H, W);
    CK(warp_backward(I_dev, I_batch_stride_zero ? 0 : v.V, u_dev, gW_dev, gu_dev, B, v, (cudaStream_t)stream));
    return DARC_OK;
}

size_t darc_loss_workspace(int B, int D, int H, int W)
{
    const Vol v = make_vol(D, H, W);
    return align256(sizeof(double) * 2 * (size_t)B * nblk_max(v));
}

int darc_mse(const float* J_dev, const float* A_dev, float* loss_dev, float* gJ_dev, void* work_dev, int B, int D,
             int H, int W, void* stream)
{
    if (!J_dev || !A_dev || !loss_dev || !work_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    const Vol v = make_vol(D, H, W);
    cudaStream_t s = (cudaStream_t)stream;
    double* part = (double*)work_dev;
    CK(mse_partials(J_dev, A_dev, gJ_dev, part, B, v, 0, s));
    CK(reduce_partials(part, voxel_blocks(v), 1, 1.0, loss_dev, 1, B, s));
    return DARC_OK;
}

int darc_l1(const float* J_dev, const float* A_dev, float* loss_dev, float* gJ_dev, void* work_dev, int B, int D,
            int H, int W, void* stream)
{
    if (!J_dev || !A_dev || !loss_dev || !work_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    const Vol v = make_vol(D, H, W);
    cudaStream_t s = (cudaStream_t)stream;
    double* part = (double*)work_dev;
    CK(mse_partials(J_dev, A_dev, gJ_dev, part, B, v, 1, s));
    CK(reduce_partials(part, voxel_blocks(v), 1, 1.0, loss_dev, 1, B, s));
    return DARC_OK;
}

int darc_median(const float* X_dev, int n, int D, int H, int W, float* out_dev, void* stream)
{
    if (!X_dev || !out_dev) return fail(DARC_ERR_ARG, "null argument");
    if (n < 1) return fail(DARC_ERR_ARG, "n must be >= 1");
    if (median_threads(n) == 0) return fail(DARC_ERR_ARG, "n too large for the median kernel (at most 1600)");
    int rc = check_dims(1, D, H, W);
    if (rc) return rc;
    CK(median(X_dev, n, (long long)D * H * W, out_dev, (cudaStream_t)stream));
    return DARC_OK;
}

size_t darc_lncc_workspace(int B, int D, int H, int W)
{
    const Vol v = make_vol(D, H, W);
    return align256(sizeof(float) * 2 * (size_t)v.V) + align256(sizeof(float) * 3 * (size_t)B * v.V) +
           align256(sizeof(float) * (size_t)B * v.V) + darc_loss_workspace(B, D, H, W) +
           align256(sizeof(float) * 3 * (size_t)B * v.V);
}

}  // extern "C"

namespace {

// the patch-wise operator (metric 0: local NCC, 1: SSIM) with the NCC
// workspace layout
int patch_op(int metric, const float* J_dev, const float* A_dev, int window, float eps, float* loss_dev,
             float* gJ_dev, float* gA_dev, void* work_dev, int B, int D, int H, int W, void* stream)
{
    if (!J_dev || !A_dev || !loss_dev || !work_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    rc = check_window(window, D, H, W);
    if (rc) return rc;
    const Vol v = make_vol(D, H, W);
    cudaStream_t s = (cudaStream_t)stream;
    const int r = window / 2;
    Carve cv(work_dev);
    float* stats = cv.take<float>(2 * (size_t)v.V);
    float* coef = cv.take<float>(3 * (size_t)B * v.V);
    float* gAb = cv.take<float>((size_t)B * v.V);
    double* part = cv.take<double>(2 * (size_t)B * nblk_max(v));
    float* P = cv.take<float>(3 * (size_t)B * v.V);
    CK(atlas_stats(A_dev, stats, r, v, P, s));
    CK(lncc_forward(J_dev, nullptr, A_dev, stats, r, eps, 0, metric, coef, part, B, v, P, s));
    CK(reduce_partials(part, box_blocks(v, B), 1, 1.0, loss_dev, 1, B, s));
    if (gJ_dev) CK(lncc_backward(J_dev, nullptr, A_dev, coef, r, 0, gJ_dev, B, v, P, s));
    if (gA_dev) {
        CK(lncc_forward(J_dev, nullptr, A_dev, stats, r, eps, 1, metric, coef, part, B, v, P, s));
        CK(lncc_backward(J_dev, nullptr, A_dev, coef, r, 1, gAb, B, v, P, s));
        CK(sum_images(gAb, B, gA_dev, v, s));
    }
    return DARC_OK;
}

}  // namespace

extern "C" {

int darc_lncc(const float* J_dev, const float* A_dev, int window, float eps, float* loss_dev, float* gJ_dev,
              float* gA_dev, void* work_dev, int B, int D, int H, int W, void* stream)
{
    return patch_op(0, J_dev, A_dev, window, eps, loss_dev, gJ_dev, gA_dev, work_dev, B, D, H, W, stream);
}

int darc_ssim(const float* J_dev, const float* A_dev, int window, float* loss_dev, float* gJ_dev, float* gA_dev,
              void* work_dev, int B, int D, int H, int W, void* stream)
{
    return patch_op(1, J_dev, A_dev, window, 0.f, loss_dev, gJ_dev, gA_dev, work_dev, B, D, H, W, stream);
}

int darc_diffusion_reg(const float* u_dev, float* loss_dev, float* gu_dev, void* work_dev, int B, int D, int H,
                       int W, void* stream)
{
    if (!u_dev || !loss_dev || !work_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    const Vol v = make_vol(D, H, W);
    cudaStream_t s = (cudaStream_t)stream;
    double* part = (double*)work_dev;
    CK(reg_partials(u_dev, gu_dev, part, B, v, s));
    CK(reduce_partials(part, voxel_blocks(v), 1, 1.0, loss_dev, 1, B, s));
    return DARC_OK;
}

size_t darc_subject_grad_workspace(const darc_config* cfg, int B, int D, int H, int W)
{
    if (!cfg) return 0;
    const size_t V = (size_t)D * H * W, F = 3 * V * B, F4 = 4 * V * B;
    const int T = std::max(cfg->n_squarings, 1);
    const size_t fields = (size_t)CkPlan(T, cfg->checkpoint_stride).fields();
    return align256(sizeof(float) * F4 * fields) + align256(sizeof(float) * F) + align256(sizeof(float) * 2 * F4) +
           align256(sizeof(float) * V * B) + align256(sizeof(float) * 3 * V * B) + align256(sizeof(float) * 2 * V) +
           2 * darc_loss_workspace(B, D, H, W) + align256(sizeof(float) * 3 * V * B) +
           align256(sizeof(int) * exp_far_flags(B, make_vol(D, H, W)));
}

int darc_subject_grad(const darc_config* cfg, const float* I_dev, const float* A_dev, const float* v_dev,
                      float* energy_dev, float* gv_dev, void* work_dev, int B, int D, int H, int W, void* stream)
{
    if (!I_dev || !A_dev || !v_dev || !energy_dev || !gv_dev || !work_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    rc = check_config(cfg, D, H, W);
    if (rc) return rc;
    const Vol v = make_vol(D, H, W);
    cudaStream_t s = (cudaStream_t)stream;
    const int T = cfg->n_squarings;
    const size_t F = 3 * (size_t)v.V * B, F4 = 4 * (size_t)v.V * B;
    Carve cv(work_dev);
    const CkPlan plan(T, cfg->checkpoint_stride);
    // packed squaring fields and the gather adjoint chain, as in the cohort's
    // step; the last adjoint step writes the planar gv
    float* u_all = cv.take<float>(F4 * plan.fields());
    float* gT = cv.take<float>(F);
    float4* gbuf = reinterpret_cast<float4*>(cv.take<float>(2 * F4));
    float* Wimg = cv.take<float>((size_t)v.V * B);
    float* coef = cv.take<float>(3 * (size_t)v.V * B);
    float* stats = cv.take<float>(2 * (size_t)v.V);
    double* pL = cv.take<double>(2 * (size_t)B * nblk_max(v));
    double* pR = cv.take<double>(2 * (size_t)B * nblk_max(v));
    float* P = cv.take<float>(3 * (size_t)B * v.V);
    int* flags = cv.take<int>(exp_far_flags(B, v));
    CK(cudaMemsetAsync(flags, 0, sizeof(int) * exp_far_flags(B, v), s));
    const float s0 = std::ldexp(1.0f, -T);
    auto sq = [&](const float* src, float scale, float* dst) {
        return exp_square_packed(src, src != v_dev, scale, reinterpret_cast<float4*>(dst), B, v, s);
    };
    CK(exp_forward_plan(plan, v_dev, u_all, F4, s0, sq));
    const float* uT = u_all + (size_t)plan.slot(T - 1) * F4;
    if (pointwise(cfg->dissim)) {
        CK(mse_warp_reg(I_dev, v.V, A_dev, uT, cfg->lambda, gT, pL, B, v, cfg->dissim == DARC_L1, s, 1));
        CK(reduce_partials(pL, voxel_blocks(v), 2, 1.0, energy_dev, 2, B, s));
    } else {
        const int r = cfg->ncc_window / 2;
        CK(atlas_stats(A_dev, stats, r, v, P, s));
        CK(warp_packed(I_dev, v.V, reinterpret_cast<const float4*>(uT), Wimg, B, v, s));
        CK(lncc_forward(Wimg, nullptr, A_dev, stats, r, cfg->ncc_eps, 0, patch_metric(cfg->dissim), coef, pL, B,
                        v, P, s));
        CK(lncc_backward_warp_reg(Wimg, A_dev, coef, r, I_dev, v.V, uT, cfg->lambda, gT, pR, B, v, P, s, 1));
        CK(reduce_partials(pL, box_blocks(v, B), 1, 1.0, energy_dev, 2, B, s));
        CK(reduce_partials(pR, box_blocks(v, B), 1, 1.0, energy_dev + 1, 2, B, s));
    }
    // gradients alternate between the two gbuf halves; the last step writes gv
    // (the scatter adjoint: into a cleared interleaved buffer, then unpacked)
    const bool gather = cfg->adjoint == DARC_ADJOINT_GATHER;
    float* g4[2] = {reinterpret_cast<float*>(gbuf), reinterpret_cast<float*>(gbuf + (size_t)B * v.V)};
    const float* gin = gT;
    int in4 = 0;
    const float* last = nullptr;
    auto adj = [&](int t, const float* src, float scale) {
        cudaError_t e;
        if (!gather) {
            float4* gout = reinterpret_cast<float4*>(g4[(T - 1 - t) % 2]);
            e = cudaMemsetAsync(gout, 0, (size_t)B * v.V * sizeof(float4), s);
            if (e == cudaSuccess) e = exp_square_adjoint4(src, t != 0, scale, gin, in4, gout, scale, B, v, s);
            gin = last = reinterpret_cast<const float*>(gout);
            in4 = 1;
            return e;
        }
        const int out4 = adj_out4(t, T);
        float* gout = t == 0 ? gv_dev : g4[(T - 1 - t) % 2];
        e = exp_adjoint_step(src, t != 0, scale, gin, in4, gout, out4, scale, flags, B, v, s);
        gin = gout;
        in4 = out4;
        return e;
    };
    CK(exp_backward_plan(plan, v_dev, u_all, F4, s0, sq, adj));
    if (!gather) CK(unpack_field(reinterpret_cast<const float4*>(last), gv_dev, B, v, s));
    return DARC_OK;
}

int darc_adam(float* theta_dev, float* m_dev, float* s_dev, const float* g_dev, size_t N, int k, float lr,
              float beta1, float beta2, float eps, void* stream)
{
    if (!theta_dev || !m_dev || !s_dev || !g_dev) return fail(DARC_ERR_ARG, "null argument");
    if (k < 1) return fail(DARC_ERR_ARG, "step k must be >= 1");
    if (N == 0) return DARC_OK;
    const double c1 = 1.0 - std::pow((double)beta1, k), c2 = 1.0 - std::pow((double)beta2, k);
    CK(adam_flat(theta_dev, m_dev, s_dev, g_dev, N, (float)(lr / c1), (float)(1.0 / std::sqrt(c2)), beta1, beta2,
                 eps, (cudaStream_t)stream));
    return DARC_OK;
}

size_t darc_centrality_workspace(int n, int D, int H, int W)
{
    (void)n;
    return align256(sizeof(double) * 2 * (size_t)centrality_blocks(make_vol(D, H, W)));
}

int darc_centrality(float* v_dev, double* metrics_dev, void* work_dev, int n, int D, int H, int W, void* stream)
{
    if (!v_dev || !work_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(1, D, H, W);
    if (rc) return rc;
    if (n < 1) return fail(DARC_ERR_ARG, "n must be >= 1");
    CK(centrality(v_dev, n, make_vol(D, H, W), (double*)work_dev, metrics_dev, (cudaStream_t)stream));
    return DARC_OK;
}

size_t darc_atlas_mean_workspace(int n, int D, int H, int W)
{
    const size_t V = (size_t)D * H * W;
    const int chunk = std::min(n, 8);
    return align256(sizeof(double) * V) + align256(sizeof(float) * 2 * 3 * V * chunk) + align256(sizeof(int) * n);
}

int darc_atlas_mean(const float* I_dev, const float* v_dev, float* A_dev, void* work_dev, int n, int D, int H, int W,
                    int T, void* stream)
{
    if (!I_dev || !v_dev || !A_dev || !work_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(std::min(n, 8), D, H, W);
    if (rc) return rc;
    if (T < 1 || T > 20) return fail(DARC_ERR_ARG, "T must be 1..20");
    const Vol v = make_vol(D, H, W);
    cudaStream_t s = (cudaStream_t)stream;
    const int chunk = std::min(n, 8);
    Carve cv(work_dev);
    double* acc = cv.take<double>(v.V);
    float* u2 = cv.take<float>(2 * 3 * (size_t)v.V * chunk);
    int* iota = cv.take<int>(n);
    std::vector<int> h(n);
    for (int i = 0; i < n; ++i) h[i] = i;
    CK(cudaMemcpyAsync(iota, h.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(acc, 0, sizeof(double) * v.V, s));
    for (int f = 0; f < n; f += chunk) {
        const int cnt = std::min(chunk, n - f);
        float* uT = nullptr;
        CK(exp_forward_pingpong(v_dev + (size_t)f * 3 * v.V, u2, cnt, v, T, 1.f, s, &uT));
        CK(warp_accumulate(I_dev, iota + f, uT, acc, cnt, v, s));
    }
    CK(finalize_mean(acc, 1.0 / n, A_dev, v, s));
    return DARC_OK;
}

int darc_label_gather(const uint8_t* labels_dev, const float* u_dev, uint8_t* out_dev, int B, int D, int H, int W,
                      void* stream)
{
    if (!labels_dev || !u_dev || !out_dev) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    CK(label_gather(labels_dev, u_dev, out_dev, B, make_vol(D, H, W), (cudaStream_t)stream));
    return DARC_OK;
}

size_t darc_dice_workspace(int B, int n_labels)
{
    if (B < 1 || n_labels < 2 || n_labels > 256) return 0;
    return sizeof(unsigned long long) * 3 * (size_t)B * n_labels;
}

int darc_dice(const uint8_t* a_dev, const uint8_t* b_dev, int B, long long V, int n_labels, void* work_dev,
              double* dice_host, void* stream)
{
    if (!a_dev || !b_dev || !work_dev || !dice_host) return fail(DARC_ERR_ARG, "null argument");
    if (B < 1 || V < 1) return fail(DARC_ERR_ARG, "B and V must be >= 1");
    if (n_labels < 2 || n_labels > 256) return fail(DARC_ERR_ARG, "n_labels must be 2..256");
    if (B > 65535) return fail(DARC_ERR_ARG, "at most 65535 label maps a call");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* cnt = static_cast<unsigned long long*>(work_dev);
    const size_t nc = 3 * (size_t)B * n_labels;
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * nc, s));
    CK(label_overlap(a_dev, b_dev, B, V, n_labels, cnt, s));
    std::vector<unsigned long long> h(nc);
    CK(cudaMemcpyAsync(h.data(), cnt, sizeof(unsigned long long) * nc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int b = 0; b < B; ++b)
        for (int l = 1; l < n_labels; ++l) {
            const unsigned long long* q = h.data() + ((size_t)b * n_labels + l) * 3;
            dice_host[(size_t)b * (n_labels - 1) + l - 1] =
                (q[0] + q[1]) ? 2.0 * (double)q[2] / (double)(q[0] + q[1]) : -1.0;
        }
    return DARC_OK;
}

int darc_warp_points(const float* u_dev, int D, int H, int W, const float* pts_dev, long long P, float* out_dev,
                     void* stream)
{
    if (!u_dev || !pts_dev || !out_dev) return fail(DARC_ERR_ARG, "null argument");
    if (P < 0) return fail(DARC_ERR_ARG, "negative point count");
    int rc = check_dims(1, D, H, W);
    if (rc) return rc;
    if (P == 0) return DARC_OK;
    CK(warp_points(u_dev, make_vol(D, H, W), pts_dev, P, out_dev, (cudaStream_t)stream));
    return DARC_OK;
}

int darc_compose(const float* a_dev, const float* b_dev, float* out_dev, int B, int D, int H, int W, void* stream)
{
    if (!a_dev || !b_dev || !out_dev) return fail(DARC_ERR_ARG, "null argument");
    if (out_dev == a_dev || out_dev == b_dev) return fail(DARC_ERR_ARG, "out must not alias a or b");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    CK(compose(a_dev, b_dev, out_dev, B, make_vol(D, H, W), (cudaStream_t)stream));
    return DARC_OK;
}

int darc_jacobian_det(const float* u_dev, float* det_dev, unsigned long long* count_dev, int B, int D, int H, int W,
                      void* stream)
{
    if (!u_dev || (!det_dev && !count_dev)) return fail(DARC_ERR_ARG, "null argument");
    int rc = check_dims(B, D, H, W);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (count_dev) CK(cudaMemsetAsync(count_dev, 0, sizeof(unsigned long long) * B, s));
    CK(jacobian_det(u_dev, det_dev, count_dev, B, make_vol(D, H, W), s));
    return DARC_OK;
}

}  // extern "C"
