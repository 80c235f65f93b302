/*
 * darc_oracle.c -- plain FP64 CPU oracle of DARC's per-subject update, the
 * centrality activation, the atlas re-estimate and one-shot label propagation
 * (Zou et al., "An Efficient Model-Driven Groupwise Approach for Atlas
 * Construction", arXiv 2508.10743).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA library and neither links
 * the other.
 *
 * Style: every quantity is computed the plain way its definition reads, in
 * double precision, with loops a reader can check against the paper.  OpenMP
 * only splits loops whose iterations are independent (gathers, per-subject
 * work); every scatter runs sequentially inside one subject.
 *
 * Conventions (the paper writes volumes as M x N x H, Sec. "Methodology"):
 *   a volume has n[0] x n[1] x n[2] = D x H x W voxels (z, y, x), x fastest;
 *   a field is planar [3][V]; channel a is the displacement along axis a
 *   (0 = z, 1 = y, 2 = x) in voxel units; an image is [V].
 *
 * Readings of passages the paper leaves silent or ambiguous are stated at the
 * function that takes them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* configuration (mirrors the knobs Algorithm 1 and Sec. "Experiments" name) */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dissim;        /* 0 = MSE, 1 = local (windowed) NCC, 2 = L1, 3 = SSIM  */
    int window;        /* NCC window edge w (odd)                              */
    int T;             /* scaling-and-squaring steps                           */
    int inner_steps;   /* K2: Adam steps per subject per sweep                 */
    int atlas_epochs;  /* K3: epochs of atlas SGD (NCC)                        */
    int atlas_batch;   /* mini-batch size of the atlas SGD                      */
    int reset_each_sweep; /* 1: Algorithm 1 literally (v and Adam restart)     */
    int pad_;
    double lambda;     /* weight of the diffusion regulariser                  */
    double lr, beta1, beta2, adam_eps;  /* Adam                                */
    double ncc_eps;    /* stabiliser in the NCC denominator                    */
    uint64_t seed;     /* mini-batch shuffling                                  */
} ora_cfg;

int ora_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

static inline long lin3(const int n[3], long z, long y, long x)
{
    return (z * n[1] + y) * n[2] + x;
}

/* ------------------------------------------------------------------------ */
/* Trilinear sampling S(f, p) (the warp "I o phi" of Eq. 2).                  */
/*                                                                          */
/* Reading (the paper does not define the interpolation or the padding):    */
/* trilinear, with "border" padding -- each coordinate is clamped to        */
/* [0, n_a - 1]; the cell is i_a = min(floor(p_a), n_a - 2), t_a = p_a - i_a. */
/* dS/dp_a is the derivative of the trilinear weights, and 0 on an axis     */
/* whose coordinate was clamped (strictly outside the volume).              */
/* ------------------------------------------------------------------------ */
typedef struct {
    long idx[8];       /* linear indices of the 8 corners                     */
    double w[8];       /* trilinear weights                                   */
    double dw[8][3];   /* d w / d p_a (already 0 on clamped axes)             */
} corners_t;

static void tri_corners(const int n[3], const double p[3], corners_t *c)
{
    long i[3];
    double t[3];
    int clamped[3];
    for (int a = 0; a < 3; ++a) {
        double q = p[a];
        clamped[a] = 0;
        if (q < 0.0) { q = 0.0; clamped[a] = 1; }
        else if (q > (double)(n[a] - 1)) { q = (double)(n[a] - 1); clamped[a] = 1; }
        long f = (long)floor(q);
        if (f > n[a] - 2) f = n[a] - 2;
        i[a] = f;
        t[a] = q - (double)f;
    }
    int k = 0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx, ++k) {
                double wz = cz ? t[0] : 1.0 - t[0], dz = cz ? 1.0 : -1.0;
                double wy = cy ? t[1] : 1.0 - t[1], dy = cy ? 1.0 : -1.0;
                double wx = cx ? t[2] : 1.0 - t[2], dx = cx ? 1.0 : -1.0;
                c->idx[k] = lin3(n, i[0] + cz, i[1] + cy, i[2] + cx);
                c->w[k] = wz * wy * wx;
                c->dw[k][0] = clamped[0] ? 0.0 : dz * wy * wx;
                c->dw[k][1] = clamped[1] ? 0.0 : wz * dy * wx;
                c->dw[k][2] = clamped[2] ? 0.0 : wz * wy * dx;
            }
}

/* S(f, p) and, when grad != NULL, dS/dp. */
static double tri_sample(const double *f, const corners_t *c, double grad[3])
{
    double val = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int k = 0; k < 8; ++k) {
        double fv = f[c->idx[k]];
        val += c->w[k] * fv;
        g0 += c->dw[k][0] * fv;
        g1 += c->dw[k][1] * fv;
        g2 += c->dw[k][2] * fv;
    }
    if (grad) { grad[0] = g0; grad[1] = g1; grad[2] = g2; }
    return val;
}

/* the sample point x + u(x) of voxel (z, y, x) */
static inline void sample_point(const double *u, long V, long l, long z, long y, long x, double p[3])
{
    p[0] = (double)z + u[l];
    p[1] = (double)y + u[V + l];
    p[2] = (double)x + u[2 * V + l];
}

/* public single-point sampler (used by the pin tests) */
double ora_sample(const double *f, int D, int H, int W, double pz, double py, double px, double *grad)
{
    const int n[3] = {D, H, W};
    const double p[3] = {pz, py, px};
    corners_t c;
    tri_corners(n, p, &c);
    return tri_sample(f, &c, grad);
}

/* ------------------------------------------------------------------------ */
/* Exp by scaling and squaring (Sec. "Diffeomorphisms": phi = Exp(v), seven  */
/* squarings; Algorithm 1 "phi = Exp(v)").                                  */
/*   u_0 = sign * 2^-T v,   u_{t+1}(x) = u_t(x) + S(u_t, x + u_t(x)),        */
/*   phi(x) = x + u_T(x).  sign = -1 gives Exp(-v) (Eq. oneshot).            */
/* u_all holds u_0 .. u_T, (T + 1) fields of [3][V].                         */
/* ------------------------------------------------------------------------ */
int ora_exp(const double *v, int D, int H, int W, int T, double sign, double *u_all)
{
    const int n[3] = {D, H, W};
    const long V = (long)D * H * W;
    const double scale = sign * ldexp(1.0, -T);
    for (long e = 0; e < 3 * V; ++e) u_all[e] = scale * v[e];
    for (int t = 0; t < T; ++t) {
        const double *ut = u_all + (long)t * 3 * V;
        double *un = u_all + (long)(t + 1) * 3 * V;
#pragma omp parallel for schedule(static)
        for (long z = 0; z < D; ++z)
            for (long y = 0; y < H; ++y)
                for (long x = 0; x < W; ++x) {
                    const long l = lin3(n, z, y, x);
                    double p[3];
                    corners_t c;
                    sample_point(ut, V, l, z, y, x, p);
                    tri_corners(n, p, &c);
                    for (int ch = 0; ch < 3; ++ch)
                        un[ch * V + l] = ut[ch * V + l] + tri_sample(ut + ch * V, &c, NULL);
                }
    }
    return 0;
}

/* Tangent (forward-mode derivative) of Exp: du_T for a perturbation dv.
 * d u_{t+1,c}(x) = du_{t,c}(x) + S(du_{t,c}, p) + sum_a dS(u_{t,c}, p)/dp_a du_{t,a}(x).
 * Independent of the adjoint below; the two are tied by <J dv, g> = <dv, J^T g>. */
int ora_exp_jvp(const double *u_all, const double *dv, int D, int H, int W, int T, double sign,
                double *du_out)
{
    const int n[3] = {D, H, W};
    const long V = (long)D * H * W;
    const double scale = sign * ldexp(1.0, -T);
    double *du = (double *)malloc(sizeof(double) * 3 * V);
    double *dn = (double *)malloc(sizeof(double) * 3 * V);
    if (!du || !dn) { free(du); free(dn); return -1; }
    for (long e = 0; e < 3 * V; ++e) du[e] = scale * dv[e];
    for (int t = 0; t < T; ++t) {
        const double *ut = u_all + (long)t * 3 * V;
#pragma omp parallel for schedule(static)
        for (long z = 0; z < D; ++z)
            for (long y = 0; y < H; ++y)
                for (long x = 0; x < W; ++x) {
                    const long l = lin3(n, z, y, x);
                    double p[3], g[3];
                    corners_t c;
                    sample_point(ut, V, l, z, y, x, p);
                    tri_corners(n, p, &c);
                    for (int ch = 0; ch < 3; ++ch) {
                        double val = du[ch * V + l] + tri_sample(du + ch * V, &c, NULL);
                        tri_sample(ut + ch * V, &c, g);
                        val += g[0] * du[l] + g[1] * du[V + l] + g[2] * du[2 * V + l];
                        dn[ch * V + l] = val;
                    }
                }
        double *tmp = du; du = dn; dn = tmp;
    }
    memcpy(du_out, du, sizeof(double) * 3 * V);
    free(du);
    free(dn);
    return 0;
}

/* Adjoint (reverse-mode derivative) of Exp: given gT = dE/du_T, returns
 * gv = dE/dv.  Each squaring u_{t+1} = u_t + S(u_t, x + u_t(x)) sends its
 * incoming gradient g_{t+1} three ways: to u_t(x) itself (identity), to the
 * sample point through dS/dp (Jacobian term), and to the 8 corners with the
 * trilinear weights (transpose of the interpolation -- a scatter).  The
 * scatter runs sequentially. */
int ora_exp_vjp(const double *u_all, const double *gT, int D, int H, int W, int T, double sign,
                double *gv)
{
    const int n[3] = {D, H, W};
    const long V = (long)D * H * W;
    double *g = (double *)malloc(sizeof(double) * 3 * V);
    double *gn = (double *)malloc(sizeof(double) * 3 * V);
    if (!g || !gn) { free(g); free(gn); return -1; }
    memcpy(g, gT, sizeof(double) * 3 * V);
    for (int t = T - 1; t >= 0; --t) {
        const double *ut = u_all + (long)t * 3 * V;
        memset(gn, 0, sizeof(double) * 3 * V);
        for (long z = 0; z < D; ++z)
            for (long y = 0; y < H; ++y)
                for (long x = 0; x < W; ++x) {
                    const long l = lin3(n, z, y, x);
                    double p[3], dS[3][3];
                    corners_t c;
                    sample_point(ut, V, l, z, y, x, p);
                    tri_corners(n, p, &c);
                    for (int ch = 0; ch < 3; ++ch) tri_sample(ut + ch * V, &c, dS[ch]);
                    for (int ch = 0; ch < 3; ++ch) {
                        const double gc = g[ch * V + l];
                        gn[ch * V + l] += gc;                       /* identity   */
                        for (int k = 0; k < 8; ++k)                 /* transpose  */
                            gn[ch * V + c.idx[k]] += c.w[k] * gc;
                    }
                    for (int a = 0; a < 3; ++a)                     /* Jacobian   */
                        gn[a * V + l] += g[l] * dS[0][a] + g[V + l] * dS[1][a] + g[2 * V + l] * dS[2][a];
                }
        double *tmp = g; g = gn; gn = tmp;
    }
    const double scale = sign * ldexp(1.0, -T);
    for (long e = 0; e < 3 * V; ++e) gv[e] = scale * g[e];
    free(g);
    free(gn);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Warp (I o phi)(x) = S(I, x + u(x)) (Eq. 2, "spatial transformation").     */
/* grad_p (nullable, [3][V]) receives dS(I, p)/dp at every voxel.            */
/* ------------------------------------------------------------------------ */
int ora_warp(const double *I, const double *u, int D, int H, int W, double *out, double *grad_p)
{
    const int n[3] = {D, H, W};
    const long V = (long)D * H * W;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < D; ++z)
        for (long y = 0; y < H; ++y)
            for (long x = 0; x < W; ++x) {
                const long l = lin3(n, z, y, x);
                double p[3], g[3];
                corners_t c;
                sample_point(u, V, l, z, y, x, p);
                tri_corners(n, p, &c);
                out[l] = tri_sample(I, &c, g);
                if (grad_p) { grad_p[l] = g[0]; grad_p[V + l] = g[1]; grad_p[2 * V + l] = g[2]; }
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Diffusion regulariser ||grad phi||^2 (Eq. 2, second term).                */
/* Reading: it acts on the displacement u of phi = id + u (grad phi = I +   */
/* grad u, so the two differ by a constant and a boundary term), with       */
/* forward differences, a mean over the voxel pairs that exist along each   */
/* axis, and a mean over the three axes:                                     */
/*   R(u) = 1/3 sum_a [ 1/P_a sum_{x, x+e_a in volume} sum_c               */
/*                      (u_c(x+e_a) - u_c(x))^2 ],  P_a = V (n_a - 1)/n_a.  */
/* Eq. 2 writes the term outside the sum over i with a free index; it is    */
/* read as inside the sum (every subject is regularised).                   */
/* ------------------------------------------------------------------------ */
double ora_reg(const double *u, int D, int H, int W, double *grad)
{
    const int n[3] = {D, H, W};
    const long V = (long)D * H * W;
    double total = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * 3 * V);
    for (int a = 0; a < 3; ++a) {
        const double P = (double)V * (double)(n[a] - 1) / (double)n[a];
        const long step = (a == 0) ? (long)H * W : (a == 1) ? (long)W : 1;
        double sum = 0.0;
        for (long z = 0; z < D; ++z)
            for (long y = 0; y < H; ++y)
                for (long x = 0; x < W; ++x) {
                    const long q[3] = {z, y, x};
                    if (q[a] + 1 >= n[a]) continue;
                    const long l = lin3(n, z, y, x);
                    for (int c = 0; c < 3; ++c) {
                        const double d = u[c * V + l + step] - u[c * V + l];
                        sum += d * d;
                        if (grad) {
                            const double gd = (2.0 / 3.0) * d / P;
                            grad[c * V + l + step] += gd;
                            grad[c * V + l] -= gd;
                        }
                    }
                }
        total += sum / P;
    }
    return total / 3.0;
}

/* ------------------------------------------------------------------------ */
/* MSE dissimilarity (Sec. "Dissimilarity metrics").  Reading of the silent  */
/* normalisation: the mean over voxels, L = 1/V sum_x (W(x) - A(x))^2.       */
/* ------------------------------------------------------------------------ */
double ora_mse(const double *Wimg, const double *A, long V, double *gW, double *gA)
{
    double s = 0.0;
    for (long l = 0; l < V; ++l) {
        const double d = Wimg[l] - A[l];
        s += d * d;
        if (gW) gW[l] = 2.0 * d / (double)V;
        if (gA) gA[l] = -2.0 * d / (double)V;
    }
    return s / (double)V;
}

/* ------------------------------------------------------------------------ */
/* Box sum over the w^3 window centred at each voxel, zero outside the       */
/* volume -- the patch statistics of the "patch-wise" NCC.  Brute force.     */
/* ------------------------------------------------------------------------ */
int ora_box(const double *f, int D, int H, int W, int w, double *out)
{
    const int n[3] = {D, H, W};
    const int r = w / 2;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < D; ++z)
        for (long y = 0; y < H; ++y)
            for (long x = 0; x < W; ++x) {
                double s = 0.0;
                for (long qz = z - r; qz <= z + r; ++qz) {
                    if (qz < 0 || qz >= D) continue;
                    for (long qy = y - r; qy <= y + r; ++qy) {
                        if (qy < 0 || qy >= H) continue;
                        for (long qx = x - r; qx <= x + r; ++qx) {
                            if (qx < 0 || qx >= W) continue;
                            s += f[lin3(n, qz, qy, qx)];
                        }
                    }
                }
                out[lin3(n, z, y, x)] = s;
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Local (windowed) NCC (Sec. "Dissimilarity metrics": NCC is patch-wise).   */
/* Reading of the silent form: squared local correlation over the w^3        */
/* window, zero padding outside the volume, normalised by the full window    */
/* count N = w^3, stabilised by eps:                                         */
/*   P  = S_JA - S_J S_A / N,  sJ = S_JJ - S_J^2 / N,  sA = S_AA - S_A^2 / N, */
/*   cc = P^2 / (sJ sA + eps),  L = -1/V sum_x cc(x).                        */
/* Gradients by the chain rule through the window sums; each window sum     */
/* reaches voxel y from every x whose window holds y, and that relation is  */
/* symmetric, so the sums over x are box sums around y:                      */
/*   dL/dJ(y) = -1/V [ sum_{x ~ y} a(x) + 2 J(y) sum b(x) + A(y) sum g(x) ]  */
/* with a = dcc/dS_J, b = dcc/dS_JJ, g = dcc/dS_JA (and the mirror for A).   */
/* cc_out (nullable) receives cc per voxel.                                  */
/* ------------------------------------------------------------------------ */
double ora_lncc(const double *J, const double *A, int D, int H, int W, int w, double eps,
                double *gJ, double *gA, double *cc_out)
{
    const int n[3] = {D, H, W};
    const long V = (long)D * H * W;
    const int r = w / 2;
    const double N = (double)w * w * w;
    double *aJ = (double *)malloc(sizeof(double) * V);
    double *bJ = (double *)malloc(sizeof(double) * V);
    double *aA = (double *)malloc(sizeof(double) * V);
    double *bA = (double *)malloc(sizeof(double) * V);
    double *gm = (double *)malloc(sizeof(double) * V);
    double *cc = (double *)malloc(sizeof(double) * V);
    if (!aJ || !bJ || !aA || !bA || !gm || !cc) {
        free(aJ); free(bJ); free(aA); free(bA); free(gm); free(cc);
        return NAN;
    }
#pragma omp parallel for schedule(static)
    for (long z = 0; z < D; ++z)
        for (long y = 0; y < H; ++y)
            for (long x = 0; x < W; ++x) {
                double sJ = 0, sA = 0, sJJ = 0, sAA = 0, sJA = 0;
                for (long qz = z - r; qz <= z + r; ++qz) {
                    if (qz < 0 || qz >= D) continue;
                    for (long qy = y - r; qy <= y + r; ++qy) {
                        if (qy < 0 || qy >= H) continue;
                        for (long qx = x - r; qx <= x + r; ++qx) {
                            if (qx < 0 || qx >= W) continue;
                            const long q = lin3(n, qz, qy, qx);
                            sJ += J[q];
                            sA += A[q];
                            sJJ += J[q] * J[q];
                            sAA += A[q] * A[q];
                            sJA += J[q] * A[q];
                        }
                    }
                }
                const long l = lin3(n, z, y, x);
                const double P = sJA - sJ * sA / N;
                const double varJ = sJJ - sJ * sJ / N;
                const double varA = sAA - sA * sA / N;
                const double Q = varJ * varA + eps;
                cc[l] = P * P / Q;
                /* dcc/dP = 2P/Q, dcc/dvarJ = -P^2 varA / Q^2, dcc/dvarA = -P^2 varJ / Q^2 */
                const double dP = 2.0 * P / Q;
                const double dvJ = -P * P * varA / (Q * Q);
                const double dvA = -P * P * varJ / (Q * Q);
                aJ[l] = dP * (-sA / N) + dvJ * (-2.0 * sJ / N);
                bJ[l] = dvJ;
                aA[l] = dP * (-sJ / N) + dvA * (-2.0 * sA / N);
                bA[l] = dvA;
                gm[l] = dP;
            }
    double L = 0.0;
    for (long l = 0; l < V; ++l) L += cc[l];
    L = -L / (double)V;
    if (gJ || gA) {
#pragma omp parallel for schedule(static)
        for (long z = 0; z < D; ++z)
            for (long y = 0; y < H; ++y)
                for (long x = 0; x < W; ++x) {
                    double saJ = 0, sbJ = 0, saA = 0, sbA = 0, sg = 0;
                    for (long qz = z - r; qz <= z + r; ++qz) {
                        if (qz < 0 || qz >= D) continue;
                        for (long qy = y - r; qy <= y + r; ++qy) {
                            if (qy < 0 || qy >= H) continue;
                            for (long qx = x - r; qx <= x + r; ++qx) {
                                if (qx < 0 || qx >= W) continue;
                                const long q = lin3(n, qz, qy, qx);
                                saJ += aJ[q]; sbJ += bJ[q];
                                saA += aA[q]; sbA += bA[q];
                                sg += gm[q];
                            }
                        }
                    }
                    const long l = lin3(n, z, y, x);
                    if (gJ) gJ[l] = -(saJ + 2.0 * J[l] * sbJ + A[l] * sg) / (double)V;
                    if (gA) gA[l] = -(saA + 2.0 * A[l] * sbA + J[l] * sg) / (double)V;
                }
    }
    if (cc_out) memcpy(cc_out, cc, sizeof(double) * V);
    free(aJ); free(bJ); free(aA); free(bA); free(gm); free(cc);
    return L;
}

/* ------------------------------------------------------------------------ */
/* L1 dissimilarity (Sec. "Dissimilarity metrics", point-wise):              */
/*   L = 1/V sum |W - A|;  dL/dW = sign(W - A) / V (0 where W = A, the       */
/*   subgradient torch's abs takes), dL/dA = -dL/dW.                         */
/* ------------------------------------------------------------------------ */
double ora_l1(const double *Wimg, const double *A, long V, double *gW, double *gA)
{
    double L = 0.0;
    for (long l = 0; l < V; ++l) {
        const double d = Wimg[l] - A[l];
        L += fabs(d);
        const double sg = (d > 0.0) ? 1.0 : ((d < 0.0) ? -1.0 : 0.0);
        if (gW) gW[l] = sg / (double)V;
        if (gA) gA[l] = -sg / (double)V;
    }
    return L / (double)V;
}

/* ------------------------------------------------------------------------ */
/* SSIM dissimilarity (Sec. "Dissimilarity metrics", patch-wise).  The      */
/* paper names the metric only; reading: the structural similarity of Wang */
/* et al. (2004) over the same w^3 windows as the local NCC (zero padding,   */
/* normalised by N = w^3), constants C1 = (0.01 * 1)^2, C2 = (0.03 * 1)^2   */
/* for intensities on [0, 1]:                                                */
/*   mu = S/N, var = S2/N - mu^2, cov = SJA/N - muJ muA,                     */
/*   ssim = (2 muJ muA + C1)(2 cov + C2) / ((muJ^2 + muA^2 + C1)(varJ + varA + C2)) */
/*   L = -(1/V) sum ssim.                                                    */
/* The gradient has the NCC form: with a = dssim/dS_J, b = dssim/dS_JJ,      */
/* g = dssim/dS_JA at each window centre,                                    */
/*   dL/dJ(y) = -1/V [ sum_{x ~ y} a(x) + 2 J(y) sum b(x) + A(y) sum g(x) ]. */
/* ------------------------------------------------------------------------ */
double ora_ssim(const double *J, const double *A, int D, int H, int W, int w, double *gJ, double *gA,
                double *ssim_out)
{
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    const int n[3] = {D, H, W};
    const long V = (long)D * H * W;
    const int r = w / 2;
    const double N = (double)w * w * w;
    double *aJ = (double *)malloc(sizeof(double) * V);
    double *bJ = (double *)malloc(sizeof(double) * V);
    double *aA = (double *)malloc(sizeof(double) * V);
    double *bA = (double *)malloc(sizeof(double) * V);
    double *gm = (double *)malloc(sizeof(double) * V);
    double *ss = (double *)malloc(sizeof(double) * V);
    if (!aJ || !bJ || !aA || !bA || !gm || !ss) {
        free(aJ); free(bJ); free(aA); free(bA); free(gm); free(ss);
        return NAN;
    }
#pragma omp parallel for schedule(static)
    for (long z = 0; z < D; ++z)
        for (long y = 0; y < H; ++y)
            for (long x = 0; x < W; ++x) {
                double sJ = 0, sA = 0, sJJ = 0, sAA = 0, sJA = 0;
                for (long qz = z - r; qz <= z + r; ++qz) {
                    if (qz < 0 || qz >= D) continue;
                    for (long qy = y - r; qy <= y + r; ++qy) {
                        if (qy < 0 || qy >= H) continue;
                        for (long qx = x - r; qx <= x + r; ++qx) {
                            if (qx < 0 || qx >= W) continue;
                            const long q = lin3(n, qz, qy, qx);
                            sJ += J[q];
                            sA += A[q];
                            sJJ += J[q] * J[q];
                            sAA += A[q] * A[q];
                            sJA += J[q] * A[q];
                        }
                    }
                }
                const long l = lin3(n, z, y, x);
                const double mJ = sJ / N, mA = sA / N;
                const double vJ = sJJ / N - mJ * mJ, vA = sAA / N - mA * mA;
                const double cJA = sJA / N - mJ * mA;
                const double a1 = 2.0 * mJ * mA + C1, a2 = 2.0 * cJA + C2;
                const double b1 = mJ * mJ + mA * mA + C1, b2 = vJ + vA + C2;
                const double S = a1 * a2 / (b1 * b2);
                ss[l] = S;
                /* d/dS_J: da1 = 2 mA/N, da2 = -2 mA/N, db1 = 2 mJ/N, db2 = -2 mJ/N */
                aJ[l] = (2.0 / N) * (mA * (a2 - a1) / (b1 * b2) - mJ * S * (1.0 / b1 - 1.0 / b2));
                aA[l] = (2.0 / N) * (mJ * (a2 - a1) / (b1 * b2) - mA * S * (1.0 / b1 - 1.0 / b2));
                bJ[l] = -S / (N * b2);           /* db2/dS_JJ = 1/N */
                bA[l] = -S / (N * b2);
                gm[l] = 2.0 * a1 / (N * b1 * b2); /* da2/dS_JA = 2/N */
            }
    double L = 0.0;
    for (long l = 0; l < V; ++l) L += ss[l];
    L = -L / (double)V;
    if (gJ || gA) {
#pragma omp parallel for schedule(static)
        for (long z = 0; z < D; ++z)
            for (long y = 0; y < H; ++y)
                for (long x = 0; x < W; ++x) {
                    double saJ = 0, sbJ = 0, saA = 0, sbA = 0, sg = 0;
                    for (long qz = z - r; qz <= z + r; ++qz) {
                        if (qz < 0 || qz >= D) continue;
                        for (long qy = y - r; qy <= y + r; ++qy) {
                            if (qy < 0 || qy >= H) continue;
                            for (long qx = x - r; qx <= x + r; ++qx) {
                                if (qx < 0 || qx >= W) continue;
                                const long q = lin3(n, qz, qy, qx);
                                saJ += aJ[q]; sbJ += bJ[q];
                                saA += aA[q]; sbA += bA[q];
                                sg += gm[q];
                            }
                        }
                    }
                    const long l = lin3(n, z, y, x);
                    if (gJ) gJ[l] = -(saJ + 2.0 * J[l] * sbJ + A[l] * sg) / (double)V;
                    if (gA) gA[l] = -(saA + 2.0 * A[l] * sbA + J[l] * sg) / (double)V;
                }
    }
    if (ssim_out) memcpy(ssim_out, ss, sizeof(double) * V);
    free(aJ); free(bJ); free(aA); free(bA); free(gm); free(ss);
    return L;
}

/* the patch-wise dissimilarity of the configuration (1: NCC, 3: SSIM) */
static double patch_loss(const ora_cfg *cfg, const double *J, const double *A, int D, int H, int W, double *gJ,
                         double *gA)
{
    if (cfg->dissim == 3) return ora_ssim(J, A, D, H, W, cfg->window, gJ, gA, NULL);
    return ora_lncc(J, A, D, H, W, cfg->window, cfg->ncc_eps, gJ, gA, NULL);
}

/* ------------------------------------------------------------------------ */
/* Adam (Sec. "Experiments": Adam, lr 1e-2, for velocities and atlas).       */
/* Reading of the silent constants: beta1 0.9, beta2 0.999, eps 1e-8, bias   */
/* corrected, eps added after the square root (Kingma & Ba).  k is 1-based.  */
/* ------------------------------------------------------------------------ */
void ora_adam(double *theta, double *m, double *s, const double *g, long N, int k,
              double lr, double b1, double b2, double eps)
{
    const double c1 = 1.0 - pow(b1, (double)k);
    const double c2 = 1.0 - pow(b2, (double)k);
    for (long e = 0; e < N; ++e) {
        m[e] = b1 * m[e] + (1.0 - b1) * g[e];
        s[e] = b2 * s[e] + (1.0 - b2) * g[e] * g[e];
        const double mh = m[e] / c1;
        const double sh = s[e] / c2;
        theta[e] -= lr * mh / (sqrt(sh) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Subject energy E = L(I o Exp(v), A) + lambda R(u_T) and dE/dv            */
/* (Eq. 2 for one subject; Algorithm 1, diffeo_pairwise_reg body).           */
/* parts (nullable) <- {L, R}.  gv (nullable) <- dE/dv.                      */
/* ------------------------------------------------------------------------ */
double ora_subject_energy(const double *I, const double *A, const double *v, int D, int H, int W,
                          const ora_cfg *cfg, double *gv, double *parts)
{
    const long V = (long)D * H * W;
    const int T = cfg->T;
    double *u_all = (double *)malloc(sizeof(double) * 3 * V * (T + 1));
    double *Wimg = (double *)malloc(sizeof(double) * V);
    double *gp = (double *)malloc(sizeof(double) * 3 * V);
    double *gW = (double *)malloc(sizeof(double) * V);
    double *gR = (double *)malloc(sizeof(double) * 3 * V);
    if (!u_all || !Wimg || !gp || !gW || !gR) {
        free(u_all); free(Wimg); free(gp); free(gW); free(gR);
        return NAN;
    }
    ora_exp(v, D, H, W, T, 1.0, u_all);
    const double *uT = u_all + (long)T * 3 * V;
    ora_warp(I, uT, D, H, W, Wimg, gp);
    double L;
    if (cfg->dissim == 0)
        L = ora_mse(Wimg, A, V, gW, NULL);
    else if (cfg->dissim == 2)
        L = ora_l1(Wimg, A, V, gW, NULL);
    else
        L = patch_loss(cfg, Wimg, A, D, H, W, gW, NULL);
    const double R = ora_reg(uT, D, H, W, gR);
    if (parts) { parts[0] = L; parts[1] = R; }
    if (gv) {
        /* dE/du_T = dL/dW * dS(I,p)/dp + lambda dR/du_T */
        double *gT = (double *)malloc(sizeof(double) * 3 * V);
        if (!gT) { free(u_all); free(Wimg); free(gp); free(gW); free(gR); return NAN; }
        for (int a = 0; a < 3; ++a)
            for (long l = 0; l < V; ++l)
                gT[a * V + l] = gW[l] * gp[a * V + l] + cfg->lambda * gR[a * V + l];
        ora_exp_vjp(u_all, gT, D, H, W, T, 1.0, gv);
        free(gT);
    }
    free(u_all); free(Wimg); free(gp); free(gW); free(gR);
    return L + cfg->lambda * R;
}

/* One Adam step of one subject (the inner loop of Algorithm 1):
 * returns E before the step; v, m, s updated; *k incremented first. */
double ora_subject_step(const double *I, const double *A, double *v, double *m, double *s, int *k,
                        int D, int H, int W, const ora_cfg *cfg, double *parts, double *g_out)
{
    const long V = (long)D * H * W;
    double *g = (double *)malloc(sizeof(double) * 3 * V);
    if (!g) return NAN;
    const double E = ora_subject_energy(I, A, v, D, H, W, cfg, g, parts);
    if (g_out) memcpy(g_out, g, sizeof(double) * 3 * V);
    *k += 1;
    ora_adam(v, m, s, g, 3 * V, *k, cfg->lr, cfg->beta1, cfg->beta2, cfg->adam_eps);
    free(g);
    return E;
}

/* ------------------------------------------------------------------------ */
/* Centrality activation (Eq. 3, fourth line; Algorithm 1 step 2):          */
/*   hat v_i = v_i - 1/n sum_j v_j.                                          */
/* Reading: applied to the velocities that parameterise phi_i = Exp(v_i)     */
/* (Sec. "Diffeomorphisms" optimises v instead of phi), in place.            */
/* ------------------------------------------------------------------------ */
void ora_centrality(double *v_all, int n, long V3)
{
#pragma omp parallel for schedule(static)
    for (long e = 0; e < V3; ++e) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += v_all[(long)i * V3 + e];
        const double mean = s / (double)n;
        for (int i = 0; i < n; ++i) v_all[(long)i * V3 + e] -= mean;
    }
}

/* Centrality error (Table 1): mean over voxels of the Euclidean norm of the
 * cohort-mean field (1/n) sum_i f_i(x).  Reading: the paper does not define
 * the norm; this one is 0 exactly when the constraint of Eq. 1 holds. */
double ora_centrality_metric(const double *f_all, int n, long V)
{
    double tot = 0.0;
    for (long l = 0; l < V; ++l) {
        double ss = 0.0;
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += f_all[(long)i * 3 * V + a * V + l];
            s /= (double)n;
            ss += s * s;
        }
        tot += sqrt(ss);
    }
    return tot / (double)V;
}

/* ------------------------------------------------------------------------ */
/* Atlas, MSE closed form (Sec. "Dissimilarity metrics", MSE equation):     */
/*   A = 1/n sum_i I_i o Exp(hat v_i).                                       */
/* ------------------------------------------------------------------------ */
int ora_atlas_mean(const double *I_all, const double *v_all, int n, int D, int H, int W, int T,
                   double *A)
{
    const long V = (long)D * H * W;
    double *u_all = (double *)malloc(sizeof(double) * 3 * V * (T + 1));
    double *Wimg = (double *)malloc(sizeof(double) * V);
    if (!u_all || !Wimg) { free(u_all); free(Wimg); return -1; }
    memset(A, 0, sizeof(double) * V);
    for (int i = 0; i < n; ++i) {
        ora_exp(v_all + (long)i * 3 * V, D, H, W, T, 1.0, u_all);
        ora_warp(I_all + (long)i * V, u_all + (long)T * 3 * V, D, H, W, Wimg, NULL);
        for (long l = 0; l < V; ++l) A[l] += Wimg[l];
    }
    for (long l = 0; l < V; ++l) A[l] /= (double)n;
    free(u_all);
    free(Wimg);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Atlas closed form for L1 (Sec. "Dissimilarity metrics"): the voxel-wise  */
/* median of the warped cohort, A(x) = median_i I_i o Exp(hat v_i)(x).       */
/* Reading for an even n: the lower of the two middle values (sorted s_0 <=  */
/* ... <= s_{n-1}, A = s_{(n-1)/2}), which minimises the L1 sum like any     */
/* value between the middle two and is the value torch.median returns.      */
/* ------------------------------------------------------------------------ */
static int cmp_double(const void *a, const void *b)
{
    const double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int ora_median(const double *X, int n, long V, double *out)
{
    double *col = (double *)malloc(sizeof(double) * n);
    if (!col) return -1;
    for (long l = 0; l < V; ++l) {
        for (int i = 0; i < n; ++i) col[i] = X[(long)i * V + l];
        qsort(col, n, sizeof(double), cmp_double);
        out[l] = col[(n - 1) / 2];
    }
    free(col);
    return 0;
}

int ora_atlas_median(const double *I_all, const double *v_all, int n, int D, int H, int W, int T, double *A)
{
    const long V = (long)D * H * W;
    double *u_all = (double *)malloc(sizeof(double) * 3 * V * (T + 1));
    double *Wall = (double *)malloc(sizeof(double) * V * n);
    if (!u_all || !Wall) { free(u_all); free(Wall); return -1; }
    for (int i = 0; i < n; ++i) {
        ora_exp(v_all + (long)i * 3 * V, D, H, W, T, 1.0, u_all);
        ora_warp(I_all + (long)i * V, u_all + (long)T * 3 * V, D, H, W, Wall + (long)i * V, NULL);
    }
    const int rc = ora_median(Wall, n, V, A);
    free(u_all);
    free(Wall);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Mini-batch order for the atlas SGD (Algorithm 1, SGD_for_atlas's         */
/* "dataloader").  The paper does not say how batches are drawn; reading: a */
/* fresh uniform shuffle per epoch, from the counter-based SplitMix64        */
/* generator (Steele, Lea & Flood, OOPSLA 2014): the k-th draw (k = 1, 2..)  */
/* is mix(s0 + k * 0x9E3779B97F4A7C15) with mix the published finaliser and  */
/* s0 = seed * 1000003 + sweep * 1009 + epoch (mod 2^64); Fisher-Yates from  */
/* the last position down, j = draw mod (i + 1).                             */
/* ------------------------------------------------------------------------ */
static uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void ora_shuffle(uint64_t seed, int sweep, int epoch, int n, int *perm)
{
    const uint64_t s0 = seed * 1000003ULL + (uint64_t)sweep * 1009ULL + (uint64_t)epoch;
    for (int i = 0; i < n; ++i) perm[i] = i;
    uint64_t k = 0;
    for (int i = n - 1; i >= 1; --i) {
        ++k;
        const uint64_t r = sm64_mix(s0 + k * 0x9E3779B97F4A7C15ULL);
        const int j = (int)(r % (uint64_t)(i + 1));
        const int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
    }
}

uint64_t ora_splitmix64(uint64_t s0, uint64_t k)
{
    return sm64_mix(s0 + k * 0x9E3779B97F4A7C15ULL);
}

/* ------------------------------------------------------------------------ */
/* Atlas by mini-batch SGD (Sec. "Dissimilarity metrics", NCC/SSIM have no  */
/* closed form; Algorithm 1 SGD_for_atlas): K3 epochs, each a pass over the */
/* shuffled cohort in mini-batches; per batch the loss is the mean patch-  */
/* wise (NCC or SSIM) dissimilarity of its warped images W_i = I_i o       */
/* Exp(hat v_i) to A, and                                                   */
/* Adam (fresh state per call, as SGD_for_atlas creates its optimiser)       */
/* updates A.  Reading: A starts from the current atlas (warm start) rather */
/* than a fresh initialize().  loss_out (nullable) <- mean loss of the last */
/* epoch.                                                                    */
/* ------------------------------------------------------------------------ */
int ora_atlas_sgd(const double *I_all, const double *v_all, int n, int D, int H, int W,
                  const ora_cfg *cfg, int sweep, double *A, double *loss_out)
{
    const long V = (long)D * H * W;
    const int T = cfg->T;
    double *u_all = (double *)malloc(sizeof(double) * 3 * V * (T + 1));
    double *Wall = (double *)malloc(sizeof(double) * V * n);
    double *gA = (double *)malloc(sizeof(double) * V);
    double *gi = (double *)malloc(sizeof(double) * V);
    double *m = (double *)calloc(V, sizeof(double));
    double *s = (double *)calloc(V, sizeof(double));
    int *perm = (int *)malloc(sizeof(int) * n);
    if (!u_all || !Wall || !gA || !gi || !m || !s || !perm) {
        free(u_all); free(Wall); free(gA); free(gi); free(m); free(s); free(perm);
        return -1;
    }
    for (int i = 0; i < n; ++i) {
        ora_exp(v_all + (long)i * 3 * V, D, H, W, T, 1.0, u_all);
        ora_warp(I_all + (long)i * V, u_all + (long)T * 3 * V, D, H, W, Wall + (long)i * V, NULL);
    }
    int k = 0;
    double last = 0.0;
    const int B = cfg->atlas_batch > 0 ? cfg->atlas_batch : n;
    for (int ep = 0; ep < cfg->atlas_epochs; ++ep) {
        ora_shuffle(cfg->seed, sweep, ep, n, perm);
        double ep_loss = 0.0;
        for (int b0 = 0; b0 < n; b0 += B) {
            const int nb = (b0 + B <= n) ? B : n - b0;
            memset(gA, 0, sizeof(double) * V);
            for (int q = 0; q < nb; ++q) {
                const int i = perm[b0 + q];
                ep_loss += patch_loss(cfg, Wall + (long)i * V, A, D, H, W, NULL, gi);
                for (long l = 0; l < V; ++l) gA[l] += gi[l] / (double)nb;
            }
            ++k;
            ora_adam(A, m, s, gA, V, k, cfg->lr, cfg->beta1, cfg->beta2, cfg->adam_eps);
        }
        last = ep_loss / (double)n;
    }
    if (loss_out) *loss_out = last;
    free(u_all); free(Wall); free(gA); free(gi); free(m); free(s); free(perm);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One sweep = one outer iteration of Algorithm 1 main (Eq. 3):             */
/*   every subject takes K2 Adam steps against the frozen atlas A^k (the    */
/*   subjects are uncoupled given A^k, so their order does not matter);     */
/*   then the centrality activation; then the atlas re-estimate.            */
/* Reading: v_i and its Adam state persist across sweeps (coordinate descent */
/* from the current iterate, Eq. 3) unless reset_each_sweep asks for the    */
/* literal restart of diffeo_pairwise_reg.                                  */
/* stats (nullable) <- {mean L, mean R, centrality before, after} where L,R */
/* are the subjects' values at their last inner step.                        */
/* ------------------------------------------------------------------------ */
int ora_sweep(const double *I_all, double *v_all, double *m_all, double *s_all, int *k_all,
              double *A, int n, int D, int H, int W, const ora_cfg *cfg, int sweep, double *stats)
{
    const long V = (long)D * H * W;
    double sumL = 0.0, sumR = 0.0;
    if (cfg->reset_each_sweep) {
        memset(v_all, 0, sizeof(double) * 3 * V * n);
        memset(m_all, 0, sizeof(double) * 3 * V * n);
        memset(s_all, 0, sizeof(double) * 3 * V * n);
        for (int i = 0; i < n; ++i) k_all[i] = 0;
    }
    double *Ls = (double *)calloc(n, sizeof(double));
    double *Rs = (double *)calloc(n, sizeof(double));
    if (!Ls || !Rs) { free(Ls); free(Rs); return -1; }
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n; ++i) {
        double parts[2] = {0, 0};
        for (int it = 0; it < cfg->inner_steps; ++it)
            ora_subject_step(I_all + (long)i * V, A, v_all + (long)i * 3 * V, m_all + (long)i * 3 * V,
                             s_all + (long)i * 3 * V, &k_all[i], D, H, W, cfg, parts, NULL);
        Ls[i] = parts[0];
        Rs[i] = parts[1];
    }
    for (int i = 0; i < n; ++i) { sumL += Ls[i]; sumR += Rs[i]; }
    free(Ls);
    free(Rs);
    const double before = ora_centrality_metric(v_all, n, V);
    ora_centrality(v_all, n, 3 * V);
    const double after = ora_centrality_metric(v_all, n, V);
    int rc;
    if (cfg->dissim == 0)
        rc = ora_atlas_mean(I_all, v_all, n, D, H, W, cfg->T, A);
    else if (cfg->dissim == 2)
        rc = ora_atlas_median(I_all, v_all, n, D, H, W, cfg->T, A);
    else
        rc = ora_atlas_sgd(I_all, v_all, n, D, H, W, cfg, sweep, A, NULL);
    if (stats) {
        stats[0] = sumL / n;
        stats[1] = sumR / n;
        stats[2] = before;
        stats[3] = after;
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* One-shot segmentation (Eq. oneshot): I_i^(S) = A^(S) o Exp(-v_i).         */
/* Labels are sampled at the nearest voxel, r(p)_a = clamp(floor(p_a + 1/2), */
/* 0, n_a - 1) (reading: round half up; the paper names no tie rule).        */
/* ------------------------------------------------------------------------ */
int ora_propagate_labels(const uint8_t *labels, const double *v, int D, int H, int W, int T,
                         uint8_t *out)
{
    const int n[3] = {D, H, W};
    const long V = (long)D * H * W;
    double *u_all = (double *)malloc(sizeof(double) * 3 * V * (T + 1));
    if (!u_all) return -1;
    ora_exp(v, D, H, W, T, -1.0, u_all);
    const double *uT = u_all + (long)T * 3 * V;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < D; ++z)
        for (long y = 0; y < H; ++y)
            for (long x = 0; x < W; ++x) {
                const long l = lin3(n, z, y, x);
                double p[3];
                long q[3];
                sample_point(uT, V, l, z, y, x, p);
                for (int a = 0; a < 3; ++a) {
                    long r = (long)floor(p[a] + 0.5);
                    if (r < 0) r = 0;
                    if (r > n[a] - 1) r = n[a] - 1;
                    q[a] = r;
                }
                out[l] = labels[lin3(n, q[0], q[1], q[2])];
            }
    free(u_all);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Jacobian determinant of phi = id + u (Sec. "Evaluation metrics", the     */
/* folding rate |J|<0 %): det(I + grad u), central differences inside,      */
/* one-sided differences on the faces.                                       */
/* ------------------------------------------------------------------------ */
int ora_jacobian_det(const double *u, int D, int H, int W, double *det)
{
    const int n[3] = {D, H, W};
    const long V = (long)D * H * W;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < D; ++z)
        for (long y = 0; y < H; ++y)
            for (long x = 0; x < W; ++x) {
                const long q[3] = {z, y, x};
                double Jm[3][3];
                for (int b = 0; b < 3; ++b) {          /* derivative along axis b */
                    long lo[3] = {z, y, x}, hi[3] = {z, y, x};
                    double h;
                    if (q[b] == 0) { hi[b] = 1; h = 1.0; }
                    else if (q[b] == n[b] - 1) { lo[b] = n[b] - 2; h = 1.0; }
                    else { lo[b] = q[b] - 1; hi[b] = q[b] + 1; h = 2.0; }
                    const long lh = lin3(n, hi[0], hi[1], hi[2]);
                    const long ll = lin3(n, lo[0], lo[1], lo[2]);
                    for (int a = 0; a < 3; ++a)
                        Jm[a][b] = (a == b ? 1.0 : 0.0) + (u[a * V + lh] - u[a * V + ll]) / h;
                }
                det[lin3(n, z, y, x)] =
                    Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) -
                    Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +
                    Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
            }
    return 0;
}

/* Dice per label 1..nlab-1 (Sec. "Evaluation metrics"): 2|X n Y|/(|X|+|Y|),
 * background (0) excluded; a label absent from both maps scores -1. */
void ora_dice(const uint8_t *a, const uint8_t *b, long V, int nlab, double *per_label)
{
    for (int lab = 1; lab < nlab; ++lab) {
        long na = 0, nb = 0, both = 0;
        for (long l = 0; l < V; ++l) {
            const int ia = a[l] == lab, ib = b[l] == lab;
            na += ia;
            nb += ib;
            both += ia && ib;
        }
        per_label[lab - 1] = (na + nb) ? 2.0 * (double)both / (double)(na + nb) : -1.0;
    }
}

/* ===================================================================== */
/* Learned warm start (an addition to the method; the paper has none).   */
/* Plain definitions of the 3-D U-Net's convolution, in fp64.            */
/* Layout: x [B][C][D][H][W]; weights [cout][cin][3][3][3] with tap       */
/* (a, b, c) reading the input at (z + a - 1, y + b - 1, x + c - 1);      */
/* zero outside the volume (a 'same' cross-correlation).                 */
/* ===================================================================== */

/* out[b][co][p] = bias[co] + sum_{ci, tap} w[co][ci][tap] x[b][ci][p + off(tap)] */
int ora_conv3d(const double *x, int B, int cin, int D, int H, int W, const double *w, const double *bias,
               int cout, double *out)
{
    const long V = (long)D * H * W;
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int bb = 0; bb < B; ++bb)
        for (int co = 0; co < cout; ++co) {
            double *o = out + ((long)bb * cout + co) * V;
            for (long l = 0; l < V; ++l) o[l] = bias ? bias[co] : 0.0;
            for (int ci = 0; ci < cin; ++ci) {
                const double *xi = x + ((long)bb * cin + ci) * V;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        for (int c = 0; c < 3; ++c) {
                            const double wt = w[(((long)co * cin + ci) * 3 + a) * 9 + b * 3 + c];
                            for (int z = 0; z < D; ++z) {
                                const int zz = z + a - 1;
                                if (zz < 0 || zz >= D) continue;
                                for (int y = 0; y < H; ++y) {
                                    const int yy = y + b - 1;
                                    if (yy < 0 || yy >= H) continue;
                                    for (int xq = 0; xq < W; ++xq) {
                                        const int xx = xq + c - 1;
                                        if (xx < 0 || xx >= W) continue;
                                        o[((long)z * H + y) * W + xq] += wt * xi[((long)zz * H + yy) * W + xx];
                                    }
                                }
                            }
                        }
            }
        }
    return 0;
}

/* Adjoint of ora_conv3d in its input: every product w * x[p + off] of the
 * forward sum sends gz[b][co][p] * w back to the input voxel p + off it read
 * (a scatter, written as the transpose of the forward map). */
int ora_conv3d_adjoint_input(const double *gz, int B, int cout, int D, int H, int W, const double *w, int cin,
                             double *gx)
{
    const long V = (long)D * H * W;
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int bb = 0; bb < B; ++bb)
        for (int ci = 0; ci < cin; ++ci) {
            double *g = gx + ((long)bb * cin + ci) * V;
            for (long l = 0; l < V; ++l) g[l] = 0.0;
            for (int co = 0; co < cout; ++co) {
                const double *gzo = gz + ((long)bb * cout + co) * V;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        for (int c = 0; c < 3; ++c) {
                            const double wt = w[(((long)co * cin + ci) * 3 + a) * 9 + b * 3 + c];
                            for (int z = 0; z < D; ++z) {
                                const int zz = z + a - 1;
                                if (zz < 0 || zz >= D) continue;
                                for (int y = 0; y < H; ++y) {
                                    const int yy = y + b - 1;
                                    if (yy < 0 || yy >= H) continue;
                                    for (int xq = 0; xq < W; ++xq) {
                                        const int xx = xq + c - 1;
                                        if (xx < 0 || xx >= W) continue;
                                        g[((long)zz * H + yy) * W + xx] += wt * gzo[((long)z * H + y) * W + xq];
                                    }
                                }
                            }
                        }
            }
        }
    return 0;
}

/* Gradients of sum_{b,co,p} gz[b][co][p] out[b][co][p] in the weights and
 * biases: dw[co][ci][tap] = sum_{b,p} gz[b][co][p] x[b][ci][p + off(tap)],
 * db[co] = sum_{b,p} gz[b][co][p] (db may be NULL). */
int ora_conv3d_wgrad(const double *x, const double *gz, int B, int cin, int cout, int D, int H, int W, double *dw,
                     double *db)
{
    const long V = (long)D * H * W;
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int co = 0; co < cout; ++co)
        for (int ci = 0; ci < cin; ++ci)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    for (int c = 0; c < 3; ++c) {
                        double s = 0.0;
                        for (int bb = 0; bb < B; ++bb) {
                            const double *xi = x + ((long)bb * cin + ci) * V;
                            const double *gzo = gz + ((long)bb * cout + co) * V;
                            for (int z = 0; z < D; ++z) {
                                const int zz = z + a - 1;
                                if (zz < 0 || zz >= D) continue;
                                for (int y = 0; y < H; ++y) {
                                    const int yy = y + b - 1;
                                    if (yy < 0 || yy >= H) continue;
                                    for (int xq = 0; xq < W; ++xq) {
                                        const int xx = xq + c - 1;
                                        if (xx < 0 || xx >= W) continue;
                                        s += gzo[((long)z * H + y) * W + xq] * xi[((long)zz * H + yy) * W + xx];
                                    }
                                }
                            }
                        }
                        dw[(((long)co * cin + ci) * 3 + a) * 9 + b * 3 + c] = s;
                    }
    if (db)
        for (int co = 0; co < cout; ++co) {
            double s = 0.0;
            for (int bb = 0; bb < B; ++bb)
                for (long l = 0; l < V; ++l) s += gz[((long)bb * cout + co) * V + l];
            db[co] = s;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Composition of two maps given as displacements (Sec. "Diffeomorphisms":   */
/* phi = id + u): (phi_b o phi_a)(x) = x + a(x) + b(x + a(x)), so the        */
/* displacement is out(x) = a(x) + S(b, x + a(x)), trilinear, border padded. */
/* ------------------------------------------------------------------------ */
int ora_compose(const double *a, const double *b, int D, int H, int W, double *out)
{
    const long V = (long)D * H * W;
    const int n[3] = {D, H, W};
#pragma omp parallel for schedule(static)
    for (long z = 0; z < D; ++z)
        for (long y = 0; y < H; ++y)
            for (long x = 0; x < W; ++x) {
                const long l = lin3(n, z, y, x);
                const double pz = (double)z + a[l], py = (double)y + a[V + l], px = (double)x + a[2 * V + l];
                for (int ch = 0; ch < 3; ++ch)
                    out[ch * V + l] = a[ch * V + l] + ora_sample(b + ch * V, D, H, W, pz, py, px, NULL);
            }
    return 0;
}

/* Diffeomorphism report of one velocity field (Sec. "Evaluation metrics":
 * folding rate |J|<0 %; Sec. "Diffeomorphisms": Exp(-v) inverts Exp(v)):
 * stats[0] = fraction of voxels with det(I + grad u+) <= 0, u+ = Exp(v);
 * stats[1], stats[2] = mean and max over voxels of |r(x)|, r the
 * displacement of Exp(-v) o Exp(v) (zero for an exact inverse);
 * stats[3] = min det(I + grad u+). */
int ora_diffeo_report(const double *v, int D, int H, int W, int T, double *stats)
{
    const long V = (long)D * H * W;
    double *up = (double *)malloc(sizeof(double) * 3 * V * (T + 1));
    double *um = (double *)malloc(sizeof(double) * 3 * V * (T + 1));
    double *r = (double *)malloc(sizeof(double) * 3 * V);
    double *det = (double *)malloc(sizeof(double) * V);
    if (!up || !um || !r || !det) {
        free(up); free(um); free(r); free(det);
        return -1;
    }
    ora_exp(v, D, H, W, T, 1.0, up);
    ora_exp(v, D, H, W, T, -1.0, um);
    const double *uP = up + (long)T * 3 * V, *uM = um + (long)T * 3 * V;
    ora_compose(uP, uM, D, H, W, r);
    ora_jacobian_det(uP, D, H, W, det);
    long neg = 0;
    double sum = 0.0, mx = 0.0, mn = det[0];
    for (long l = 0; l < V; ++l) {
        const double e = sqrt(r[l] * r[l] + r[V + l] * r[V + l] + r[2 * V + l] * r[2 * V + l]);
        sum += e;
        if (e > mx) mx = e;
        if (det[l] <= 0.0) ++neg;
        if (det[l] < mn) mn = det[l];
    }
    stats[0] = (double)neg / (double)V;
    stats[1] = sum / (double)V;
    stats[2] = mx;
    stats[3] = mn;
    free(up); free(um); free(r); free(det);
    return 0;
}
