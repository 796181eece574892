/*
 * enuf_oracle.c -- plain, slow, FP64 CPU oracle for the ENUF-DPD hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see enuf_oracle.h). Nothing here is blocked,
 * fused or reordered beyond what the equations state: the real-space sum is a
 * plain double loop over pairs, the direct reciprocal sum a plain loop over
 * integer k, and the naive ENUF plain window loops plus plain per-dimension
 * DFTs. Build with -ffp-contract=off so that no multiply-add is fused behind
 * the reader's back. Every decision (wrap, grid base, pair cutoff) is taken
 * in FP64 on the inputs as given; an FP32 caller passes float-rounded inputs.
 */
#include "enuf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------ */
/* Geometry                                                            */
/* ------------------------------------------------------------------ */

double orc_wrap(double x, double L)
{
    if (x >= 0.0 && x < L) return x;
    double w = x - L * floor(x / L);
    if (w >= L || w < 0.0) w = 0.0; /* only reachable through rounding */
    return w;
}

/* Wrapped copy of the positions. */
static double* wrapped_positions(const orc_params* P, int n, const double* pos)
{
    double* w = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!w) return NULL;
    for (int i = 0; i < 3 * n; ++i) w[i] = orc_wrap(pos[i], P->L);
    return w;
}

/* Minimum-image displacement d = x_i - x_j and the cutoff decision r < rc.
 * Returns 1 and sets d, r when the pair is inside the cutoff. With
 * r_c <= L/2 the minimum image is the only periodic image inside r_c, so this
 * is the n-sum of Eq. 16 restricted to |r_ij + nL| < r_c. */
static int pair_within(const orc_params* P, const double* xi, const double* xj,
                       double rc, double d[3], double* r)
{
    const double L = P->L;
    for (int t = 0; t < 3; ++t) {
        double dd = xi[t] - xj[t];
        if (dd > 0.5 * L) dd -= L;
        else if (dd < -0.5 * L) dd += L;
        d[t] = dd;
    }
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < rc * rc)) return 0;
    if (r2 <= 0.0) return 0; /* coincident beads: no direction */
    *r = sqrt(r2);
    return 1;
}

/* ------------------------------------------------------------------ */
/* Slater-smeared pair interaction (Eq. 27, Eq. 28, Fig. 2)            */
/* ------------------------------------------------------------------ */

double orc_B1(double beta, double r)
{
    if (beta <= 0.0) return 1.0;
    return 1.0 - (1.0 + beta * r) * exp(-2.0 * beta * r);
}

double orc_B2(double beta, double r)
{
    if (beta <= 0.0) return 1.0;
    return 1.0 - (1.0 + 2.0 * beta * r * (1.0 + beta * r)) * exp(-2.0 * beta * r);
}

double orc_slater_energy(double beta, double r) { return orc_B1(beta, r) / r; }
double orc_slater_force(double beta, double r) { return orc_B2(beta, r) / (r * r); }

/* ------------------------------------------------------------------ */
/* Real space: erfc Ewald term (Eq. 31) plus the Slater correction      */
/* -(1+beta r)e^{-2 beta r}/r, i.e. phi_S(r) - erf(alpha r)/r.          */
/* Pair energy u(r), and f(r) = -du/dr (the corrected Eq. 32).         */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n
 * (initial guesses cos(pi (i - 1/4)/(n + 1/2))). */
#define GL_N 16
static void gauss_legendre(double* x, double* w)
{
    for (int i = 0; i < GL_N; ++i) {
        double z = cos(M_PI * (i + 0.75) / (GL_N + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= GL_N; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = GL_N * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void orc_slater_I(const orc_params* P, double r, int rho_one, double* I, double* dI)
{
    double gx[GL_N], gw[GL_N];
    gauss_legendre(gx, gw);
    const double a = P->alpha, be = P->beta;
    /* e^{-k^2/(4 alpha^2)} < 1e-21 beyond kmax; 512 panels of 16 nodes */
    const double kmax = 2.0 * a * sqrt(50.0);
    const int npan = 512;
    const double h = kmax / npan;
    double si = 0.0, sd = 0.0;
    for (int pnl = 0; pnl < npan; ++pnl) {
        const double k0 = pnl * h;
        for (int t = 0; t < GL_N; ++t) {
            const double k = k0 + 0.5 * h * (gx[t] + 1.0);
            double wk = exp(-k * k / (4.0 * a * a));
            if (!rho_one) {
                const double c = 1.0 + k * k / (4.0 * be * be);
                wk /= c * c;
            }
            const double kr = k * r;
            si += 0.5 * h * gw[t] * wk * (r == 0.0 ? 0.0 : sin(kr) / k);
            sd += 0.5 * h * gw[t] * wk * cos(kr);
        }
    }
    *I = 2.0 / M_PI * si;
    *dI = 2.0 / M_PI * sd;
}

/* Reading C real-space pair: u = phi_S(r) - I(r)/r, f = -du/dr. */
static void real_pair_c(const orc_params* P, double r, double* u, double* f)
{
    double I, dI;
    orc_slater_I(P, r, 0, &I, &dI);
    *u = orc_slater_energy(P->beta, r) - I / r;
    *f = orc_slater_force(P->beta, r) + (dI * r - I) / (r * r);
}

static void real_pair(const orc_params* P, double r, double* u, double* f)
{
    if (P->slater_k) {
        real_pair_c(P, r, u, f);
        return;
    }
    const double a = P->alpha;
    double uu = erfc(a * r) / r;
    double ff = erfc(a * r) / (r * r) + (2.0 * a / sqrt(M_PI)) * exp(-a * a * r * r) / r;
    if (P->beta > 0.0) {
        const double be = P->beta;
        const double e = exp(-2.0 * be * r);
        uu -= (1.0 + be * r) * e / r;
        ff -= (1.0 + 2.0 * be * r + 2.0 * be * be * r * r) * e / (r * r);
    }
    *u = uu;
    *f = ff;
}

int orc_real_space(const orc_params* P, int n, const double* pos, const double* q,
                   double* F, double* EW, const int* sample, int nsample)
{
    if (n < 0 || P->r_cut > 0.5 * P->L || (P->slater_k && P->beta <= 0.0)) return ORC_EINVAL;
    double* x = wrapped_positions(P, n, pos);
    if (!x) return ORC_ENOMEM;
    const double rc = P->r_cut, kap = P->kappa;

    /* energy and virial: every charged pair i < j once */
    if (EW) {
        double E = 0.0, W = 0.0;
        for (int i = 0; i < n; ++i) {
            if (q[i] == 0.0) continue;
            for (int j = i + 1; j < n; ++j) {
                if (q[j] == 0.0) continue;
                double d[3], r, u, f;
                if (!pair_within(P, &x[3 * i], &x[3 * j], rc, d, &r)) continue;
                real_pair(P, r, &u, &f);
                E += kap * q[i] * q[j] * u;
                W += kap * q[i] * q[j] * f * r;
            }
        }
        EW[0] = E;
        EW[1] = W;
    }
    /* forces: F_i = sum_j kappa q_i q_j f(r) r_ij / r */
    if (F) {
        const int nout = sample ? nsample : n;
        #pragma omp parallel for schedule(dynamic, 16)
        for (int s = 0; s < nout; ++s) {
            const int i = sample ? sample[s] : s;
            double Fi[3] = {0.0, 0.0, 0.0};
            if (q[i] != 0.0) {
                for (int j = 0; j < n; ++j) {
                    if (j == i || q[j] == 0.0) continue;
                    double d[3], r, u, f;
                    if (!pair_within(P, &x[3 * i], &x[3 * j], rc, d, &r)) continue;
                    real_pair(P, r, &u, &f);
                    for (int t = 0; t < 3; ++t) Fi[t] += kap * q[i] * q[j] * f * d[t] / r;
                }
            }
            for (int t = 0; t < 3; ++t) F[3 * s + t] = Fi[t];
        }
    }
    free(x);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Mode set I_M (Eq. 9) read as |k_t| <= n_c = M/2 - 1                  */
/* ------------------------------------------------------------------ */

static int in_mask(const orc_params* P, int kx, int ky, int kz)
{
    const int nc = P->M / 2 - 1;
    if (kx == 0 && ky == 0 && kz == 0) return 0;
    if (abs(kx) > nc || abs(ky) > nc || abs(kz) > nc) return 0;
    if (P->kmask == 1 && kx * kx + ky * ky + kz * kz > nc * nc) return 0;
    return 1;
}

/* Ewald influence function of Eq. 18 for integer k: e^{-(pi k)^2/(alpha L)^2}/k^2 */
/* Slater form factor (1 + k^2/(4 beta^2))^{-2}, k = 2 pi |m| / L, as (1 + t)^{-2} */
static double slater_t(const orc_params* P, double m2)
{
    const double bL = P->beta * P->L;
    return M_PI * M_PI * m2 / (bL * bL);
}
static double influence(const orc_params* P, int kx, int ky, int kz)
{
    const double k2 = (double)kx * kx + (double)ky * ky + (double)kz * kz;
    const double aL = P->alpha * P->L;
    double f = exp(-M_PI * M_PI * k2 / (aL * aL)) / k2;
    if (P->slater_k) {
        const double t = 1.0 + slater_t(P, k2);
        f /= t * t;
    }
    return f;
}

/* Virial weight of one mode: -L d/dL of its energy term over the term. */
static double virial_weight(const orc_params* P, int kx, int ky, int kz)
{
    const double k2 = (double)kx * kx + (double)ky * ky + (double)kz * kz;
    const double aL = P->alpha * P->L;
    double w = 1.0 - 2.0 * M_PI * M_PI * k2 / (aL * aL);
    if (P->slater_k) {   /* the form factor depends on L through k = 2 pi |m| / L */
        const double t = slater_t(P, k2);
        w -= 4.0 * t / (1.0 + t);
    }
    return w;
}

/* ------------------------------------------------------------------ */
/* Direct reciprocal sum (Eq. 18, 19, 22-24)                           */
/* ------------------------------------------------------------------ */

int orc_recip_direct(const orc_params* P, int n, const double* pos, const double* q,
                     double* F, double* EW, const int* sample, int nsample)
{
    const int nc = P->M / 2 - 1;
    if (n < 0 || nc < 1) return ORC_EINVAL;
    double* x = wrapped_positions(P, n, pos);
    if (!x) return ORC_ENOMEM;
    const double L = P->L, kap = P->kappa;
    const int K = 2 * nc + 1;
    const size_t nk = (size_t)K * K * K;
    double* Sre = (double*)calloc(nk, sizeof(double));
    double* Sim = (double*)calloc(nk, sizeof(double));
    if (!Sre || !Sim) { free(x); free(Sre); free(Sim); return ORC_ENOMEM; }

    /* structure factor S(k) = sum_j q_j exp(-2 pi i k.x_j), x_j = r_j / L (Eq. 19) */
    #pragma omp parallel for schedule(dynamic, 4)
    for (int ix = 0; ix < K; ++ix) {
        for (int iy = 0; iy < K; ++iy) {
            for (int iz = 0; iz < K; ++iz) {
                const int kx = ix - nc, ky = iy - nc, kz = iz - nc;
                if (!in_mask(P, kx, ky, kz)) continue;
                double sr = 0.0, si = 0.0;
                for (int j = 0; j < n; ++j) {
                    if (q[j] == 0.0) continue;
                    const double ph = 2.0 * M_PI * (kx * x[3 * j] + ky * x[3 * j + 1] + kz * x[3 * j + 2]) / L;
                    sr += q[j] * cos(ph);
                    si -= q[j] * sin(ph);
                }
                const size_t id = ((size_t)ix * K + iy) * K + iz;
                Sre[id] = sr;
                Sim[id] = si;
            }
        }
    }
    /* energy U^{E,K} = kappa/(2 pi L) sum_{k != 0} f(k) |S(k)|^2 (Eq. 18) */
    if (EW) {
        double E = 0.0, W = 0.0;
        for (int ix = 0; ix < K; ++ix)
            for (int iy = 0; iy < K; ++iy)
                for (int iz = 0; iz < K; ++iz) {
                    const int kx = ix - nc, ky = iy - nc, kz = iz - nc;
                    if (!in_mask(P, kx, ky, kz)) continue;
                    const size_t id = ((size_t)ix * K + iy) * K + iz;
                    const double e = influence(P, kx, ky, kz) * (Sre[id] * Sre[id] + Sim[id] * Sim[id]);
                    E += e;
                    W += e * virial_weight(P, kx, ky, kz);
                }
        EW[0] = kap / (2.0 * M_PI * L) * E;
        EW[1] = kap / (2.0 * M_PI * L) * W;
    }
    /* force F_i = kappa (2 q_i / L^2) sum_k k f(k) Im{S(k) exp(2 pi i k.x_i)} (Eq. 24) */
    if (F) {
        const int nout = sample ? nsample : n;
        #pragma omp parallel for schedule(dynamic, 8)
        for (int s = 0; s < nout; ++s) {
            const int i = sample ? sample[s] : s;
            double Fi[3] = {0.0, 0.0, 0.0};
            if (q[i] != 0.0) {
                for (int ix = 0; ix < K; ++ix)
                    for (int iy = 0; iy < K; ++iy)
                        for (int iz = 0; iz < K; ++iz) {
                            const int kx = ix - nc, ky = iy - nc, kz = iz - nc;
                            if (!in_mask(P, kx, ky, kz)) continue;
                            const size_t id = ((size_t)ix * K + iy) * K + iz;
                            const double ph = 2.0 * M_PI * (kx * x[3 * i] + ky * x[3 * i + 1] + kz * x[3 * i + 2]) / L;
                            /* Im{(Sre + i Sim)(cos ph + i sin ph)} */
                            const double im = Sre[id] * sin(ph) + Sim[id] * cos(ph);
                            const double w = influence(P, kx, ky, kz) * im;
                            Fi[0] += kx * w;
                            Fi[1] += ky * w;
                            Fi[2] += kz * w;
                        }
            }
            for (int t = 0; t < 3; ++t) F[3 * s + t] = kap * 2.0 * q[i] / (L * L) * Fi[t];
        }
    }
    free(x);
    free(Sre);
    free(Sim);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Naive ENUF (Table 2 step 4(ii))                                     */
/* ------------------------------------------------------------------ */

/* Gaussian window in grid units: psi(u) = (pi b)^{-1/2} exp(-u^2 / b). */
static double window(double b, double u) { return exp(-u * u / b) / sqrt(M_PI * b); }

/* Its Fourier factor per dimension, c(k) = n * psi_hat(k) = exp(-b (pi k / n)^2):
 * the DFT of the periodised window sampled on the n-grid equals c(k) times the
 * phase of the bead, up to the aliasing and truncation errors. */
static double window_hat(double b, int k, int ng)
{
    const double t = M_PI * (double)k / (double)ng;
    return exp(-b * t * t);
}

/* Grid coordinate of a wrapped position x_w in [0, L): u = n x_w / L in
 * [0, n) (Eq. 14 evaluates the window at n x - l), base = floor(u), and the
 * fraction u - base; u = n (reached only by rounding) wraps to 0. */
static void grid_coord(double xw, double L, int ng, int* base, double* frac)
{
    double u = (double)ng * (xw / L);   /* n times the fractional coordinate */
    if (u >= (double)ng) u -= (double)ng;
    const double bse = floor(u);
    *base = (int)bse;
    *frac = u - bse;
}

static int imod(int a, int m)
{
    int r = a % m;
    return r < 0 ? r + m : r;
}

int orc_recip_enuf(const orc_params* P, int n, const double* pos, const double* q,
                   double* F, double* EW, double* grid, double* hfield,
                   const int* sample, int nsample)
{
    const int M = P->M, nc = M / 2 - 1, p = P->p, sg = P->sigma_s;
    const int ng = sg * M;
    if (n < 0 || nc < 1 || p < 1 || sg < 2 || 2 * p > ng) return ORC_EINVAL;
    if (P->deriv && p > 8) return ORC_EINVAL;   /* the gradient path keeps 2p <= 16 taps */
    const double L = P->L, kap = P->kappa;
    const double b = 2.0 * sg * p / ((2.0 * sg - 1.0) * M_PI);
    const int K = 2 * nc + 1, T = 2 * p;
    const size_t ng3 = (size_t)ng * ng * ng;

    double* x = wrapped_positions(P, n, pos);
    double* cs = (double*)malloc(sizeof(double) * ng);
    double* sn = (double*)malloc(sizeof(double) * ng);
    int* base = (int*)malloc(sizeof(int) * 3 * (size_t)(n > 0 ? n : 1));
    double* wgt = (double*)malloc(sizeof(double) * 3 * T * (size_t)(n > 0 ? n : 1));
    double* g = (double*)calloc(ng3, sizeof(double));
    if (!x || !cs || !sn || !base || !wgt || !g) {
        free(x); free(cs); free(sn); free(base); free(wgt); free(g);
        return ORC_ENOMEM;
    }
    for (int m = 0; m < ng; ++m) {
        cs[m] = cos(2.0 * M_PI * m / ng);
        sn[m] = sin(2.0 * M_PI * m / ng);
    }

    /* per-bead taps: l_t = base_t - p + 1 + a, a = 0..2p-1, weight psi(u_t - l_t) */
    for (int j = 0; j < n; ++j) {
        for (int t = 0; t < 3; ++t) {
            double fr;
            grid_coord(x[3 * j + t], L, ng, &base[3 * j + t], &fr);
            for (int a = 0; a < T; ++a)
                wgt[((size_t)j * 3 + t) * T + a] = window(b, fr + (double)(p - 1 - a));
        }
    }

    /* transposed NFFT, part 1: spread g(l) = sum_j q_j prod_t psi(u_jt - l_t) (Eq. 14/19) */
    for (int j = 0; j < n; ++j) {
        if (q[j] == 0.0) continue;
        const double* wx = &wgt[((size_t)j * 3 + 0) * T];
        const double* wy = &wgt[((size_t)j * 3 + 1) * T];
        const double* wz = &wgt[((size_t)j * 3 + 2) * T];
        for (int c = 0; c < T; ++c) {
            const int lz = imod(base[3 * j + 2] - p + 1 + c, ng);
            for (int bb = 0; bb < T; ++bb) {
                const int ly = imod(base[3 * j + 1] - p + 1 + bb, ng);
                for (int a = 0; a < T; ++a) {
                    const int lx = imod(base[3 * j] - p + 1 + a, ng);
                    g[((size_t)lz * ng + ly) * ng + lx] += q[j] * wx[a] * wy[bb] * wz[c];
                }
            }
        }
    }
    if (grid) memcpy(grid, g, sizeof(double) * ng3);

    /* transposed NFFT, part 2: Fhat(k) = sum_l g(l) exp(-2 pi i k.l / n), |k_t| <= n_c,
     * one plain DFT per dimension: x, then y, then z. */
    const size_t nA1 = (size_t)K * ng * ng, nA2 = (size_t)K * K * ng, nF = (size_t)K * K * K;
    double* A1r = (double*)calloc(nA1, sizeof(double));
    double* A1i = (double*)calloc(nA1, sizeof(double));
    double* A2r = (double*)calloc(nA2, sizeof(double));
    double* A2i = (double*)calloc(nA2, sizeof(double));
    double* Fr = (double*)calloc(nF, sizeof(double));
    double* Fi = (double*)calloc(nF, sizeof(double));
    if (!A1r || !A1i || !A2r || !A2i || !Fr || !Fi) {
        free(x); free(cs); free(sn); free(base); free(wgt); free(g);
        free(A1r); free(A1i); free(A2r); free(A2i); free(Fr); free(Fi);
        return ORC_ENOMEM;
    }
    /* A1[kx][lz][ly] = sum_lx g[lz][ly][lx] e^{-2 pi i kx lx / n} */
    #pragma omp parallel for schedule(static)
    for (int ix = 0; ix < K; ++ix) {
        const int kx = ix - nc;
        for (int lz = 0; lz < ng; ++lz)
            for (int ly = 0; ly < ng; ++ly) {
                double sr = 0.0, si = 0.0;
                for (int lx = 0; lx < ng; ++lx) {
                    const int m = imod(kx * lx, ng);
                    const double v = g[((size_t)lz * ng + ly) * ng + lx];
                    sr += v * cs[m];
                    si -= v * sn[m];
                }
                A1r[((size_t)ix * ng + lz) * ng + ly] = sr;
                A1i[((size_t)ix * ng + lz) * ng + ly] = si;
            }
    }
    /* A2[kx][ky][lz] = sum_ly A1[kx][lz][ly] e^{-2 pi i ky ly / n} */
    #pragma omp parallel for schedule(static)
    for (int ix = 0; ix < K; ++ix)
        for (int iy = 0; iy < K; ++iy) {
            const int ky = iy - nc;
            for (int lz = 0; lz < ng; ++lz) {
                double sr = 0.0, si = 0.0;
                for (int ly = 0; ly < ng; ++ly) {
                    const int m = imod(ky * ly, ng);
                    const double ar = A1r[((size_t)ix * ng + lz) * ng + ly];
                    const double ai = A1i[((size_t)ix * ng + lz) * ng + ly];
                    /* (ar + i ai)(cos - i sin) */
                    sr += ar * cs[m] + ai * sn[m];
                    si += ai * cs[m] - ar * sn[m];
                }
                A2r[((size_t)ix * K + iy) * ng + lz] = sr;
                A2i[((size_t)ix * K + iy) * ng + lz] = si;
            }
        }
    /* Fhat[kx][ky][kz] = sum_lz A2[kx][ky][lz] e^{-2 pi i kz lz / n} */
    #pragma omp parallel for schedule(static)
    for (int ix = 0; ix < K; ++ix)
        for (int iy = 0; iy < K; ++iy)
            for (int iz = 0; iz < K; ++iz) {
                const int kz = iz - nc;
                double sr = 0.0, si = 0.0;
                for (int lz = 0; lz < ng; ++lz) {
                    const int m = imod(kz * lz, ng);
                    const double ar = A2r[((size_t)ix * K + iy) * ng + lz];
                    const double ai = A2i[((size_t)ix * K + iy) * ng + lz];
                    sr += ar * cs[m] + ai * sn[m];
                    si += ai * cs[m] - ar * sn[m];
                }
                Fr[((size_t)ix * K + iy) * K + iz] = sr;
                Fi[((size_t)ix * K + iy) * K + iz] = si;
            }
    free(A1r); free(A1i); free(A2r); free(A2i);

    /* S(k) ~ Fhat(k) / prod_t c(k_t); U^{E,K} = kappa/(2 pi L) sum f(k)|S|^2 (Eq. 20);
     * g_hat_a(k) = k_a f(k) S(k) (Eq. 24), divided once more by prod_t c(k_t) so
     * that the conjugated NFFT below reproduces sum_k g_hat e^{2 pi i k.x}. */
    double* Gr = (double*)calloc(3 * nF, sizeof(double));
    double* Gi = (double*)calloc(3 * nF, sizeof(double));
    if (!Gr || !Gi) {
        free(x); free(cs); free(sn); free(base); free(wgt); free(g); free(Fr); free(Fi);
        free(Gr); free(Gi);
        return ORC_ENOMEM;
    }
    const int deriv = P->deriv;
    const int nfield = deriv ? 1 : 3;
    double E = 0.0, W = 0.0;
    for (int ix = 0; ix < K; ++ix)
        for (int iy = 0; iy < K; ++iy)
            for (int iz = 0; iz < K; ++iz) {
                const int kx = ix - nc, ky = iy - nc, kz = iz - nc;
                if (!in_mask(P, kx, ky, kz)) continue;
                const size_t id = ((size_t)ix * K + iy) * K + iz;
                const double c = window_hat(b, kx, ng) * window_hat(b, ky, ng) * window_hat(b, kz, ng);
                const double Sr = Fr[id] / c, Si = Fi[id] / c;
                const double f = influence(P, kx, ky, kz);
                const double e = f * (Sr * Sr + Si * Si);
                E += e;
                W += e * virial_weight(P, kx, ky, kz);
                if (deriv) {   /* the potential-like field: f S / c */
                    Gr[id] = f * Sr / c;
                    Gi[id] = f * Si / c;
                } else {
                    const int kv[3] = {kx, ky, kz};
                    for (int a = 0; a < 3; ++a) {
                        Gr[a * nF + id] = kv[a] * f * Sr / c;
                        Gi[a * nF + id] = kv[a] * f * Si / c;
                    }
                }
            }
    if (EW) {
        EW[0] = kap / (2.0 * M_PI * L) * E;
        EW[1] = kap / (2.0 * M_PI * L) * W;
    }

    /* conjugated NFFT: h_a(l) = sum_k g_hat'_a(k) e^{+2 pi i k.l / n} (plain inverse DFT
     * per dimension: z, then y, then x), then g_{i,a} = sum_l psi(u_i - l) h_a(l) and
     * F_{i,a} = kappa (2 q_i / L^2) Im g_{i,a} (Eq. 25). */
    const int nout = sample ? nsample : n;
    if (F)
        for (int s = 0; s < nout; ++s)
            for (int t = 0; t < 3; ++t) F[3 * s + t] = 0.0;
    if (F || hfield) {
        double* B1r = (double*)malloc(sizeof(double) * K * K * ng);
        double* B1i = (double*)malloc(sizeof(double) * K * K * ng);
        double* B2r = (double*)malloc(sizeof(double) * K * ng * ng);
        double* B2i = (double*)malloc(sizeof(double) * K * ng * ng);
        double* Hi = (double*)malloc(sizeof(double) * ng3);
        if (!B1r || !B1i || !B2r || !B2i || !Hi) {
            free(B1r); free(B1i); free(B2r); free(B2i); free(Hi);
            free(x); free(cs); free(sn); free(base); free(wgt); free(g); free(Fr); free(Fi);
            free(Gr); free(Gi);
            return ORC_ENOMEM;
        }
        for (int a = 0; a < nfield; ++a) {
            const double* gr = &Gr[a * nF];
            const double* gi = &Gi[a * nF];
            /* B1[kx][ky][lz] = sum_kz G[kx][ky][kz] e^{+2 pi i kz lz / n} */
            #pragma omp parallel for schedule(static)
            for (int ix = 0; ix < K; ++ix)
                for (int iy = 0; iy < K; ++iy)
                    for (int lz = 0; lz < ng; ++lz) {
                        double sr = 0.0, si = 0.0;
                        for (int iz = 0; iz < K; ++iz) {
                            const int m = imod((iz - nc) * lz, ng);
                            const size_t id = ((size_t)ix * K + iy) * K + iz;
                            /* (gr + i gi)(cos + i sin) */
                            sr += gr[id] * cs[m] - gi[id] * sn[m];
                            si += gi[id] * cs[m] + gr[id] * sn[m];
                        }
                        B1r[((size_t)ix * K + iy) * ng + lz] = sr;
                        B1i[((size_t)ix * K + iy) * ng + lz] = si;
                    }
            /* B2[kx][lz][ly] = sum_ky B1[kx][ky][lz] e^{+2 pi i ky ly / n} */
            #pragma omp parallel for schedule(static)
            for (int ix = 0; ix < K; ++ix)
                for (int lz = 0; lz < ng; ++lz)
                    for (int ly = 0; ly < ng; ++ly) {
                        double sr = 0.0, si = 0.0;
                        for (int iy = 0; iy < K; ++iy) {
                            const int m = imod((iy - nc) * ly, ng);
                            const double br = B1r[((size_t)ix * K + iy) * ng + lz];
                            const double bi = B1i[((size_t)ix * K + iy) * ng + lz];
                            sr += br * cs[m] - bi * sn[m];
                            si += bi * cs[m] + br * sn[m];
                        }
                        B2r[((size_t)ix * ng + lz) * ng + ly] = sr;
                        B2i[((size_t)ix * ng + lz) * ng + ly] = si;
                    }
            /* Im h[lz][ly][lx] = Im sum_kx B2[kx][lz][ly] e^{+2 pi i kx lx / n}
             * (deriv = 1: the real part, h being real) */
            #pragma omp parallel for schedule(static)
            for (int lz = 0; lz < ng; ++lz)
                for (int ly = 0; ly < ng; ++ly)
                    for (int lx = 0; lx < ng; ++lx) {
                        double sr = 0.0, si = 0.0;
                        for (int ix = 0; ix < K; ++ix) {
                            const int m = imod((ix - nc) * lx, ng);
                            const double br = B2r[((size_t)ix * ng + lz) * ng + ly];
                            const double bi = B2i[((size_t)ix * ng + lz) * ng + ly];
                            sr += br * cs[m] - bi * sn[m];
                            si += bi * cs[m] + br * sn[m];
                        }
                        Hi[((size_t)lz * ng + ly) * ng + lx] = deriv ? sr : si;
                    }
            if (hfield) memcpy(&hfield[(size_t)a * ng3], Hi, sizeof(double) * ng3);
            if (F && deriv) {
                /* F_{i,t} = -(kappa q_i n/(pi L^2)) sum_l dPsi_t(n x_i - l) h(l) */
                #pragma omp parallel for schedule(static)
                for (int s = 0; s < nout; ++s) {
                    const int i = sample ? sample[s] : s;
                    if (q[i] == 0.0) continue;
                    double w[3][16], dw[3][16];
                    for (int t = 0; t < 3; ++t) {
                        double fr;
                        int bt;
                        grid_coord(x[3 * i + t], L, ng, &bt, &fr);
                        for (int aa = 0; aa < T; ++aa) {
                            const double d = fr + (double)(p - 1 - aa);   /* n x - l */
                            w[t][aa] = wgt[((size_t)i * 3 + t) * T + aa];
                            dw[t][aa] = -2.0 * d / b * w[t][aa];
                        }
                    }
                    double acc[3] = {0.0, 0.0, 0.0};
                    for (int c = 0; c < T; ++c) {
                        const int lz = imod(base[3 * i + 2] - p + 1 + c, ng);
                        for (int bb = 0; bb < T; ++bb) {
                            const int ly = imod(base[3 * i + 1] - p + 1 + bb, ng);
                            for (int aa = 0; aa < T; ++aa) {
                                const int lx = imod(base[3 * i] - p + 1 + aa, ng);
                                const double hv = Hi[((size_t)lz * ng + ly) * ng + lx];
                                acc[0] += dw[0][aa] * w[1][bb] * w[2][c] * hv;
                                acc[1] += w[0][aa] * dw[1][bb] * w[2][c] * hv;
                                acc[2] += w[0][aa] * w[1][bb] * dw[2][c] * hv;
                            }
                        }
                    }
                    for (int t = 0; t < 3; ++t) F[3 * s + t] = -kap * q[i] * ng / (M_PI * L * L) * acc[t];
                }
            }
            if (F && !deriv) {
                #pragma omp parallel for schedule(static)
                for (int s = 0; s < nout; ++s) {
                    const int i = sample ? sample[s] : s;
                    if (q[i] == 0.0) continue;
                    const double* wx = &wgt[((size_t)i * 3 + 0) * T];
                    const double* wy = &wgt[((size_t)i * 3 + 1) * T];
                    const double* wz = &wgt[((size_t)i * 3 + 2) * T];
                    double acc = 0.0;
                    for (int c = 0; c < T; ++c) {
                        const int lz = imod(base[3 * i + 2] - p + 1 + c, ng);
                        for (int bb = 0; bb < T; ++bb) {
                            const int ly = imod(base[3 * i + 1] - p + 1 + bb, ng);
                            for (int aa = 0; aa < T; ++aa) {
                                const int lx = imod(base[3 * i] - p + 1 + aa, ng);
                                acc += wx[aa] * wy[bb] * wz[c] * Hi[((size_t)lz * ng + ly) * ng + lx];
                            }
                        }
                    }
                    F[3 * s + a] = kap * 2.0 * q[i] / (L * L) * acc;
                }
            }
        }
        free(B1r); free(B1i); free(B2r); free(B2i); free(Hi);
    }
    free(x); free(cs); free(sn); free(base); free(wgt); free(g); free(Fr); free(Fi);
    free(Gr); free(Gi);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Self energy (Eq. 16, third term) and neutralising background        */
/* ------------------------------------------------------------------ */

void orc_self_neutral(const orc_params* P, int n, const double* q, double* out)
{
    double q2 = 0.0, Q = 0.0;
    for (int i = 0; i < n; ++i) {
        q2 += q[i] * q[i];
        Q += q[i];
    }
    const double V = P->L * P->L * P->L;
    if (P->slater_k && P->beta > 0.0) {
        double I, I0;
        orc_slater_I(P, 0.0, 0, &I, &I0);   /* lim_{r->0} I(r)/r = I'(0) */
        out[0] = -0.5 * P->kappa * I0 * q2;
        out[1] = -P->kappa * Q * Q * (M_PI / (P->alpha * P->alpha) + 2.0 * M_PI / (P->beta * P->beta)) / (2.0 * V);
    } else {
        out[0] = -P->kappa * P->alpha / sqrt(M_PI) * q2;
        out[1] = -P->kappa * M_PI * Q * Q / (2.0 * V * P->alpha * P->alpha);
    }
    out[2] = 3.0 * out[1];
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 and the DPD random variable theta_ij (Eq. 5)          */
/* ------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

double orc_theta(uint64_t seed, uint64_t step, int i, int j)
{
    const uint32_t lo = (uint32_t)(i < j ? i : j), hi = (uint32_t)(i < j ? j : i);
    const uint32_t ctr[4] = {lo, hi, (uint32_t)step, (uint32_t)(step >> 32)};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    const double u = ((double)out[0] + 0.5) / 4294967296.0;
    return sqrt(3.0) * (2.0 * u - 1.0);
}

/* ------------------------------------------------------------------ */
/* DPD forces (Eq. 2-7) and harmonic bonds (Sec. 2)                    */
/* ------------------------------------------------------------------ */

int orc_dpd_forces(const orc_params* P, const orc_dpd_params* D, int n,
                   const double* pos, const double* vel, const int* type,
                   int nb, const int* bonds, uint64_t step,
                   double* F, double* E2, const int* sample, int nsample)
{
    if (n < 0 || 1.0 > 0.5 * P->L) return ORC_EINVAL;
    double* x = wrapped_positions(P, n, pos);
    if (!x) return ORC_ENOMEM;
    const double rdt = 1.0 / sqrt(D->dt);
    const int nout = sample ? nsample : n;

    #pragma omp parallel for schedule(dynamic, 64)
    for (int s = 0; s < nout; ++s) {
        const int i = sample ? sample[s] : s;
        double Fi[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3], r;
            if (!pair_within(P, &x[3 * i], &x[3 * j], 1.0, d, &r)) continue;
            const double e[3] = {d[0] / r, d[1] / r, d[2] / r};
            const double w = 1.0 - r;                                     /* w^R = w^C, Eq. 7 */
            const double aij = D->a[type[i] * D->ntypes + type[j]];
            const double vr = (vel[3 * i] - vel[3 * j]) * e[0] + (vel[3 * i + 1] - vel[3 * j + 1]) * e[1] +
                              (vel[3 * i + 2] - vel[3 * j + 2]) * e[2];
            const double fc = aij * w;                                    /* Eq. 3 */
            const double fd = -D->gamma * w * w * vr;                     /* Eq. 4 */
            const double fr = D->sigma * w * orc_theta(D->seed, step, i, j) * rdt; /* Eq. 5 */
            for (int t = 0; t < 3; ++t) Fi[t] += (fc + fd + fr) * e[t];
        }
        for (int t = 0; t < 3; ++t) F[3 * s + t] = Fi[t];
    }

    /* harmonic bonds F_i = -sum_j K (r_ij - r_eq) r_hat_ij */
    int* slot = NULL;
    if (nb > 0) {
        slot = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
        if (!slot) { free(x); return ORC_ENOMEM; }
        for (int i = 0; i < n; ++i) slot[i] = sample ? -1 : i;
        if (sample)
            for (int s = 0; s < nsample; ++s) slot[sample[s]] = s;
    }
    double Eb = 0.0;
    for (int k = 0; k < nb; ++k) {
        const int i = bonds[2 * k], j = bonds[2 * k + 1];
        double d[3];
        for (int t = 0; t < 3; ++t) {
            double dd = x[3 * i + t] - x[3 * j + t];
            if (dd > 0.5 * P->L) dd -= P->L;
            else if (dd < -0.5 * P->L) dd += P->L;
            d[t] = dd;
        }
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        Eb += 0.5 * D->K_bond * (r - D->r0_bond) * (r - D->r0_bond);
        if (r <= 0.0) continue;
        const double fm = -D->K_bond * (r - D->r0_bond) / r;
        for (int t = 0; t < 3; ++t) {
            if (slot[i] >= 0) F[3 * slot[i] + t] += fm * d[t];
            if (slot[j] >= 0) F[3 * slot[j] + t] -= fm * d[t];
        }
    }
    free(slot);

    if (E2 && !sample) {
        double Ec = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                double d[3], r;
                if (!pair_within(P, &x[3 * i], &x[3 * j], 1.0, d, &r)) continue;
                Ec += 0.5 * D->a[type[i] * D->ntypes + type[j]] * (1.0 - r) * (1.0 - r);
            }
        E2[0] = Ec;
        E2[1] = Eb;
    }
    free(x);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Table 2: total force and the modified velocity-Verlet step          */
/* ------------------------------------------------------------------ */

int orc_total_forces(const orc_params* P, const orc_dpd_params* D, int n,
                     const double* pos, const double* vel, const int* type,
                     const double* q, int nb, const int* bonds, uint64_t step,
                     double* F, double* E)
{
    double* Fr = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* Fk = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!Fr || !Fk) { free(Fr); free(Fk); return ORC_ENOMEM; }
    double E2[2] = {0.0, 0.0}, ER[2], EK[2], ES[3];
    int rc = orc_dpd_forces(P, D, n, pos, vel, type, nb, bonds, step, F, E2, NULL, 0); /* step 3 */
    if (!rc) rc = orc_real_space(P, n, pos, q, Fr, ER, NULL, 0);                  /* step 4(i) */
    if (!rc) rc = orc_recip_enuf(P, n, pos, q, Fk, EK, NULL, NULL, NULL, 0);      /* step 4(ii) */
    if (!rc) {
        orc_self_neutral(P, n, q, ES);                                             /* step 4(iii) */
        for (int i = 0; i < 3 * n; ++i) F[i] += Fr[i] + Fk[i];                    /* step 5 */
        if (E) {
            E[0] = ER[0];
            E[1] = EK[0];
            E[2] = ES[0] + ES[1];
            E[3] = ER[0] + EK[0] + ES[0] + ES[1];
            E[4] = E2[0];
            E[5] = E2[1];
        }
    }
    free(Fr);
    free(Fk);
    return rc;
}

int orc_dpd_run(const orc_params* P, const orc_dpd_params* D, int n,
                double* pos, double* vel, double* F, const int* type,
                const double* q, int nb, const int* bonds, uint64_t* step,
                int nsteps, double* E)
{
    double* v0 = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!v0) return ORC_ENOMEM;
    const double dt = D->dt, lam = D->lambda_vv;
    int rc = 0;
    for (int s = 0; s < nsteps && !rc; ++s) {
        for (int i = 0; i < 3 * n; ++i) {
            v0[i] = vel[i] + lam * F[i] * dt;   /* step 0 (m = 1) */
            vel[i] = vel[i] + 0.5 * F[i] * dt;  /* step 1 */
            pos[i] = pos[i] + vel[i] * dt;      /* step 2 */
        }
        *step += 1;
        rc = orc_total_forces(P, D, n, pos, v0, type, q, nb, bonds, *step, F, E); /* steps 3-5 */
        for (int i = 0; i < 3 * n; ++i) vel[i] = vel[i] + 0.5 * F[i] * dt;        /* step 6 */
    }
    free(v0);
    return rc;
}
