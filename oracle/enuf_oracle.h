/*
 * enuf_oracle.h -- plain, slow, FP64 CPU oracle for the ENUF-DPD hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library. It shares no code,
 * header, table or helper with the CUDA path in paper_1303_4523_gb300/.
 *
 * Reference: Wang, Laaksonen & Lu, "Implementation of non-uniform FFT based
 * Ewald summation in Dissipative Particle Dynamics method" (arXiv 1303.4523).
 * Every function names the equation, table or section it follows.
 *
 * Units are reduced DPD units (R_c = m = k_B T = 1, Sec. 2). Positions are
 * cartesian in a cubic periodic box of edge L; they may lie outside [0, L)
 * and are wrapped with orc_wrap().
 *
 * Readings of points the paper leaves open:
 *  - Slater smearing enters the real-space pair sum only, as the exact
 *    correction -(1+beta r) e^{-2 beta r}/r to the erfc term (Sec. 5 applies
 *    the corrections B1 and B2 to the real-space part alone); reciprocal
 *    space is the plain Ewald sum (Eq. 18).
 *  - The garbled real-space force (Eq. 32) is taken as the exact gradient
 *    of Eq. 31.
 *  - The NFFT window (Sec. 4 names only its Gaussian kind) is the Gaussian
 *    psi(u) = (pi b)^{-1/2} exp(-u^2/b), u in grid units, with
 *    b = 2 sigma p / ((2 sigma - 1) pi), truncated to 2p taps per dimension.
 *  - The mode set I_M (Eq. 9) is taken symmetric, |k_t| <= n_c = M/2 - 1.
 *  - theta_ij (Eq. 5) is uniform on [-sqrt3, sqrt3], drawn from
 *    Philox4x32-10 (Salmon et al., SC'11) keyed by (seed) with counter
 *    (min(i,j), max(i,j), step_lo, step_hi).
 */
#ifndef ENUF_ORACLE_H
#define ENUF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double L;       /* cubic box edge */
    double alpha;   /* Ewald splitting parameter (Eq. 16) */
    double r_cut;   /* real-space cutoff r_c (Eq. 29), must be <= L/2 */
    double beta;    /* R_c / lambda_e (Eq. 27); <= 0 means point charges */
    double kappa;   /* Coulomb prefactor 1/(4 pi eps0 eps_r) in reduced units */
    int    M;       /* base grid per dimension (even); n_c = M/2 - 1 */
    int    p;       /* NFFT window cutoff: 2p taps per dimension */
    int    sigma_s; /* oversampling factor; grid n = sigma_s * M */
    int    kmask;   /* 0: cubic |k_t| <= n_c; 1: spherical |k| <= n_c */
    int    deriv;   /* ENUF forces: 0 = ik-differentiation (Eq. 24-25); 1 = analytic
                       gradient of the window (one real field, see orc_recip_enuf) */
    int    slater_k;/* where the Slater smearing enters (Eq. 26-28):
                       0 = real space only, the correction -(1+beta r)e^{-2 beta r}/r
                           on the erfc pair term (Sec. 5: B1, B2 applied in real space);
                       1 = k space: the influence times the Slater form factor
                           rho(k) = (1 + k^2/(4 beta^2))^{-2} (k = 2 pi |m|/L), the real
                           space pair kernel phi_S(r) - I(r)/r with
                           I(r) = (2/pi) int_0^inf rho(k) e^{-k^2/(4 alpha^2)} sin(kr)/k dk,
                           self term -(kappa/2) lim I(r)/r sum q^2 and background term
                           -kappa Q^2 (pi/alpha^2 + 2 pi/beta^2)/(2V). Needs beta > 0.
                       Both give the same total energy for untruncated sums. */
} orc_params;

/* The radial integral of the k-space Slater kernel and its r-derivative,
 *   I(r)  = (2/pi) int_0^inf w(k) e^{-k^2/(4 alpha^2)} sin(k r)/k dk,
 *   I'(r) = (2/pi) int_0^inf w(k) e^{-k^2/(4 alpha^2)} cos(k r) dk,
 * w(k) = (1 + k^2/(4 beta^2))^{-2}, or w = 1 when rho_one (then I = erf(alpha r)),
 * by composite Gauss-Legendre quadrature; r = 0 gives I'(0) = lim I(r)/r. */
void orc_slater_I(const orc_params* P, double r, int rho_one, double* I, double* dI);

/* Position wrapping into [0, L): identity inside, else x - L floor(x/L). */
double orc_wrap(double x, double L);

/* Slater correction factors of Eq. 27/28 (Fig. 2) and the Slater pair
 * energy/force kernels. beta <= 0 returns the point-charge limit. */
double orc_B1(double beta, double r);
double orc_B2(double beta, double r);
double orc_slater_energy(double beta, double r);   /* B1 / r      (Eq. 27) */
double orc_slater_force(double beta, double r);    /* B2 / r^2    (Eq. 28) */

/* Real-space Ewald sum with Slater correction (Eq. 31, Eq. 27-28).
 * F (n x 3, overwritten; may be NULL), EW[0] = energy, EW[1] = virial.
 * If sample != NULL only the nsample listed beads get forces (row s of F is
 * bead sample[s]); EW always covers the whole system. Returns 0 or a
 * negative error code. */
int orc_real_space(const orc_params* P, int n, const double* pos, const double* q,
                   double* F, double* EW, const int* sample, int nsample);

/* Reciprocal Ewald sum by an explicit loop over integer k (Eq. 18-19,
 * Eq. 22-24). Same outputs as orc_real_space. */
int orc_recip_direct(const orc_params* P, int n, const double* pos, const double* q,
                     double* F, double* EW, const int* sample, int nsample);

/* Reciprocal sum by the naive ENUF: transposed NFFT -> energy -> g_n ->
 * conjugated NFFT (Table 2 step 4(ii); Eq. 14, 19-20, 24-25), with plain
 * window loops and plain per-dimension DFTs.
 * Optional intermediate outputs (NULL to skip):
 *   grid   : n_g^3 spread grid, index (lz*n_g + ly)*n_g + lx      (n_g = sigma_s*M)
 *   hfield : 3 x n_g^3, Im of the conjugated-NFFT field of g_n/c for a = x,y,z
 *            (deriv = 1: n_g^3, the real field h below)
 * deriv = 1 replaces Eq. 24-25 by the exact gradient of the NFFT energy:
 * with h(l) = sum_k f(k) S(k)/c(k) e^{2 pi i k.l/n} (real) and d = n x_i - l,
 *   F_{i,a} = -(kappa q_i n / (pi L^2)) sum_l psi'(d_a) prod_{t!=a} psi(d_t) h(l),
 *   psi'(d) = -(2 d / b) psi(d)
 * (derivation: differentiate kappa/(2 pi L) sum_k f |Fhat/c|^2 through the
 * spread of Eq. 14; one inverse transform instead of three).
 * F/EW/sample as in orc_real_space. */
int orc_recip_enuf(const orc_params* P, int n, const double* pos, const double* q,
                   double* F, double* EW, double* grid, double* hfield,
                   const int* sample, int nsample);

/* Self energy and neutralising-background term (Eq. 16 third term; the
 * background term is the standard one for a net charge Q). out[0] = E_self,
 * out[1] = E_neutral, out[2] = virial of the background term (3 E_neutral). */
void orc_self_neutral(const orc_params* P, int n, const double* q, double* out);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* theta_ij of Eq. 5: uniform on [-sqrt3, sqrt3], symmetric in (i, j). */
double orc_theta(uint64_t seed, uint64_t step, int i, int j);

typedef struct {
    int    ntypes;
    const double* a;   /* ntypes x ntypes conservative amplitudes a_ij (Eq. 3) */
    double gamma;      /* dissipation strength (Eq. 4) */
    double sigma;      /* noise amplitude (Eq. 5); sigma^2 = 2 gamma kT (Eq. 6) */
    double dt;         /* time step */
    double lambda_vv;  /* velocity prediction parameter (Table 2 step 0) */
    double K_bond;     /* harmonic spring constant (Sec. 2) */
    double r0_bond;    /* equilibrium bond length */
    uint64_t seed;
} orc_dpd_params;

/* DPD pair forces F^C + F^D + F^R/sqrt(dt) (Eq. 2-7, R_c = 1) on every bead
 * (or the sampled ones), using velocities vel for F^D. Also adds harmonic
 * bond forces (Sec. 2) when nb > 0. E2 (may be NULL): [0] conservative
 * energy sum_{i<j} a_ij (1-r)^2/2, [1] bond energy. */
int orc_dpd_forces(const orc_params* P, const orc_dpd_params* D, int n,
                   const double* pos, const double* vel, const int* type,
                   int nb, const int* bonds, uint64_t step,
                   double* F, double* E2, const int* sample, int nsample);

/* Full ENUF-DPD force: DPD pairs + bonds + electrostatics (real + naive ENUF
 * reciprocal), Table 2 steps 3-5. E (may be NULL) receives
 * [E_real, E_recip, E_self+E_neutral, E_elec_total, E_conservative, E_bond]. */
int orc_total_forces(const orc_params* P, const orc_dpd_params* D, int n,
                     const double* pos, const double* vel, const int* type,
                     const double* q, int nb, const int* bonds, uint64_t step,
                     double* F, double* E);

/* nsteps of the modified velocity-Verlet scheme of Table 2 (steps 0-6).
 * pos, vel, F are updated in place; F must hold the force of the current
 * configuration on entry (as computed by orc_total_forces with the current
 * vel); *step is advanced by nsteps. */
int orc_dpd_run(const orc_params* P, const orc_dpd_params* D, int n,
                double* pos, double* vel, double* F, const int* type,
                const double* q, int nb, const int* bonds, uint64_t* step,
                int nsteps, double* E);

#ifdef __cplusplus
}
#endif
#endif
