/*
 * enuf.h -- C ABI of the GB300-native ENUF-DPD hot path.
 *
 * Method: Wang, Laaksonen & Lu, "Implementation of non-uniform FFT based
 * Ewald summation in Dissipative Particle Dynamics method" (arXiv 1303.4523).
 * The library evaluates, for beads with charges q_i at positions r_i in a
 * cubic periodic box of edge L (reduced DPD units, R_c = m = k_B T = 1):
 *
 *   E = E_real + E_recip + E_self + E_neutral                       (Eq. 16)
 *   E_real  = kappa sum_{i<j, r<r_c} q_i q_j [erfc(alpha r) - (1 + beta r) e^{-2 beta r}] / r
 *             (Eq. 31 with the Slater correction of Eq. 27, applied in real space only, Sec. 5)
 *   E_recip = kappa/(2 pi L) sum_{k != 0, |k_t| <= n_c} e^{-(pi k)^2/(alpha L)^2}/k^2 |S(k)|^2
 *             with S(k) from the transposed NFFT (Eq. 14, 18-20, Table 2 step 4(ii))
 *   F_i     = -grad_i E_real + kappa (2 q_i/L^2) Im g_i,  g_i from the conjugated NFFT (Eq. 24-25)
 *   E_self  = -kappa alpha/sqrt(pi) sum q_i^2,  E_neutral = -kappa pi Q^2 / (2 V alpha^2)
 *
 * and, for DPD systems, the pair forces of Eq. 2-7, harmonic bonds (Sec. 2)
 * and the modified velocity-Verlet step of Table 2.
 *
 * Conventions for every entry point:
 *  - Functions return an enuf_status; none aborts or exits. On failure the
 *    plan's message is available from enuf_last_error().
 *  - Arrays are dense, C order. Positions/forces/velocities are [n][3].
 *    Floating arrays use double for ENUF_FP64 plans and float for ENUF_FP32
 *    plans ("real" below). Positions may lie outside [0, L); they are
 *    wrapped internally.
 *  - "device" pointers are CUDA device memory on the plan's device; "host"
 *    pointers are host memory (pinned memory makes copies faster). The caller
 *    owns every array it passes; plans and systems own their workspace.
 *  - Work is enqueued on the plan's stream. A call returns after enqueueing,
 *    except when it must return host results (energies), in which case it
 *    synchronises that stream.
 */
#ifndef ENUF_H
#define ENUF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ENUF_OK = 0,
    ENUF_ERR_INVALID = 1,     /* bad argument or parameter combination */
    ENUF_ERR_OOM = 2,         /* device allocation failed */
    ENUF_ERR_CUDA = 3,        /* a CUDA call failed (message has the CUDA error) */
    ENUF_ERR_TIMEOUT = 4,     /* a bounded device wait ran out */
    ENUF_ERR_UNSUPPORTED = 5  /* grid size / window combination not supported */
} enuf_status;

typedef enum {
    ENUF_FP64 = 0,  /* every stage in double */
    ENUF_FP32 = 1   /* spread, FFT, convolution, gather and pair forces in float;
                       influence table, self/neutral terms and all energy and
                       virial reductions (Kahan-compensated) in double */
} enuf_precision;

/* Parameters of one ENUF evaluation (Table 1; Sec. 5). */
typedef struct {
    double L;         /* cubic box edge */
    double alpha;     /* Ewald splitting parameter (Eq. 16) */
    double r_cut;     /* real-space cutoff r_c, 0 < r_c <= L/2 (Eq. 29) */
    double beta;      /* R_c / lambda_e of the Slater density (Eq. 26-27); <= 0: point charges */
    double kappa;     /* Coulomb prefactor 1/(4 pi eps0 eps_r) in reduced units */
    int    M;         /* base grid per dimension, even, >= 4; n_c = M/2 - 1.
                         0: M = 1.6 L rounded to the nearest even 2^a 3^b 5^c */
    int    p;         /* NFFT window cutoff: 2p taps per dimension, 1 <= p <= 8 */
    int    sigma_s;   /* oversampling factor; only 2 is supported (Sec. 5) */
    int    kmask;     /* 0: cubic mode set |k_t| <= n_c; 1: spherical |k| <= n_c */
    int    prec;      /* enuf_precision */
    int    tile;      /* spreading tile edge in grid points; 0 = automatic */
    int    deriv;     /* reciprocal forces: 0 = ik-differentiation, three fields
                         -i k_a D F (Eq. 24-25); 1 = gradient of the window: one
                         field h = D F and F_i = -(kappa q_i n/(pi L^2)) sum_l
                         grad Psi(n x_i - l) h(l), the exact derivative of the NFFT
                         energy (one inverse transform instead of three) */
    int    slater_k;  /* where the Slater smearing of Eq. 26-27 enters (needs beta > 0):
                         0 = the real-space pair term carries the correction
                             -(1 + beta r) e^{-2 beta r}/r (B1, B2 in real space, Sec. 5);
                         1 = the influence function carries the Slater form factor
                             (1 + k^2/(4 beta^2))^{-2} and the real-space kernel is
                             phi_S(r) - I(r)/r, I(r) = (2/pi) int rho(k) e^{-k^2/(4 alpha^2)}
                             sin(kr)/k dk, interpolated from a table built at plan time;
                             self and background terms change to match. Same total
                             energy for converged sums. */
    int    fft_path;  /* 0: automatic (FP32 grids with n <= 112: whole z-planes in shared
                         memory, x+y and y+x fused); 1: always the five line passes x, y, z, y, x */
    int    fft_radix; /* line transforms: 0 = automatic: FP32 grids whose n = f1 f2 with
                         f1, f2 in {4, 5, 6, 8, 10, 12, 16, 20} take the two-factor
                         kernels (both DFTs in registers, one twiddle pass); other grids
                         and FP64 the Stockham stages as for 2;
                         1 = Stockham stages over radices 2, 3, 4, 5, 8 only;
                         2 = Stockham stages, the fewest over 2, 3, 4, 5, 8, and for FP32
                         grids from n = 128 on the composite radices 6, 10, 12, 16, 20
                         when that saves a stage. Same result to rounding. */
    int    spread;    /* spreading kernel (FP32; FP64 always takes 1): 0 = automatic (below);
                         1 = tile form (one CTA per T^3 tile: column-stationary for
                         T in 8, 10, 12, 16, 20, 24, shared-memory atomics otherwise);
                         2 = footprint form on bricks of whole x rows (or x runs) of
                         T x T rows, one warp per z-plane, no work on zero weights;
                         3 = form 2 fused with the forward x pass (the grid is never
                         written: needs the two-factor kernels, the five-pass FFT and
                         an even T);
                         4 = scatter form: one CTA per region of T^3 (T >= 16) or 2^3
                         tiles, each bead whose window meets the region spread by a
                         warp with integer shared-memory atomics in 32-bit fixed point
                         (scale 2^k with sum over the region's beads of |q| psi(0)^3
                         below 2^30), work on its taps inside the region only (needs
                         p = 4, the region dividing n and n >= 2 (region + T + 8)).
                         Automatic (0): 4 where admitted and n >= 128, else 1.
                         Same result to rounding. */
    int    pairs;     /* DPD systems: 1 = two launches, the DPD pairs right after the
                         cell list (before the charged-bead binning is done), then the
                         real-space pairs; 2 = one launch whose blocks take either role,
                         after both cell structures exist. Automatic (0): 2 in FP32, 1 in
                         FP64 (measured at the 81000-bead polyelectrolyte, interleaved
                         steps: FP32 131.0 against 139.4 us, FP64 449.0 against 453.4 us).
                         Same result to rounding. */
} enuf_params;

typedef struct enuf_plan_s* enuf_plan_t;

/* Derived sizes of a plan. */
typedef struct {
    int    M, n, n_c;          /* base grid, oversampled grid n = sigma_s M, kept modes */
    int    tile, n_tiles;      /* spreading tile edge and tile count */
    int    n_max;              /* capacity in beads */
    int    fft_kernels;        /* FFT kernels per evaluation: 3 with the fused plane passes
                                  (see enuf_params.fft_path), else 5 */
    size_t device_bytes;       /* device memory the plan holds */
    int    fft_stages;         /* stages of one length-n line transform (2 for the
                                  two-factor kernels) */
    int    fft_radix[8];       /* their radices in order (two-factor: f1, f2) */
    int    fft_two_factor;     /* 1: the two-factor kernels (enuf_params.fft_radix) */
    int    spread;             /* spreading kernel taken (enuf_params.spread: 1 to 4) */
    int    brick_x;            /* x extent of a spreading brick (forms 2 and 3) */
    int    pairs;              /* DPD pair launches taken (enuf_params.pairs: 1 or 2) */
} enuf_plan_info;

/* Create a plan for systems of up to n_max beads with the given parameters
 * (Table 2 step 4). cuda_stream is a cudaStream_t (NULL: the plan creates
 * its own). Allocates the plan's device workspace and builds the FP64
 * influence/deconvolution table on the host. Errors: ENUF_ERR_INVALID for
 * n_max outside [0, 2^29], L <= 0, alpha <= 0, r_c outside (0, L/2], odd or too small M,
 * p outside [1, 8], sigma_s != 2, kappa not finite; ENUF_ERR_UNSUPPORTED when
 * no tile edge divides n; ENUF_ERR_OOM / ENUF_ERR_CUDA. *out is NULL on error. */
enuf_status enuf_plan(const enuf_params* params, int n_max, void* cuda_stream, enuf_plan_t* out);

/* Ewald parameters from a required accuracy delta (0 < delta < 1), by the two
 * conditions of Eq. 29: alpha is the smallest value with
 * erfc(alpha r_c) <= delta (the exact left side of the real-space condition),
 * and the base grid M = 2 (n_c + 1) with n_c >= (alpha L / pi) sqrt(-ln delta),
 * rounded up to an even 2^a 3^b 5^c integer. Reads params->L and
 * params->r_cut; writes params->alpha and params->M, leaves the rest.
 * Host only. Errors: ENUF_ERR_INVALID for delta outside (0, 1), L <= 0 or
 * r_c outside (0, L/2]; ENUF_ERR_UNSUPPORTED when the grid would exceed
 * n = 1024. */
enuf_status enuf_accuracy_params(double delta, enuf_params* params);

/* Device bytes a plan with these parameters would hold (admission control). */
enuf_status enuf_footprint(const enuf_params* params, int n_max, size_t* bytes);

enuf_status enuf_get_info(enuf_plan_t plan, enuf_plan_info* info);

/* The derived sizes a plan with these parameters would have (info as
 * enuf_get_info gives it), computed on the host: no device, no allocation.
 * Errors: those of enuf_plan's parameter validation. */
enuf_status enuf_plan_shape(const enuf_params* params, int n_max, enuf_plan_info* info);

/* Electrostatic energy and forces (Eq. 16-25; Table 2 step 4).
 *   n      : number of beads, 0 <= n <= n_max
 *   pos    : device real[n][3]
 *   q      : device real[n]; beads with q = 0 take no part
 *   F      : device real[n][3], OVERWRITTEN with F_real + F_recip (zero for q = 0)
 *   E      : host double[4] = {E_real, E_recip, E_self + E_neutral, E_total}, or NULL
 *   virial : host double[1] = -L dE/dL at fixed fractional coordinates, or NULL
 * The call runs as one CUDA graph on the plan's stream (captured on first use
 * and again whenever n or a pointer changes). With E and virial NULL it
 * returns after enqueueing. */
enuf_status enuf_energy_forces(enuf_plan_t plan, int n, const void* pos, const void* q,
                               void* F, double* E, double* virial);

/* Energies of the last evaluation (or DPD step) this plan completed, without
 * synchronising: E = host double[8] laid out as dpd_step's E (the first four
 * entries are enuf_energy_forces' E), virial may be NULL. The caller must know
 * the work has finished (e.g. an event recorded after the call has completed);
 * every evaluation copies its totals to pinned host memory as its last step;
 * DPD steps copy theirs only when asked (dpd_copy_energies, or E given). */
enuf_status enuf_last_energies(enuf_plan_t plan, double* E, double* virial);

/* Same, with HOST pos, q and F: the call copies the inputs to the device,
 * evaluates, copies F back and synchronises. */
enuf_status enuf_energy_forces_host(enuf_plan_t plan, int n, const void* pos, const void* q,
                                    void* F, double* E, double* virial);

/* Copy an internal buffer of the last evaluation to host memory (tests):
 *   ENUF_BUF_GRID  : spread grid, real[n^3], index (z*n + y)*n + x        (Eq. 14, first half)
 *   ENUF_BUF_FIELD : the conjugated-NFFT fields before the gather: real[3][n^3]
 *                    (deriv 0, Eq. 25) or the one field h, real[1][n^3] (deriv 1)
 * bytes must equal the buffer size. Synchronises the plan's stream. */
enum { ENUF_BUF_GRID = 0, ENUF_BUF_FIELD = 1 };
enuf_status enuf_debug_buffer(enuf_plan_t plan, int which, void* host, size_t bytes);

/* Kernel timing: when enabled, the next captured graph records CUDA events
 * around the kernels of the given stage; enuf_stage_time() returns the
 * device time of that stage in the last evaluation (ms). While timing is
 * on, the two branches of an evaluation or step (binning -> spreading -> FFT,
 * and the real-space / DPD pairs) run one after the other, so each stage's
 * events time its kernels alone. Stages: */
enum { ENUF_STAGE_BIN = 0,      /* charged-bead binning (3 kernels) */
       ENUF_STAGE_SPREAD = 1,   /* spreading kernel */
       ENUF_STAGE_FFT = 2,      /* the five FFT passes incl. the fused convolution */
       ENUF_STAGE_GATHER = 3,   /* gather kernel */
       ENUF_STAGE_REAL = 4,     /* real-space electrostatics kernel (in a DPD step with
                                   one pair launch, pairs = 2: that launch of both pair sums) */
       ENUF_STAGE_DPD = 5,      /* DPD pair + bond kernel (two pair launches, pairs = 1, only) */
       ENUF_STAGE_ALL = 6,      /* the whole evaluation / DPD step */
       ENUF_STAGE_CELL = 7,     /* all-bead cell list (3 kernels) */
       ENUF_NUM_STAGES = 8 };
enuf_status enuf_enable_timing(enuf_plan_t plan, int on);
enuf_status enuf_stage_time(enuf_plan_t plan, int stage, float* ms);
/* Number of kernel launches one evaluation (or one DPD step) enqueues. */
int enuf_launches_per_eval(enuf_plan_t plan);
/* Device index checks of a library built with -DENUF_CHECK (the debug
 * build): *mask receives the failure bits recorded since the last reset
 * (bit k = check site k of the kernels; 0 = every check held; always 0 in a
 * release build), after synchronising the plan's stream; reset != 0 clears
 * them. The checks record and skip nothing else: a set bit means the result
 * of that evaluation is not to be trusted. */
enuf_status enuf_check_word(enuf_plan_t plan, unsigned int* mask, int reset);
/* 1 when the library was built with the device index checks, else 0. */
int enuf_built_with_checks(void);
/* Failure injection for tests, on the host: of the library's device
 * allocations (a plan's workspace, the host-buffer staging of
 * enuf_energy_forces_host, a DPD system's state) the next `after` proceed and
 * the `count` that follow fail as if the device were out of memory, without
 * calling the allocator; the call that made one returns ENUF_ERR_OOM and
 * frees what it held. count = 0 ends the injection. Process-wide.
 * Errors: ENUF_ERR_INVALID for a negative argument. */
enuf_status enuf_debug_fail_allocs(int after, int count);

void enuf_destroy(enuf_plan_t plan);
const char* enuf_status_string(enuf_status s);
const char* enuf_last_error(enuf_plan_t plan);

/* ------------------------------------------------------------------ */
/* DPD systems (Eq. 2-7, Sec. 2 bonds, Table 2 integrator)              */
/* ------------------------------------------------------------------ */

typedef struct {
    int           ntypes;     /* number of bead types */
    const double* a;          /* host double[ntypes][ntypes] conservative amplitudes a_ij (Eq. 3) */
    double        gamma;      /* dissipation strength (Eq. 4) */
    double        sigma;      /* noise amplitude (Eq. 5), sigma^2 = 2 gamma k_B T (Eq. 6) */
    double        dt;         /* time step */
    double        lambda_vv;  /* velocity-prediction parameter (Table 2 step 0) */
    double        K_bond;     /* harmonic spring constant (Sec. 2) */
    double        r0_bond;    /* equilibrium bond length */
    uint64_t      seed;       /* key of the Philox4x32-10 stream of theta_ij (Eq. 5) */
} dpd_params;

typedef struct dpd_system_s* dpd_system_t;

/* Create a device-resident DPD system on a plan (the plan's precision and
 * box). pos, vel: HOST real[n][3]; type: host int[n] in [0, ntypes);
 * q: host real[n]; bonds: host int[n_bonds][2] (may be NULL when n_bonds = 0).
 * The system copies everything to the device, builds the per-bead bond list
 * and evaluates the initial force at step 0. Requires L >= 3 (1 + 1e-5): a
 * cell list of at least 3 cells of edge > 1 per box edge (ENUF_ERR_INVALID
 * otherwise). The plan must outlive the system. */
enuf_status dpd_create(enuf_plan_t plan, const dpd_params* params, int n, const void* pos,
                       const void* vel, const int* type, const void* q, int n_bonds,
                       const int* bonds, dpd_system_t* out);

/* Advance nsteps steps of Table 2 (steps 0-6): predict v0, half kick, drift,
 * DPD pair + bond forces (theta keyed by the new step number), electrostatics
 * (real + ENUF reciprocal), half kick. E: host double[8] or NULL =
 * {E_real, E_recip, E_self + E_neutral, E_elec, E_conservative, E_bond,
 *  E_kinetic, virial_elec} of the last step, or of the force evaluation of
 *  dpd_create / dpd_set_state when no step has run since (nsteps = 0 reads
 *  them without stepping); synchronises when non-NULL. */
enuf_status dpd_step(dpd_system_t sys, int nsteps, double* E);
/* Stream-ordered copy of the energies of the last step (or force evaluation)
 * of this system to the plan's pinned host buffer, read with
 * enuf_last_energies once the work has completed. A step keeps its energies
 * in device memory and copies them only when asked: by this call, or by
 * dpd_step / dpd_step_host with E (each of which synchronises). Not in the
 * paper (a host-interface detail). */
enuf_status dpd_copy_energies(dpd_system_t sys);

/* Checkpoint / restart: copy the state to or from HOST real[n][3] arrays
 * (any pointer may be NULL). The force F is part of the state because the
 * next step's velocity prediction (Table 2 step 0) uses it. dpd_set_state
 * with F = NULL recomputes the force of the new configuration at the given
 * step (taking v0 = vel); with F given, set_state(get_state()) resumes the
 * run exactly (the random stream is keyed by the step number). */
enuf_status dpd_get_state(dpd_system_t sys, void* pos, void* vel, void* F, uint64_t* step);
enuf_status dpd_set_state(dpd_system_t sys, const void* pos, const void* vel, const void* F, uint64_t step);
/* Current total force (HOST real[n][3]). */
enuf_status dpd_get_forces(dpd_system_t sys, void* F);
/* Host-state step: copies pos, vel, F (HOST real[n][3]; pinned memory lets the
 * copies run at full speed; a NULL array keeps the device copy) to the device,
 * advances nsteps steps (step counter unchanged by the upload), copies the new
 * pos, vel and F back into the same arrays and synchronises once. E as in
 * dpd_step (may be NULL). Equivalent to dpd_set_state(pos, vel, F, step) +
 * dpd_step + dpd_get_state with one host synchronisation instead of three. */
enuf_status dpd_step_host(dpd_system_t sys, int nsteps, void* pos, void* vel, void* F, double* E);
/* Device pointers of the resident state (real[n][3] each; owned by the system). */
enuf_status dpd_device_state(dpd_system_t sys, void** pos, void** vel, void** F);
void dpd_destroy(dpd_system_t sys);

/* ------------------------------------------------------------------ */
/* Batches: many independent systems in one captured launch sequence    */
/* ------------------------------------------------------------------ */

typedef struct enuf_batch_s* enuf_batch_t;

/* One plan per system (params[s], capacity n[s]); all systems share the
 * given stream and are evaluated by one captured CUDA graph.
 * When every system is FP32 and its plan runs the fused-plane two-factor
 * FFT, the column spreading form and the one-kernel binning offsets (the
 * defaults for grids up to n = 112 of n = f1 f2), the graph is one launch
 * sequence for all systems: each kernel of the evaluation (binning, window
 * weights, real space, spreading -- one launch per tile edge present --,
 * the three FFT passes, gather) is launched once over the concatenated grids
 * of all systems, its blocks reading their system's arguments from a device
 * table; the systems' energies go to one device array read back by one
 * copy. Otherwise the graph holds one branch per system (enuf_batch_mode).
 * The batch tables are written when the arrays change between calls
 * (after waiting for the previous evaluation). */
enuf_status enuf_batch_plan(int nsys, const enuf_params* params, const int* n, void* cuda_stream,
                            enuf_batch_t* out);
/* pos[s], q[s], F[s]: device pointers as in enuf_energy_forces, for n[s] beads.
 * E: host double[nsys][4] or NULL (synchronises when non-NULL). */
enuf_status enuf_batch_energy_forces(enuf_batch_t batch, const void* const* pos,
                                     const void* const* q, void* const* F, double* E);
/* Kernel launches in one replay of the batch graph. */
int enuf_batch_launches(enuf_batch_t batch);
/* 1: one launch sequence over all systems; 0: one graph branch per system. */
int enuf_batch_mode(enuf_batch_t batch);
void enuf_batch_destroy(enuf_batch_t batch);

/* ------------------------------------------------------------------ */
/* Allocation-free spreading                                           */
/* ------------------------------------------------------------------ */

/* The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate device memory: code running inside someone else's
 * memory pool or arena, framework hot paths where a cudaMalloc (which can
 * synchronise the whole device) is forbidden, and plugins whose GPU memory
 * budget is fixed before they run.
 *
 * It bins the charged beads and spreads them onto the oversampled grid --
 * the same result as the spread grid of enuf_energy_forces (ENUF_BUF_GRID) --
 * using no memory but the caller's arrays and one fixed scratch region that
 * belongs to the library: a 16 MiB device array in the library image, held on
 * every GPU that loads the library until the process exits.
 *   params : as for enuf_plan (precision selects float or double arrays)
 *   n      : number of beads, >= 0
 *   pos    : device real[n][3];  q: device real[n]
 *   grid   : device real[n_g^3] (n_g = sigma_s * M), OVERWRITTEN,
 *            index (z * n_g + y) * n_g + x
 *   cuda_stream : cudaStream_t to enqueue on (NULL: the legacy default stream)
 * One 16-byte word of the scratch must start at zero, the binning's arrival
 * counter: each call clears it with a memset on cuda_stream before the
 * binning (this allocates nothing); every other scratch word is written by
 * the call before it is read. Returns after enqueueing.
 * Limits and rules:
 *  - ENUF_ERR_INVALID, with a message on stderr, when the bins and sorted
 *    beads of this call need more than the 16 MiB scratch (about 200000
 *    beads in FP32 or 120000 in FP64 at the default tile), or for bad
 *    parameters. No device memory is ever allocated or freed.
 *  - The first call on a device looks up the scratch address for that device
 *    (with that device current); make that first call before any stream
 *    capture on the device.
 *  - All calls share the one scratch region: calls whose work can overlap on
 *    the GPU (different streams, or other host threads) race and corrupt each
 *    other's bins. Serialise them, e.g. on one stream. */
enuf_status enuf_spread_noalloc(const enuf_params* params, int n, const void* pos, const void* q,
                                void* grid, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
