// enuf_internal.h -- plan layout shared by the C-ABI layer and the kernel
// translation units (one per precision).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "enuf_fft.cuh"

namespace enuf {

// Geometry and constants every kernel needs, passed by value.
// Debug builds (-DENUF_CHECK): device-side index checks. ENUF_GUARD(word,
// cond, bit) is cond, and when cond fails sets bit `bit` of the plan's check
// word (read by enuf_check_word); the caller skips the access it guards.
// Release builds compile it to true.
#ifdef ENUF_CHECK
__device__ __forceinline__ bool enuf_guard(unsigned int* word, bool ok, int bit) {
    if (!ok && word != nullptr) atomicOr(word, 1u << bit);
    return ok;
}
#define ENUF_GUARD(word, cond, bit) enuf_guard((word), (cond), (bit))
#else
#define ENUF_GUARD(word, cond, bit) true
#endif

// dynamic shared memory of the binning count kernel at most (its static share
// is a few words; the part allows 227 KB per CTA)
constexpr int kBinSmem = 224 * 1024;

struct Geo {
    int n;        // oversampled grid per dimension (sigma_s * M)
    int nc;       // kept modes per side, |k_t| <= nc
    int K;        // 2 nc + 1
    int p;        // window cutoff (2p taps per dimension)
    int T;        // spreading tile edge (grid points)
    int ntd;      // tiles per dimension
    int ntiles;   // ntd^3
    int rs;       // real-space stencil radius in tiles
    int nbin;     // blocks of the charged-bead binning
    int chunk;    // beads per binning block
    int kmask;
    int nf;       // reciprocal force fields: 3 (ik-differentiation) or 1 (window gradient)
    int bin_last; // 1: the last binning block computes the tile offsets and starts
                  //    (ntiles x nbin small); 0: separate offsets and scan kernels
    double L, alpha, beta, kappa, rc;
    double b;      // Gaussian window parameter 2 sigma p / ((2 sigma - 1) pi)
    double wnorm;  // (pi b)^{-1/2}
    double ratio;  // n / L: grid coordinate u = x * ratio (one FP64 product)
    double rb;     // 1 / b
    double pref;   // kappa * 2 / L^2 (Eq. 25 prefactor); gradient mode: -kappa n / (pi L^2)
    double c2a;    // 2 alpha / sqrt(pi)
    float xmaxf;   // largest float below L: float x is inside [0, L) iff 0 <= x <= xmaxf
    float rhi, rlo;  // n/L split into two floats (compensated float grid coordinate)
    double c_self;   // -kappa alpha / sqrt(pi)           (E_self = c_self * sum q^2)
    double c_neut;   // -kappa pi / (2 V alpha^2)         (E_neutral = c_neut * Q^2)
    double c_recip;  // kappa / (2 pi L)                  (E_recip = c_recip * sum D |F|^2)
    int slater_k;    // 1: Slater form factor in k space (real-space kernel J = B1 - I)
    int kn;          // real-space kernel table intervals on [0, r_c] (0: no table)
    double kinv;     // kn / r_c
    double kh;       // r_c / kn
    const void* ktab;  // real [kn][kKtStride]: quintic coefficients of J(r) = r u(r) per interval
    int nmax;          // capacity in beads (sorted charged-bead arrays)
    unsigned int* check;  // debug builds: failure bits of the device index checks
};

// Beads of one DPD cell block plus its halo that the pair kernel stages in
// shared memory (blocks with more take the unstaged path).
constexpr int kDpdCap = 896;

// Footprint spreading on bricks (k_spread_brick): staging capacities and the
// shared memory of a brick of T x T rows of BX points (fx_bytes: the fused x
// pass's twiddles and line buffers, which reuse the staging region).
constexpr int kBrickCand = 512;    // candidates staged per round
constexpr int kBrickItems = 64;    // items per weight batch
constexpr int kBrickRanges = 18;   // contiguous runs of sorted beads around a brick
constexpr int kBrickTaps = 16;     // weight row length (2p <= 16)
template <typename R>
__host__ __device__ constexpr int brick_stage_bytes() {
    return kBrickCand * (4 + 4 + (int)sizeof(R) + 4) +
           kBrickItems * (3 * kBrickTaps * (int)sizeof(R) + 4 + (int)sizeof(R));
}
template <typename R>
__host__ __device__ constexpr int brick_smem(int T, int BX, int fx_bytes) {
    return T * T * BX * (int)sizeof(R) + (brick_stage_bytes<R>() > fx_bytes ? brick_stage_bytes<R>() : fx_bytes);
}

// Row length of the real-space kernel table (16-byte aligned rows).
constexpr int kKtStride64 = 6;   // c_0..c_5 in double
constexpr int kKtStride32 = 8;   // c_0..c_5 in float, 2 padding

// Lines per CTA of each FFT pass.
struct FftShape {
    int lx;    // complex lines (pairs of real rows) per CTA, forward x
    int ly;    // lines per CTA, forward y
    int lz;    // lines per CTA, z pass (forward + convolve + 3 inverses)
    int liy;   // lines per CTA, inverse y
    int lix;   // complex lines per CTA, inverse x
    int tx, ty, tz, tiy, tix;   // threads per CTA of each pass
    int smem_x, smem_y, smem_z, smem_iy, smem_ix;   // dynamic smem bytes
    int grid_x, grid_y_z, grid_z, grid_iy, grid_ix; // CTAs (grid_y_z: z-chunks of the y pass)
    // small grids: a whole z-plane per CTA, forward x+y and inverse y+x fused
    // (two kernels instead of four); spec2 is then plane-major [z][kx][ky]
    int fused;
    int t_xy, t_yx, smem_xy, smem_yx;
    int composite;   // the radix plan uses 6, 10, 12, 16 or 20 (FP32): the CR kernel instances
    int two;         // FP32 two-factor kernels (FftPlanDev::f1, f2), same shapes and layouts
    // spreading: 1 tile form, 2 footprint bricks into the grid, 3 bricks fused with
    // the forward x pass (the x pass kernel is then not launched), 4 scatter form
    // over regions of edge sc_E
    int spread;
    int brick_x, brick_threads, brick_smem, brick_grid, brick_lp;
    int sc_E;
};

// Device workspace of one plan (all pointers device memory, one allocation).
struct Work {
    // charged binning
    int* cnt_blk;    // [nbin] charged beads of each binning block
    int* bhist;      // [nbin][ntiles] per-block tile counts
    int* boff;       // [nbin][ntiles] offset of each block's beads within each tile
    int* ttot;       // [ntiles] beads per tile
    int* tstart;     // [ntiles + 1]
    int* ticket;     // [4] arrival counters of last-block reductions (0 between launches)
    unsigned int* check;  // [1] failure bits of the ENUF_CHECK index checks
    int* ctile;      // [nbin * chunk] tile of each compacted charged bead
    void* cpos;      // real4 [nbin * chunk] wrapped x, y, z, q of each compacted charged bead
    void* cfrac;     // real4 [nbin * chunk] fractional grid coordinates, original index bits
    int* cbase;      // [nbin * chunk] packed base grid index
    void* sq;        // real4 [n_max]  wrapped x, y, z, q (sorted)
    void* sw;        // real4 [n_max]  fractional grid coordinates, original index bits
    int* sb;         // [n_max]  packed base grid index
    void* wb;        // real [n_max][3][2p]  window weights psi(u - l) of each sorted bead
    // grids and spectra
    void* grid;      // real [n^3]
    void* spec1;     // cplx [n][nc+1][n]      after forward x   ([z][kx][y])
    void* spec2;     // cplx [nc+1][K][n]      after forward y   ([kx][ky][z])
    void* spec3;     // cplx [3][n][nc+1][K]   after z pass      ([a][z][kx][ky])
    void* spec4;     // cplx [3][n][n][nc+1]   after inverse y   ([a][z][y][kx])
    void* h;         // real [3][n^3]          conjugated-NFFT fields
    double* tab;     // [nc+1][K][K] influence/deconvolution table D(k) (0 outside the mode set)
    double* tabv;    // [nc+1][K][K] D(k) times the virial weight 1 - 2 pi^2 k^2/(alpha L)^2
    void* tabr;      // real copy of tab
    void* tw;        // cplx [n] twiddles e^{-2 pi i t/n}
    void* ktab;      // real [kn][kKtStride] real-space kernel table (FP64, or slater_k = 1)
    double* part;    // per-block partial sums
    double* Edev;    // [16] reduced totals
    // partial-sum segments (offsets into part, in doubles)
    int off_q, off_real, off_recip, off_dpd, off_kin;
    int nblk_real, nblk_conv, nblk_dpd, nblk_kin, nblk_gather;
    int off_pre;   // 8 doubles: the step's quantities 0-7 reduced beside the gather
};

// Arguments of one electrostatics evaluation.
struct EvalArgs {
    int N;
    const void* pos;   // real [N][3] (device)
    const void* q;     // real [N]
    void* F;           // real [N][3]
    bool zeroF;        // overwrite F (pure electrostatics) vs add into it (DPD step)
};

// Where the final FP64 totals read their per-block partials (offsets into
// Work::part, counts) and write Edev; ticket is the arrival counter of the
// kernel whose last block reduces them. Edev == nullptr: no totals.
struct TotalsArgs {
    const double* part;
    int off_q, nq, off_real, nreal, off_recip, nrecip, off_dpd, ndpd, off_kin, nkin;
    double* Edev;
    int* ticket;
    // pre (or nullptr): quantities 0-7 already reduced (k_totals_pre); the
    // closing totals then reduce the kinetic partials only
    double* pre;
};

// DPD device state and cell list (one per system).
struct DpdDev {
    unsigned int* check;   // the plan's check word (debug builds)
    int N, ntypes, ncd, ncells;
    int B;             // cells per block edge of the DPD kernel (<= 4, B + 2 <= ncd)
    double L, gamma, sigma, dt, lambda_vv, K_bond, r0_bond;
    double rdt;    // 1 / sqrt(dt)
    double cinv;   // ncd / L
    float xmaxf;   // largest float below L
    uint64_t seed;
    // Philox4x32-10 round keys of the seed (key bumped by the Weyl constants
    // each round), formed on the host: the kernel's rounds read them as
    // launch constants
    uint32_t rk0[10], rk1[10];
    void* pos; void* vel; void* v0; void* F; void* q;   // real
    int* type;
    void* atab;        // real [ntypes^2]
    int nbonds;
    int* bnd;                // bond pairs [nbonds][2]
    int* ckey; int* ccount; int* cstart; int* ccur;
    void* sp; void* sv;      // real4 [N] sorted: (x, y, z, orig) and (v0, type)
    uint64_t* step_dev;      // device copy of the step counter
};

constexpr int kStageCount = 8;

// Host-side record of the launches one enqueue made (for the launch count).
struct LaunchLog {
    int kernels = 0;
};

struct Events {
    cudaEvent_t start[kStageCount];
    cudaEvent_t stop[kStageCount];
    bool on = false;
};

// One system of a batched launch sequence (FP32): its plan's geometry,
// shapes, workspace and this evaluation's arrays; Edev receives its totals.
struct BatchSys {
    Geo g;
    FftShape fs;
    FftPlanDev fp;
    Work w;
    int N;
    const void* pos;
    const void* q;
    void* F;
    double* Edev;
};

// Launch parameters of one batched kernel: its argument table and block map
// (device), the blocks of all systems together, threads and shared memory
// (the largest any system needs).
struct BatchKernel {
    void* tab = nullptr;
    int* cmap = nullptr;
    int blocks = 0, threads = 0, smem = 0;
    int T = 0;   // spreading: the tile edge of this group; gather: the common tap count 2p (0: mixed)
};
struct BatchLaunch {
    BatchKernel bin_count, bin_scatter, bin_weights, real, fft_xy, fft_z, fft_yx, gather;
    BatchKernel spread[6];   // one per tile edge present (8, 10, 12, 16, 20, 24)
    int nspread = 0;
};

template <typename R> cudaError_t configure_kernels(int max_smem);
template <typename R> int spread_smem(const Geo& g);
// dpd (a DPD step with fused pair kernels, or nullptr): the real-space launch
// also runs the DPD pair forces (k_pairs), which enqueue_dpd_forces then leaves out.
// evZ, evT (DPD steps, or nullptr): after the FFT the side stream reduces the
// step's energies other than the kinetic one (k_totals_pre, beside the
// gather) and records evT, on which the closing half kick must wait.
template <typename R>
cudaError_t enqueue_enuf(const Geo& g, const FftShape& fs, const FftPlanDev& fp, const Work& w,
                         const EvalArgs& a, cudaStream_t s0, cudaStream_t s1, cudaEvent_t evFork,
                         cudaEvent_t evJoin, Events* ev, LaunchLog* log, bool fuse_totals,
                         const DpdDev* dpd = nullptr, cudaEvent_t evZ = nullptr, cudaEvent_t evT = nullptr);
template <typename R>
cudaError_t enqueue_totals(const Geo& g, const Work& w, bool dpd, cudaStream_t s, LaunchLog* log, bool pdl);
template <typename R>
cudaError_t enqueue_dpd_forces(const Work& w, const DpdDev& d, cudaStream_t s, Events* ev, LaunchLog* log,
                               bool pair_kernel = true);
template <typename R>
cudaError_t enqueue_vv_pre(const DpdDev& d, cudaStream_t s, LaunchLog* log);
template <typename R>
cudaError_t enqueue_vv_post(const Geo& g, const Work& w, const DpdDev& d, cudaStream_t s, LaunchLog* log, bool pdl,
                            bool pre = false);
template <typename R>
cudaError_t enqueue_spread_only(const Geo& g, const Work& w, const EvalArgs& a, void* grid_out, cudaStream_t s);
// Batched launch sequence (FP32): a system qualifies when its plan runs the
// fused-plane two-factor FFT, the column spreading form and the one-kernel
// binning offsets. batch_bytes: the device tables' size; batch_build writes
// them (argument tables and block maps) into dbuf and fills the launch
// parameters; batch_enqueue launches the sequence (fork/join on s1 for the
// real-space pairs).
bool batch_eligible(const BatchSys& s);
template <typename R> size_t batch_bytes(const BatchSys* sys, int nsys);
template <typename R>
cudaError_t batch_build(void* dbuf, const BatchSys* sys, int nsys, BatchLaunch* out);
template <typename R>
cudaError_t batch_enqueue(const BatchLaunch& L, cudaStream_t s0, cudaStream_t s1, cudaEvent_t evFork, cudaEvent_t evJoin,
                          LaunchLog* log);

}  // namespace enuf
