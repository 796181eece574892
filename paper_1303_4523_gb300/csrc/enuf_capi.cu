// enuf_capi.cu -- host side of the C ABI declared in include/enuf.h: plan
// construction (grid sizes, FP64 influence/deconvolution table, workspace),
// CUDA-graph capture of one evaluation / one DPD step, DPD systems and batches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "enuf.h"
#include "enuf_internal.h"

using namespace enuf;

namespace {

constexpr int kMaxTiles = 32768;      // shared-memory histogram limit (128 KB)
constexpr int kMaxBeads = 1 << 29;    // the kernels index per-bead components as int (3 i + 2, 4 i + 3)
constexpr int kMaxSmem = 200 * 1024;  // dynamic shared memory the kernels may request
constexpr int kSMs = 152;

// Kernel attributes (dynamic shared-memory opt-in) belong to the device that
// was current when they were set: configured once per device and precision.
constexpr int kMaxDevices = 64;
std::mutex g_config_mu;
bool g_configured[kMaxDevices][2] = {};

// Configure the kernels of one precision on the current device (once).
cudaError_t ensure_configured(int prec) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const int pi = prec == ENUF_FP32 ? 0 : 1;
    std::lock_guard<std::mutex> lock(g_config_mu);
    if (g_configured[dev][pi]) return cudaSuccess;
    e = prec == ENUF_FP32 ? configure_kernels<float>(kMaxSmem) : configure_kernels<double>(kMaxSmem);
    if (e == cudaSuccess) g_configured[dev][pi] = true;
    return e;
}

// Failure injection on the host (enuf_debug_fail_allocs): after g_fail_after
// more device allocations of plans, host-buffer staging and DPD systems, the
// next g_fail_count report cudaErrorMemoryAllocation without calling
// cudaMalloc, so the out-of-memory paths run without exhausting the device.
std::mutex g_fail_mu;
int g_fail_after = 0, g_fail_count = 0;

cudaError_t dev_alloc(void** p, size_t bytes) {
    bool inject = false;
    {
        std::lock_guard<std::mutex> lock(g_fail_mu);
        if (g_fail_count > 0) {
            if (g_fail_after > 0) {
                --g_fail_after;
            } else {
                --g_fail_count;
                inject = true;
            }
        }
    }
    if (inject) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool smooth(int m) {
    if (m <= 0) return false;
    for (int f : {2, 3, 5})
        while (m % f == 0) m /= f;
    return m == 1;
}

// M = 1.6 L rounded to the nearest even 2^a 3^b 5^c integer (ties to the smaller).
int grid_rule(double L) {
    const double target = 1.6 * L;
    int best = -1;
    for (int m = 2; m < (int)(4 * target) + 8; m += 2) {
        if (!smooth(m)) continue;
        if (best < 0 || std::fabs(m - target) < std::fabs(best - target) - 1e-12) best = m;
    }
    return std::max(best, 8);
}

// The fewest Stockham stages of length n over a radix set; ties go to the
// earlier radix of the list. 0 stages: not factorable.
std::vector<int> radix_plan(int n, bool composite) {
    static const int kRad[] = {20, 16, 12, 10, 8, 6, 5, 4, 3, 2};
    std::vector<int> best(n + 1, 1 << 20), pick(n + 1, 0), out;
    best[1] = 0;
    for (int m = 2; m <= n; ++m) {
        if (n % m) continue;   // only divisors of n occur
        for (int r : kRad)
            if ((composite || (r <= 8 && r != 6)) && m % r == 0 && best[m / r] + 1 < best[m]) {
                best[m] = best[m / r] + 1;
                pick[m] = r;
            }
    }
    if (best[n] >= (1 << 20)) return out;
    for (int m = n; m > 1; m /= pick[m]) out.push_back(pick[m]);
    return out;
}

// Radices 2, 3, 4, 5, 8; in float (the composite radices 6, 10, 12, 16, 20 of
// the float kernels) the composite plan when it saves a stage and n >= 128.
// Every stage is one pass over the lines in shared memory with its index
// arithmetic, whatever its radix, but a large radix leaves n/r butterflies
// per line: measured, two-stage plans were slower below n = 128 (too few
// butterflies to fill a CTA) and 3-8% faster from n = 128 to 320.
bool fft_radices(int n, FftPlanDev& fp, bool composite) {
    fp.n = n;
    fp.nst = 0;
    if (n < 2) return false;
    std::vector<int> plan = radix_plan(n, false);
    if (composite && n >= 128) {
        const std::vector<int> alt = radix_plan(n, true);
        if (!alt.empty() && (plan.empty() || alt.size() < plan.size())) plan = alt;
    }
    if (plan.empty() || plan.size() > 8) return false;
    for (int r : plan) fp.rad[fp.nst++] = r;
    return true;
}

// Two-factor split n = f1 f2 of the FP32 two-factor kernels: both factors in
// their radix set; the most balanced split, ties to the larger f2 (phase A
// reads f2 consecutive elements per line and load). False: none.
bool fft_two_factor(int n, FftPlanDev& fp) {
    static const int kF[] = {4, 5, 6, 8, 10, 12, 16, 20};
    int best1 = 0, best2 = 0;
    for (int a : kF)
        for (int b : kF)
            if (a * b == n) {
                const int m = std::min(a, b), mb = std::min(best1, best2);
                if (!best1 || m > mb || (m == mb && b > best2)) {
                    best1 = a;
                    best2 = b;
                }
            }
    fp.f1 = best1;
    fp.f2 = best2;
    return best1 > 0;
}

// Largest float strictly below L: a float x lies in [0, L) iff 0 <= x <= this.
float largest_float_below(double L) {
    float f = (float)L;
    while ((double)f >= L) f = std::nextafter(f, 0.0f);
    return f;
}

int lines_for(int n, int nbuf, int esz, int budget, int cap) {
    const int l = (budget - n * esz) / (nbuf * n * esz);
    return std::max(1, std::min(cap, l));
}

}  // namespace

struct enuf_plan_s {
    enuf_params P{};
    int n_max = 0;
    int prec = ENUF_FP64;
    size_t rsz = 8;  // bytes of one real
    cudaStream_t stream = nullptr, aux = nullptr;
    bool own_stream = false;
    cudaEvent_t evFork = nullptr, evJoin = nullptr, evA = nullptr;
    cudaEvent_t evZ = nullptr, evT = nullptr;   // DPD steps: the side stream's energy totals
    Geo g{};
    FftShape fs{};
    FftPlanDev fp{};
    Work w{};
    void* dmem = nullptr;
    size_t dbytes = 0;
    double* hE = nullptr;  // pinned [16]
    cudaGraphExec_t gexec = nullptr;
    int g_n = -1;
    const void* g_pos = nullptr;
    const void* g_q = nullptr;
    void* g_F = nullptr;
    bool g_timing = false;
    Events ev{};
    int launches = 0;
    void* stage = nullptr;  // device staging for the host-buffer entry point
    char err[512] = {0};
};

namespace {

enuf_status fail(enuf_plan_t p, enuf_status s, const char* fmt, ...) {
    if (p) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(p->err, sizeof(p->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CU(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(plan, ENUF_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                                \
    } while (0)

// Derive every size of a plan; no allocation. Returns the device bytes.
// Radial integrals of the k-space Slater kernel (form factor rho(k) = (1 + k^2/(4 beta^2))^{-2}
// times the Ewald Gaussian e^{-k^2/(4 alpha^2)}), FP64 on the host:
//   out[0] = I(r)   = (2/pi) int_0^inf rho e^{..} sin(kr)/k dk
//   out[1] = I'(r)  = (2/pi) int_0^inf rho e^{..} cos(kr) dk          (r = 0: lim I(r)/r)
//   out[2] = I''(r) = -(2/pi) int_0^inf rho e^{..} k sin(kr) dk
// Composite 16-point Gauss-Legendre over [0, 2 alpha sqrt(50)] (the Gaussian is below
// 1e-21 beyond), 192 panels; the nodes come from Newton's method on P_16.
struct GaussLegendre16 {
    double x[16], w[16];
    GaussLegendre16() {
        for (int i = 0; i < 16; ++i) {
            double z = std::cos(M_PI * (i + 0.75) / 16.5), dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int k = 2; k <= 16; ++k) {
                    const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = 16.0 * (z * p1 - p0) / (z * z - 1.0);
                const double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

void slater_kernel(double alpha, double beta, double r, double* out) {
    static const GaussLegendre16 gl;   // thread-safe one-time setup
    const double* gx = gl.x;
    const double* gw = gl.w;
    const double kmax = 2.0 * alpha * std::sqrt(50.0);
    const int npan = 192;
    const double h = kmax / npan;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int pnl = 0; pnl < npan; ++pnl)
        for (int t = 0; t < 16; ++t) {
            const double k = (pnl + 0.5 * (gx[t] + 1.0)) * h;
            const double c = 1.0 + k * k / (4.0 * beta * beta);
            const double wk = 0.5 * h * gw[t] * std::exp(-k * k / (4.0 * alpha * alpha)) / (c * c);
            const double sn = std::sin(k * r), cs = std::cos(k * r);
            s0 += wk * sn / k;
            s1 += wk * cs;
            s2 -= wk * k * sn;
        }
    out[0] = 2.0 / M_PI * s0;
    out[1] = 2.0 / M_PI * s1;
    out[2] = 2.0 / M_PI * s2;
}

enuf_status derive(enuf_plan_t plan, const enuf_params& P, int n_max, size_t* bytes) {
    if (n_max < 0 || n_max > kMaxBeads) return fail(plan, ENUF_ERR_INVALID, "n_max = %d outside [0, 2^29]", n_max);
    if (!(P.L > 0) || !std::isfinite(P.L)) return fail(plan, ENUF_ERR_INVALID, "L must be > 0");
    if (!(P.alpha > 0) || !std::isfinite(P.alpha)) return fail(plan, ENUF_ERR_INVALID, "alpha must be > 0");
    if (!(P.r_cut > 0) || P.r_cut > 0.5 * P.L) return fail(plan, ENUF_ERR_INVALID, "r_cut must be in (0, L/2]");
    if (!std::isfinite(P.kappa) || !std::isfinite(P.beta)) return fail(plan, ENUF_ERR_INVALID, "kappa/beta not finite");
    if (P.sigma_s != 2) return fail(plan, ENUF_ERR_INVALID, "only sigma_s = 2 is supported");
    if (P.p < 1 || P.p > 8) return fail(plan, ENUF_ERR_INVALID, "p must be in [1, 8]");
    if (P.prec != ENUF_FP64 && P.prec != ENUF_FP32) return fail(plan, ENUF_ERR_INVALID, "bad precision");
    if (P.kmask != 0 && P.kmask != 1) return fail(plan, ENUF_ERR_INVALID, "kmask must be 0 or 1");
    if (P.deriv != 0 && P.deriv != 1) return fail(plan, ENUF_ERR_INVALID, "deriv must be 0 or 1");
    if (P.slater_k != 0 && P.slater_k != 1) return fail(plan, ENUF_ERR_INVALID, "slater_k must be 0 or 1");
    if (P.slater_k && !(P.beta > 0)) return fail(plan, ENUF_ERR_INVALID, "slater_k = 1 needs beta > 0");
    if (P.fft_path != 0 && P.fft_path != 1) return fail(plan, ENUF_ERR_INVALID, "fft_path must be 0 or 1");
    if (P.fft_radix < 0 || P.fft_radix > 2) return fail(plan, ENUF_ERR_INVALID, "fft_radix must be 0, 1 or 2");
    const int M = P.M == 0 ? grid_rule(P.L) : P.M;
    if (M < 4 || (M & 1)) return fail(plan, ENUF_ERR_INVALID, "M must be even and >= 4 (got %d)", M);
    const int n = P.sigma_s * M;
    if (n > 1024) return fail(plan, ENUF_ERR_UNSUPPORTED, "grid n = %d > 1024", n);
    FftPlanDev fp{};
    if (!fft_radices(n, fp, P.prec == ENUF_FP32 && P.fft_radix != 1))
        return fail(plan, ENUF_ERR_UNSUPPORTED, "grid n = %d is not 2^a 3^b 5^c", n);
    fp.f1 = fp.f2 = 0;
    if (P.prec == ENUF_FP32 && P.fft_radix == 0) fft_two_factor(n, fp);
    if (2 * P.p > n) return fail(plan, ENUF_ERR_INVALID, "window 2p = %d wider than the grid", 2 * P.p);
    // tile edge: divides n, >= p, histogram fits in shared memory
    // the spreading kernel holds a T^3 tile of the grid in shared memory: T <= 24
    // (110 KB in FP64); the binning kernels hold the tile histogram (<= 32768 tiles)
    constexpr int kMaxTile = 24;
    int T = 0;
    if (P.tile > 0) {
        T = P.tile;
        if (n % T || T < P.p || (n / T) * (n / T) * (n / T) > kMaxTiles || T > kMaxTile)
            return fail(plan, ENUF_ERR_INVALID, "tile %d does not divide n = %d, is < p, or outside [p, %d]", T, n,
                        kMaxTile);
    } else {
        // default: the smallest tile at least r_c wide (the real-space stencil is
        // then 3^3 tiles) that divides n, is >= p and keeps the histogram in shared memory
        const int tmin = std::max(P.p, (int)std::ceil(P.r_cut * n / P.L - 1e-9));
        for (int c = tmin; c <= kMaxTile && !T; ++c)
            if (n % c == 0 && (n / c) * (n / c) * (n / c) <= kMaxTiles) T = c;
        for (int c = std::max(P.p, 8); c <= kMaxTile && !T; ++c)
            if (n % c == 0 && (n / c) * (n / c) * (n / c) <= kMaxTiles) T = c;
        for (int c = P.p; c < 8 && !T; ++c)
            if (n % c == 0 && (n / c) * (n / c) * (n / c) <= kMaxTiles) T = c;
        if (!T) return fail(plan, ENUF_ERR_UNSUPPORTED, "no tile edge for n = %d, p = %d", n, P.p);
    }
    const int esz = P.prec == ENUF_FP32 ? 4 : 8;
    const int csz = 2 * esz;
    Geo g{};
    g.n = n;
    g.nc = M / 2 - 1;
    g.K = 2 * g.nc + 1;
    g.p = P.p;
    g.T = T;
    g.ntd = n / T;
    g.ntiles = g.ntd * g.ntd * g.ntd;
    const double tw = T * P.L / n;
    g.rs = (int)std::ceil(P.r_cut / tw - 1e-12);
    {   // the real-space kernel stages the stencil of one tile: at most 1024 tiles
        const int hs = std::min(2 * g.rs + 1, n / T);
        if (hs * hs * hs > 1024)
            return fail(plan, ENUF_ERR_UNSUPPORTED, "real-space stencil of %d^3 tiles too large (r_cut/tile)", hs);
    }
    // binning blocks: the count kernel holds a chunk-sized list plus the tile
    // histogram in shared memory (<= kBinSmem), one block per SM: chunks of at
    // least 2048 beads, as few whole waves of kSMs blocks as the list allows
    // (a partial second wave doubled the kernel's time at 3M beads)
    {
        const int room = kBinSmem / 4 - g.ntiles;   // list entries that fit beside the histogram
        int waves = 1;
        // chunks are whole groups of 32 beads (the count kernel deals groups to its blocks)
        auto chunk_for = [&](int w) { return std::max(2048, ((n_max + w * kSMs - 1) / (w * kSMs) + 31) & ~31); };
        g.chunk = chunk_for(1);
        while (g.chunk > room && g.chunk > 2048) g.chunk = chunk_for(++waves);
    }
    g.nbin = std::max(1, (n_max + g.chunk - 1) / g.chunk);
    // the last binning block walks ntiles x nbin counts: only when that is small
    g.bin_last = (long long)g.ntiles * g.nbin <= 65536 ? 1 : 0;
    g.kmask = P.kmask;
    g.nf = P.deriv ? 1 : 3;
    g.L = P.L;
    g.alpha = P.alpha;
    g.beta = P.beta;
    g.kappa = P.kappa;
    g.rc = P.r_cut;
    g.b = 2.0 * P.sigma_s * P.p / ((2.0 * P.sigma_s - 1.0) * M_PI);
    g.wnorm = 1.0 / std::sqrt(M_PI * g.b);

    // FFT passes: enough lines per CTA to keep ~2 CTAs per SM busy, within a
    // 64 KB shared-memory budget; threads ~ one butterfly of radix 4 per line point
    FftShape fs{};
    const int budget = 64 * 1024;
    const int nc1 = g.nc + 1;
    auto shape = [&](int total_lines, int nbuf, int& lines, int& threads, int& grid, int bud = 0) {
        const int cap = lines_for(n, nbuf, csz, bud > 0 ? bud : budget, 64);
        lines = std::max(1, std::min(cap, (total_lines + 2 * kSMs - 1) / (2 * kSMs)));
        grid = (total_lines + lines - 1) / lines;
        threads = std::min(256, std::max(64, ((lines * n / 4 + 31) / 32) * 32));
    };
    int gyz = 0;
    shape(n * n / 2, 2, fs.lx, fs.tx, fs.grid_x);
    shape(n * nc1, 2, fs.ly, fs.ty, gyz);
    fs.grid_y_z = (n + fs.ly - 1) / fs.ly;
    // z pass: forward lines (2 buffers) and the nf fields transformed together (2 nf)
    shape(nc1 * g.K, 2 + 2 * g.nf, fs.lz, fs.tz, fs.grid_z, 96 * 1024);
    fs.tz = std::min(256, std::max(fs.tz, ((g.nf * fs.lz * n / 4 + 31) / 32) * 32));
    shape(g.nf * n * nc1, 2, fs.liy, fs.tiy, fs.grid_iy);
    shape(g.nf * n * n / 2, 2, fs.lix, fs.tix, fs.grid_ix);
    // twiddles + line buffers; lines are padded to whole 128-byte bank rows plus one
    // value (the kernels swizzle the index inside a line)
    const int bank = 128 / csz;
    const int ls = (n + bank - 1) / bank * bank + 1;
    fs.smem_x = (n + 2 * fs.lx * ls) * csz;
    fs.smem_y = (n + 2 * fs.ly * ls) * csz;
    fs.smem_z = (n + (2 + 2 * g.nf) * fs.lz * ls) * csz;
    fs.smem_iy = (n + 2 * fs.liy * ls) * csz;
    fs.smem_ix = (n + 2 * fs.lix * ls) * csz;
    // fused plane passes (one CTA per z-plane) for FP32 grids whose twiddles and two
    // n^2/2-line buffers take <= 100 KB (n <= 112): measured faster there; larger planes
    // and FP64 (1 CTA per SM, FP64-bound butterflies on n CTAs) keep the five passes
    {
        const long long plane = (long long)(n + n * ls) * csz;
        fs.fused = (P.prec == ENUF_FP32 && plane <= 100 * 1024 && P.fft_path == 0) ? 1 : 0;
        fs.composite = 0;
        for (int st = 0; st < fp.nst; ++st)
            if (fp.rad[st] > 8 || fp.rad[st] == 6) fs.composite = 1;
        fs.smem_xy = fs.smem_yx = (int)plane;
        fs.t_xy = fs.t_yx = 512;
    }
    if (fp.f1) {
        // two-factor kernels: per line f1 (f2 + 1) phase-A values and n + 1 results;
        // threads: one phase-A or phase-B task per thread (f2 resp. f1 per line)
        fs.two = 1;
        const int lsa = fft2_lsa(fp.f1, fp.f2), lsb = fft2_lsb(n), per_line = (lsa + lsb) * csz;
        const int fmax = std::max(fp.f1, fp.f2);
        auto shape2 = [&](int total_lines, int mult, int& lines, int& threads, int& grid, int bud) {
            const int cap = std::max(1, std::min(64, (bud - n * csz) / (mult * per_line)));
            lines = std::max(1, std::min(cap, (total_lines + 2 * kSMs - 1) / (2 * kSMs)));
            grid = (total_lines + lines - 1) / lines;
            threads = std::min(512, std::max(64, ((mult * lines * fmax + 31) / 32) * 32));
        };
        // persistent passes (x, inverse y, inverse x): the next group's input (extra
        // bytes per line) double-buffered in shared memory; ~72 KB keeps three CTAs
        // per SM, the grid is what stays resident
        auto pipe_shape = [&](int total_lines, int extra, int& lines, int& threads, int& grid, int& smem) {
            lines = std::max(1, std::min(64, (72 * 1024 - n * csz - 16) / (per_line + extra)));
            threads = std::min(512, std::max(64, ((lines * fmax + 31) / 32) * 32));
            smem = n * csz + lines * (per_line + extra) + 16;   // + alignment of the input buffers
            const int groups = (total_lines + lines - 1) / lines;
            const int by_smem = (228 * 1024) / (smem + 1024), by_threads = 2048 / threads;
            const int by_regs = 65536 / (64 * threads);
            const int per_sm = std::max(1, std::min(std::min(by_smem, by_threads), std::min(by_regs, 32)));
            grid = std::min(groups, per_sm * kSMs);
        };
        shape2(n * nc1, 1, fs.ly, fs.ty, gyz, budget);
        fs.grid_y_z = (n + fs.ly - 1) / fs.ly;
        // the z pass holds one inverse line per line, two with three fields (and
        // ~83 registers a thread): a smaller budget keeps several CTAs per SM
        const int zmul = g.nf == 3 ? 2 : 1;
        shape2(nc1 * g.K, zmul, fs.lz, fs.tz, fs.grid_z, 56 * 1024);
        fs.smem_z = n * csz + zmul * fs.lz * per_line;
        pipe_shape(n * n / 2, 4 * n * (int)sizeof(float), fs.lx, fs.tx, fs.grid_x, fs.smem_x);
        // inverse y: one CTA per group (its input lines are contiguous already; the
        // persistent form measured slower, 123 against 106 us at n = 320)
        shape2(g.nf * n * nc1, 1, fs.liy, fs.tiy, fs.grid_iy, budget);
        fs.smem_iy = n * csz + fs.liy * per_line;
        pipe_shape(g.nf * n * n / 2, 4 * nc1 * csz, fs.lix, fs.tix, fs.grid_ix, fs.smem_ix);
        fs.smem_y = n * csz + fs.ly * per_line;
        fs.smem_xy = (n + (n / 2) * (lsa + lsb)) * csz;
        fs.smem_yx = (n + (n / 2) * lsa + nc1 * lsb) * csz;
        fs.fused = (fs.smem_xy <= 100 * 1024 && P.fft_path == 0) ? 1 : 0;
        fs.composite = 0;
        // five passes: the z pass persistent as well (lines contiguous in spec2);
        // the fused plane path keeps one CTA per line group (spec2 plane-major)
        if (!fs.fused) {
            pipe_shape(nc1 * g.K, (zmul - 1) * per_line + 2 * n * csz, fs.lz, fs.tz, fs.grid_z, fs.smem_z);
            fs.tz = std::min(512, std::max(64, ((zmul * fs.lz * fmax + 31) / 32) * 32));
        }
    }
    // spreading form (FP32): bricks of whole x rows fused with the x pass where the
    // two-factor five-pass FFT runs and the brick fits; footprint bricks into the
    // grid otherwise from n = 128 on; the tile form below
    if (P.spread < 0 || P.spread > 4) return fail(plan, ENUF_ERR_INVALID, "spread must be 0..4");
    if (P.pairs < 0 || P.pairs > 2) return fail(plan, ENUF_ERR_INVALID, "pairs must be 0, 1 or 2");
    fs.spread = 1;
    if (P.prec == ENUF_FP32) {
        const int rsz = (int)sizeof(float);
        const int stage = brick_stage_bytes<float>();
        // fused: LP line pairs of the x transform after the brick (shared with the staging)
        int lp = 0, fx_smem = 0;
        const bool fx_ok = fs.two && !fs.fused && T % 2 == 0;
        if (fx_ok) {
            const int per_line = (fft2_lsa(fp.f1, fp.f2) + fft2_lsb(n)) * csz;
            const int acc = T * T * n * rsz;
            lp = std::min(std::min(16, T * T / 2), (kMaxSmem - acc - n * csz) / per_line);
            if (lp >= 2) fx_smem = brick_smem<float>(T, n, n * csz + lp * per_line);
        }
        const bool fx_fits = fx_smem > 0 && fx_smem <= kMaxSmem;
        // scatter form: regions of one tile (T = 16, 20, 24) or 2^3 tiles (T = 8, 10, 12)
        const int scE = T >= 16 ? T : 2 * T, scRT = scE / T;
        const bool sc_ok = 2 * P.p == 8 && (scE == 16 || scE == 20 || scE == 24) && g.ntd % scRT == 0 &&
                           g.ntd >= scRT + 2 && n % 4 == 0 && n >= 2 * (scE + T + 2 * P.p);
        // automatic: the scatter form where it is admitted and the grid has at least
        // 128 points per edge (measured faster than the tile form from the 192k-bead
        // electrolyte, n = 128, to 3M; at n = 96 its 64 regions leave most SMs idle);
        // the tile form otherwise (faster than forms 2 and 3 at every size measured)
        int want = P.spread == 0 ? ((sc_ok && n >= 128) ? 4 : 1) : P.spread;
        if (want == 4 && !sc_ok)
            return fail(plan, ENUF_ERR_INVALID, "spread = 4 needs p = 4, a tile edge of 8, 10, 12, 16, 20 or 24 "
                                                "whose region (%d) divides n = %d, and n >= %d",
                        scE, n, 2 * (scE + T + 2 * P.p));
        if (want == 4) {
            fs.spread = 4;
            fs.sc_E = scE;
        }
        if (want == 3 && !fx_fits)
            return fail(plan, ENUF_ERR_INVALID, "spread = 3 needs the two-factor five-pass FFT, an even tile and "
                                                "a brick that fits in shared memory");
        if (want == 3) {
            fs.spread = 3;
            fs.brick_x = n;
            fs.brick_lp = lp;
            fs.brick_smem = fx_smem;
        } else if (want == 2) {
            // the longest x run (a multiple of T dividing n) that keeps >= 4 bricks per SM
            int bx = T;
            for (int c = n; c >= T; c -= T)
                if (n % c == 0 && (long long)(n / c) * g.ntd * g.ntd >= 4 * kSMs &&
                    brick_smem<float>(T, c, 0) <= 96 * 1024) {
                    bx = c;
                    break;
                }
            if (brick_smem<float>(T, bx, 0) > kMaxSmem)
                return fail(plan, ENUF_ERR_INVALID, "spread = 2: brick of %d x %d x %d does not fit", bx, T, T);
            fs.spread = 2;
            fs.brick_x = bx;
            fs.brick_lp = 0;
            fs.brick_smem = brick_smem<float>(T, bx, 0);
        }
        if (fs.spread == 2 || fs.spread == 3) {
            fs.brick_threads = 32 * T;
            fs.brick_grid = (n / fs.brick_x) * g.ntd * g.ntd;
        }
        (void)stage;
    } else if (P.spread > 1) {
        return fail(plan, ENUF_ERR_INVALID, "spread = %d is an FP32 form", P.spread);
    }
    g.ratio = (double)n / P.L;
    g.rb = 1.0 / g.b;
    g.pref = P.deriv ? -P.kappa * n / (M_PI * P.L * P.L) : P.kappa * 2.0 / (P.L * P.L);
    g.c2a = 2.0 * P.alpha / std::sqrt(M_PI);
    g.xmaxf = largest_float_below(P.L);
    g.slater_k = P.slater_k;
    g.nmax = std::max(n_max, 1);
    if (P.slater_k || P.prec == ENUF_FP64) {
        // real-space kernel table on [0, r_c]: quintic Hermite nodes every <= 0.004
        // (interpolation error of J' ~ h^5, far below FP64 parity)
        g.kn = std::max(64, (int)std::ceil(P.r_cut / 0.004));
        g.kh = P.r_cut / g.kn;
        g.kinv = g.kn / P.r_cut;
    }
    if (P.slater_k) {
        // I'(0) = lim I(r)/r gives the self term
        double i0[3];
        slater_kernel(P.alpha, P.beta, 0.0, i0);
        g.c_self = -0.5 * P.kappa * i0[1];
        g.c_neut = -P.kappa * (M_PI / (P.alpha * P.alpha) + 2.0 * M_PI / (P.beta * P.beta)) /
                   (2.0 * P.L * P.L * P.L);
    } else {
        g.c_self = -P.kappa * P.alpha / std::sqrt(M_PI);
        g.c_neut = -P.kappa * M_PI / (2.0 * P.L * P.L * P.L * P.alpha * P.alpha);
    }
    g.c_recip = P.kappa / (2.0 * M_PI * P.L);
    g.rhi = (float)g.ratio;
    g.rlo = (float)(g.ratio - (double)g.rhi);

    Work w{};
    w.nblk_real = std::min(8 * kSMs, g.ntiles);   // one tile per CTA at most
    w.nblk_conv = fs.grid_z;
    w.nblk_dpd = 4 * kSMs;
    w.nblk_kin = kSMs;   // one block per SM: its FP64 block sum runs on each SM's few FP64 units once
    w.nblk_gather = 4 * kSMs;
    w.off_q = 0;
    w.off_real = w.off_q + 2 * g.nbin;
    w.off_recip = w.off_real + 2 * w.nblk_real;
    w.off_dpd = w.off_recip + 2 * w.nblk_conv;
    w.off_kin = w.off_dpd + 2 * w.nblk_dpd;
    w.off_pre = w.off_kin + w.nblk_kin;
    const int npart = w.off_pre + 8;

    const size_t nm = (size_t)std::max(n_max, 1);
    const size_t n3 = (size_t)n * n * n;
    const size_t ntab = (size_t)nc1 * g.K * g.K;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align256(b); return o; };
    // record offsets in w as integers for now (cast later)
    const size_t ncmp = (size_t)g.nbin * g.chunk;   // compacted-bead slots
    size_t o_cnt = take((size_t)g.nbin * 4), o_bhist = take((size_t)g.nbin * g.ntiles * 4),
           o_boff = take((size_t)g.nbin * g.ntiles * 4), o_ttot = take((size_t)g.ntiles * 4),
           o_tstart = take((size_t)(g.ntiles + 1) * 4), o_tk = take(16), o_ck = take(16), o_ctile = take(ncmp * 4),
           o_cpos = take(ncmp * 4 * esz),
           o_cfrac = take(ncmp * 4 * esz), o_cbase = take(ncmp * 4),
           o_sq = take(nm * 4 * esz), o_sw = take(nm * 4 * esz), o_sb = take(nm * 4),
           o_wb = take(nm * 3 * 2 * P.p * esz), o_grid = take(n3 * esz),
           o_s1 = take((size_t)n * nc1 * n * csz), o_s2 = take((size_t)nc1 * g.K * n * csz),
           o_s3 = take((size_t)g.nf * n * nc1 * g.K * csz), o_s4 = take((size_t)g.nf * n * n * nc1 * csz),
           o_h = take(g.nf * n3 * esz), o_tab = take(ntab * 8), o_tabv = take(ntab * 8), o_tabr = take(ntab * esz),
           o_tw = take((size_t)n * csz), o_part = take((size_t)npart * 8), o_E = take(16 * 8),
           o_ktab = take((size_t)g.kn * (P.prec == ENUF_FP64 ? kKtStride64 : kKtStride32) * esz);
    if (bytes) *bytes = off;
    if (plan) {
        plan->P = P;
        plan->P.M = M;
        plan->P.tile = T;
        plan->n_max = n_max;
        plan->prec = P.prec;
        plan->rsz = esz;
        plan->g = g;
        plan->fs = fs;
        plan->fp = fp;
        // stash offsets; bound to the allocation in bind()
        w.cnt_blk = (int*)o_cnt; w.bhist = (int*)o_bhist; w.boff = (int*)o_boff; w.ttot = (int*)o_ttot;
        w.tstart = (int*)o_tstart; w.ticket = (int*)o_tk; w.check = (unsigned int*)o_ck; w.ctile = (int*)o_ctile;
        w.cpos = (void*)o_cpos; w.cfrac = (void*)o_cfrac;
        w.cbase = (int*)o_cbase;
        w.sq = (void*)o_sq; w.sw = (void*)o_sw; w.sb = (int*)o_sb; w.wb = (void*)o_wb; w.grid = (void*)o_grid;
        w.spec1 = (void*)o_s1; w.spec2 = (void*)o_s2; w.spec3 = (void*)o_s3; w.spec4 = (void*)o_s4;
        w.h = (void*)o_h; w.tab = (double*)o_tab; w.tabv = (double*)o_tabv; w.tabr = (void*)o_tabr;
        w.tw = (void*)o_tw; w.part = (double*)o_part; w.Edev = (double*)o_E; w.ktab = (void*)o_ktab;
        plan->w = w;
        plan->dbytes = off;
    }
    return ENUF_OK;
}

void bind(enuf_plan_t p) {
    char* b = static_cast<char*>(p->dmem);
    Work& w = p->w;
    auto at = [&](auto ptr) { return reinterpret_cast<decltype(ptr)>(b + reinterpret_cast<size_t>(ptr)); };
    w.cnt_blk = at(w.cnt_blk); w.bhist = at(w.bhist); w.boff = at(w.boff); w.ttot = at(w.ttot);
    w.tstart = at(w.tstart); w.ticket = at(w.ticket); w.check = at(w.check); w.ctile = at(w.ctile);
    w.cpos = at(w.cpos); w.cfrac = at(w.cfrac);
    w.cbase = at(w.cbase);
    w.sq = at(w.sq); w.sw = at(w.sw); w.sb = at(w.sb); w.wb = at(w.wb); w.grid = at(w.grid);
    w.spec1 = at(w.spec1); w.spec2 = at(w.spec2); w.spec3 = at(w.spec3); w.spec4 = at(w.spec4);
    w.h = at(w.h); w.tab = at(w.tab); w.tabv = at(w.tabv); w.tabr = at(w.tabr);
    w.tw = at(w.tw); w.part = at(w.part); w.Edev = at(w.Edev); w.ktab = at(w.ktab);
    p->g.ktab = p->g.kn > 0 ? w.ktab : nullptr;
    p->g.check = w.check;
}

// FP64 influence x deconvolution table over the half space kx = 0..nc:
// D(k) = e^{-(pi k)^2/(alpha L)^2} / (k^2 prod_t c(k_t)^2), c(k) = e^{-b (pi k/n)^2}
// (Eq. 18/20 divided by the window's Fourier factor twice: once for the
// transposed, once for the conjugated NFFT); 0 at k = 0 and outside the mode set.
enuf_status upload_tables(enuf_plan_t plan) {
    const Geo& g = plan->g;
    const int nc = g.nc, K = g.K, n = g.n;
    const size_t ntab = (size_t)(nc + 1) * K * K;
    std::vector<double> D(ntab, 0.0), Dv(ntab, 0.0);
    std::vector<double> c(K);
    for (int i = 0; i < K; ++i) {
        const double t = M_PI * (i - nc) / n;
        c[i] = std::exp(-g.b * t * t);
    }
    const double aL = g.alpha * g.L;
    for (int kx = 0; kx <= nc; ++kx)
        for (int iy = 0; iy < K; ++iy)
            for (int iz = 0; iz < K; ++iz) {
                const int ky = iy - nc, kz = iz - nc;
                const double k2 = (double)kx * kx + (double)ky * ky + (double)kz * kz;
                if (k2 == 0) continue;
                if (g.kmask == 1 && k2 > (double)nc * nc) continue;
                const double cc = c[kx + nc] * c[iy] * c[iz];
                double d = std::exp(-M_PI * M_PI * k2 / (aL * aL)) / k2 / (cc * cc);
                double vw = 1.0 - 2.0 * M_PI * M_PI * k2 / (aL * aL);   // -L d/dL per mode
                if (g.slater_k) {   // form factor (1 + t)^{-2}, t = (pi |m| / (beta L))^2
                    const double bL = g.beta * g.L;
                    const double t = M_PI * M_PI * k2 / (bL * bL);
                    d /= (1.0 + t) * (1.0 + t);
                    vw -= 4.0 * t / (1.0 + t);
                }
                const size_t id = ((size_t)kx * K + iy) * K + iz;
                D[id] = d;
                Dv[id] = d * vw;
            }
    CU(cudaMemcpy(plan->w.tab, D.data(), ntab * 8, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(plan->w.tabv, Dv.data(), ntab * 8, cudaMemcpyHostToDevice));
    if (g.kn > 0) {
        // J(r) = r u(r) and its first two derivatives at the nodes r = j h, in FP64:
        // J = erfc(alpha r) - (1 + beta r) e^{-2 beta r} (the Slater term for beta > 0),
        // or with the form factor in k space J = B1(r) - I(r) (the two terms nearly
        // cancel over the cutoff range, so they are formed here, not in the kernel)
        const int kn = g.kn;
        std::vector<double> J((size_t)(kn + 1) * 3);
        const double al = g.alpha, be = g.beta, c2a = 2.0 * al / std::sqrt(M_PI);
        for (int j = 0; j <= kn; ++j) {
            const double r = j * g.kh;
            double* y = &J[3 * (size_t)j];
            if (g.slater_k) {
                const double e = std::exp(-2.0 * be * r);
                double I[3];
                slater_kernel(al, be, r, I);
                y[0] = 1.0 - (1.0 + be * r) * e - I[0];
                y[1] = be * (1.0 + 2.0 * be * r) * e - I[1];
                y[2] = -4.0 * be * be * be * r * e - I[2];
            } else {
                const double ea = c2a * std::exp(-al * al * r * r);
                y[0] = std::erfc(al * r);
                y[1] = -ea;
                y[2] = 2.0 * al * al * r * ea;
                if (be > 0) {
                    const double e = std::exp(-2.0 * be * r);
                    y[0] -= (1.0 + be * r) * e;
                    y[1] += be * (1.0 + 2.0 * be * r) * e;
                    y[2] -= 4.0 * be * be * be * r * e;
                }
            }
        }
        // quintic Hermite interpolant on [j h, (j + 1) h] in t = r/h - j, power basis:
        // c0 = y0, c1 = h y0', c2 = h^2 y0''/2, and c3..c5 from the values at t = 1
        const bool f64 = plan->prec == ENUF_FP64;
        const int st = f64 ? kKtStride64 : kKtStride32;
        std::vector<double> C((size_t)kn * st, 0.0);
        const double h = g.kh;
        for (int j = 0; j < kn; ++j) {
            const double* a = &J[3 * (size_t)j];
            const double* b = a + 3;
            const double y0 = a[0], d0 = h * a[1], s0 = h * h * a[2];
            const double y1 = b[0], d1 = h * b[1], s1 = h * h * b[2];
            double* c = &C[(size_t)j * st];
            c[0] = y0;
            c[1] = d0;
            c[2] = 0.5 * s0;
            c[3] = 10.0 * (y1 - y0) - 6.0 * d0 - 4.0 * d1 - 1.5 * s0 + 0.5 * s1;
            c[4] = -15.0 * (y1 - y0) + 8.0 * d0 + 7.0 * d1 + 1.5 * s0 - s1;
            c[5] = 6.0 * (y1 - y0) - 3.0 * d0 - 3.0 * d1 - 0.5 * s0 + 0.5 * s1;
        }
        if (f64) {
            CU(cudaMemcpy(plan->w.ktab, C.data(), C.size() * 8, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> cf(C.begin(), C.end());
            CU(cudaMemcpy(plan->w.ktab, cf.data(), cf.size() * 4, cudaMemcpyHostToDevice));
        }
    }
    std::vector<double> tw(2 * n);
    for (int t = 0; t < n; ++t) {
        tw[2 * t] = std::cos(2.0 * M_PI * t / n);
        tw[2 * t + 1] = -std::sin(2.0 * M_PI * t / n);
    }
    if (plan->prec == ENUF_FP32) {
        std::vector<float> Df(D.begin(), D.end()), twf(tw.begin(), tw.end());
        CU(cudaMemcpy(plan->w.tabr, Df.data(), ntab * 4, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(plan->w.tw, twf.data(), 2 * n * 4, cudaMemcpyHostToDevice));
    } else {
        CU(cudaMemcpy(plan->w.tabr, D.data(), ntab * 8, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(plan->w.tw, tw.data(), 2 * n * 8, cudaMemcpyHostToDevice));
    }
    return ENUF_OK;
}

// fuse_totals: the gather's last block also reduces the energies (evaluations
// outside a DPD step, where nothing follows the gather).
// step: a DPD step, whose energies but the kinetic one are reduced on the
// side stream beside the gather (plan->evT then orders the closing kick).
enuf_status enqueue_eval(enuf_plan_t plan, const EvalArgs& a, cudaStream_t s0, cudaStream_t s1,
                         cudaEvent_t evFork, cudaEvent_t evJoin, Events* ev, LaunchLog* log, bool fuse_totals,
                         const DpdDev* dpd = nullptr, bool step = false) {
    cudaError_t e;
    cudaEvent_t evZ = step ? plan->evZ : nullptr, evT = step ? plan->evT : nullptr;
    if (plan->prec == ENUF_FP32)
        e = enqueue_enuf<float>(plan->g, plan->fs, plan->fp, plan->w, a, s0, s1, evFork, evJoin, ev, log,
                                fuse_totals, dpd, evZ, evT);
    else
        e = enqueue_enuf<double>(plan->g, plan->fs, plan->fp, plan->w, a, s0, s1, evFork, evJoin, ev, log,
                                 fuse_totals, dpd, evZ, evT);
    if (e != cudaSuccess) return fail(plan, ENUF_ERR_CUDA, "enqueue: %s", cudaGetErrorString(e));
    return ENUF_OK;
}

enuf_status enqueue_tot(enuf_plan_t plan, bool dpd, cudaStream_t s, LaunchLog* log) {
    const bool pdl = !plan->ev.on;   // with stage events the predecessor is an event node
    cudaError_t e = plan->prec == ENUF_FP32 ? enqueue_totals<float>(plan->g, plan->w, dpd, s, log, pdl)
                                            : enqueue_totals<double>(plan->g, plan->w, dpd, s, log, pdl);
    if (e != cudaSuccess) return fail(plan, ENUF_ERR_CUDA, "totals: %s", cudaGetErrorString(e));
    return ENUF_OK;
}

void drop_graph(enuf_plan_t p) {
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
    p->g_n = -1;
}

// Capture one evaluation (and the D2H copy of the totals) as a graph.
enuf_status capture_eval(enuf_plan_t plan, int n, const void* pos, const void* q, void* F) {
    drop_graph(plan);
    cudaGraph_t graph = nullptr;
    CU(cudaStreamBeginCapture(plan->stream, cudaStreamCaptureModeThreadLocal));
    LaunchLog log;
    Events* ev = plan->ev.on ? &plan->ev : nullptr;
    if (ev) cudaEventRecordWithFlags(ev->start[6], plan->stream, cudaEventRecordExternal);
    EvalArgs a{n, pos, q, F, true};
    enuf_status st = enqueue_eval(plan, a, plan->stream, plan->aux, plan->evFork, plan->evJoin, ev, &log, true);
    if (st == ENUF_OK) {
        cudaError_t e = cudaMemcpyAsync(plan->hE, plan->w.Edev, 16 * sizeof(double), cudaMemcpyDeviceToHost,
                                        plan->stream);
        if (e != cudaSuccess) st = fail(plan, ENUF_ERR_CUDA, "memcpy: %s", cudaGetErrorString(e));
    }
    if (ev) cudaEventRecordWithFlags(ev->stop[6], plan->stream, cudaEventRecordExternal);
    cudaError_t e = cudaStreamEndCapture(plan->stream, &graph);
    if (st != ENUF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(plan, ENUF_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiateWithFlags(&plan->gexec, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(plan, ENUF_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
    plan->g_n = n;
    plan->g_pos = pos;
    plan->g_q = q;
    plan->g_F = F;
    plan->g_timing = plan->ev.on;
    plan->launches = log.kernels;
    return ENUF_OK;
}

enuf_status finish_energies(enuf_plan_t plan, double* E, double* virial) {
    if (!E && !virial) return ENUF_OK;
    CU(cudaStreamSynchronize(plan->stream));
    if (E)
        for (int i = 0; i < 4; ++i) E[i] = plan->hE[i];
    if (virial) *virial = plan->hE[7];
    return ENUF_OK;
}

}  // namespace

extern "C" {

const char* enuf_status_string(enuf_status s) {
    switch (s) {
        case ENUF_OK: return "ok";
        case ENUF_ERR_INVALID: return "invalid argument";
        case ENUF_ERR_OOM: return "out of device memory";
        case ENUF_ERR_CUDA: return "CUDA error";
        case ENUF_ERR_TIMEOUT: return "device wait timed out";
        case ENUF_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char* enuf_last_error(enuf_plan_t plan) { return plan ? plan->err : "no plan"; }

enuf_status enuf_accuracy_params(double delta, enuf_params* params) {
    if (!params || !(delta > 0.0 && delta < 1.0)) return ENUF_ERR_INVALID;
    const double L = params->L, rc = params->r_cut;
    if (!(L > 0.0) || !(rc > 0.0) || rc > 0.5 * L) return ENUF_ERR_INVALID;
    // Eq. 29, real space: the smallest alpha with erfc(alpha r_c) <= delta
    // (erfc falls monotonically; bisection on alpha r_c in [0, 40])
    double lo = 0.0, hi = 40.0;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        (std::erfc(mid) <= delta ? hi : lo) = mid;
    }
    const double alpha = hi / rc;
    // Eq. 29, reciprocal space: n_c >= (alpha L / pi) sqrt(-ln delta); the
    // base grid keeps n_c = M/2 - 1, rounded up to an even 2^a 3^b 5^c M
    int nc = (int)std::ceil(alpha * L / M_PI * std::sqrt(-std::log(delta)));
    // rounding of the bound: take the condition itself, exp(-(pi n_c/(alpha L))^2) <= delta
    while (std::exp(-std::pow(M_PI * nc / (alpha * L), 2)) > delta) ++nc;
    int M = 2 * (nc + 1);
    while (!smooth(M)) M += 2;
    if (2 * M > 1024) return ENUF_ERR_UNSUPPORTED;
    params->alpha = alpha;
    params->M = M;
    return ENUF_OK;
}

enuf_status enuf_footprint(const enuf_params* params, int n_max, size_t* bytes) {
    if (!params || !bytes) return ENUF_ERR_INVALID;
    return derive(nullptr, *params, n_max, bytes);
}

enuf_status enuf_plan(const enuf_params* params, int n_max, void* cuda_stream, enuf_plan_t* out) {
    if (!out || !params) return ENUF_ERR_INVALID;
    *out = nullptr;
    enuf_plan_t plan = new (std::nothrow) enuf_plan_s();
    if (!plan) return ENUF_ERR_OOM;
    enuf_status st = derive(plan, *params, n_max, nullptr);
    if (st != ENUF_OK) {
        fprintf(stderr, "enuf_plan: %s\n", plan->err);
        delete plan;
        return st;
    }
    auto bail = [&](enuf_status s) {
        fprintf(stderr, "enuf_plan: %s\n", plan->err);
        enuf_destroy(plan);
        return s;
    };
    {
        cudaError_t e = ensure_configured(plan->prec);
        if (e != cudaSuccess) return bail(fail(plan, ENUF_ERR_CUDA, "configure: %s", cudaGetErrorString(e)));
    }
    if (cuda_stream) {
        plan->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&plan->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(plan, ENUF_ERR_CUDA, "stream create failed"));
        plan->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&plan->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->evFork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->evJoin, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->evA, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->evZ, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->evT, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(plan, ENUF_ERR_CUDA, "stream/event create failed"));
    for (int i = 0; i < kStageCount; ++i)
        if (cudaEventCreate(&plan->ev.start[i]) != cudaSuccess || cudaEventCreate(&plan->ev.stop[i]) != cudaSuccess)
            return bail(fail(plan, ENUF_ERR_CUDA, "event create failed"));
    cudaError_t e = dev_alloc(&plan->dmem, plan->dbytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        plan->dmem = nullptr;
        return bail(fail(plan, ENUF_ERR_OOM, "cudaMalloc(%zu): %s", plan->dbytes, cudaGetErrorString(e)));
    }
    bind(plan);
    if (cudaMemset(plan->dmem, 0, plan->dbytes) != cudaSuccess)
        return bail(fail(plan, ENUF_ERR_CUDA, "memset failed"));
    if (cudaMallocHost(&plan->hE, 16 * sizeof(double)) != cudaSuccess)
        return bail(fail(plan, ENUF_ERR_OOM, "pinned alloc failed"));
    st = upload_tables(plan);
    if (st != ENUF_OK) return bail(st);
    *out = plan;
    return ENUF_OK;
}

// DPD pair launches of a plan: 1 (two launches) or 2 (one launch); automatic:
// one in FP32, two in FP64 (measured at the 81000-bead polyelectrolyte)
static int pair_launches(const enuf_params& P) { return P.pairs ? P.pairs : (P.prec == ENUF_FP32 ? 2 : 1); }

static void fill_info(const enuf_plan_s* plan, enuf_plan_info* info) {
    info->M = plan->P.M;
    info->n = plan->g.n;
    info->n_c = plan->g.nc;
    info->tile = plan->g.T;
    info->n_tiles = plan->g.ntiles;
    info->n_max = plan->n_max;
    info->fft_kernels = plan->fs.fused ? 3 : (plan->fs.spread == 3 ? 4 : 5);
    info->device_bytes = plan->dbytes;
    info->fft_two_factor = plan->fp.f1 ? 1 : 0;
    info->spread = plan->fs.spread;
    info->brick_x = plan->fs.spread == 2 || plan->fs.spread == 3 ? plan->fs.brick_x : 0;
    info->pairs = pair_launches(plan->P);
    if (plan->fp.f1) {
        info->fft_stages = 2;
        for (int i = 0; i < 8; ++i) info->fft_radix[i] = i == 0 ? plan->fp.f1 : (i == 1 ? plan->fp.f2 : 0);
    } else {
        info->fft_stages = plan->fp.nst;
        for (int i = 0; i < 8; ++i) info->fft_radix[i] = i < plan->fp.nst ? plan->fp.rad[i] : 0;
    }
}

enuf_status enuf_get_info(enuf_plan_t plan, enuf_plan_info* info) {
    if (!plan || !info) return ENUF_ERR_INVALID;
    fill_info(plan, info);
    return ENUF_OK;
}

enuf_status enuf_plan_shape(const enuf_params* params, int n_max, enuf_plan_info* info) {
    if (!params || !info) return ENUF_ERR_INVALID;
    std::unique_ptr<enuf_plan_s> tmp(new (std::nothrow) enuf_plan_s());
    if (!tmp) return ENUF_ERR_OOM;
    const enuf_status st = derive(tmp.get(), *params, n_max, nullptr);
    if (st != ENUF_OK) return st;
    fill_info(tmp.get(), info);
    return ENUF_OK;
}

enuf_status enuf_check_word(enuf_plan_t plan, unsigned int* mask, int reset) {
    if (!plan || !mask) return ENUF_ERR_INVALID;
    CU(cudaStreamSynchronize(plan->stream));
    CU(cudaMemcpy(mask, plan->w.check, sizeof(unsigned int), cudaMemcpyDeviceToHost));
    if (reset) CU(cudaMemset(plan->w.check, 0, sizeof(unsigned int)));
    return ENUF_OK;
}

int enuf_built_with_checks(void) {
#ifdef ENUF_CHECK
    return 1;
#else
    return 0;
#endif
}

enuf_status enuf_debug_fail_allocs(int after, int count) {
    if (after < 0 || count < 0) return ENUF_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_fail_mu);
    g_fail_after = after;
    g_fail_count = count;
    return ENUF_OK;
}

enuf_status enuf_energy_forces(enuf_plan_t plan, int n, const void* pos, const void* q, void* F, double* E,
                               double* virial) {
    if (!plan) return ENUF_ERR_INVALID;
    if (n < 0 || n > plan->n_max) return fail(plan, ENUF_ERR_INVALID, "n = %d outside [0, n_max = %d]", n, plan->n_max);
    if (n > 0 && (!pos || !q || !F)) return fail(plan, ENUF_ERR_INVALID, "null array");
    if (!plan->gexec || plan->g_n != n || plan->g_pos != pos || plan->g_q != q || plan->g_F != F ||
        plan->g_timing != plan->ev.on) {
        enuf_status st = capture_eval(plan, n, pos, q, F);
        if (st != ENUF_OK) return st;
    }
    CU(cudaGraphLaunch(plan->gexec, plan->stream));
    return finish_energies(plan, E, virial);
}

enuf_status enuf_last_energies(enuf_plan_t plan, double* E, double* virial) {
    if (!plan || !E) return ENUF_ERR_INVALID;
    for (int i = 0; i < 8; ++i) E[i] = plan->hE[i];
    if (virial) *virial = plan->hE[7];
    return ENUF_OK;
}

enuf_status enuf_energy_forces_host(enuf_plan_t plan, int n, const void* pos, const void* q, void* F, double* E,
                                    double* virial) {
    if (!plan) return ENUF_ERR_INVALID;
    if (n < 0 || n > plan->n_max) return fail(plan, ENUF_ERR_INVALID, "n = %d outside [0, n_max = %d]", n, plan->n_max);
    if (n > 0 && (!pos || !q || !F)) return fail(plan, ENUF_ERR_INVALID, "null array");
    const size_t nm = (size_t)std::max(plan->n_max, 1);
    if (!plan->stage) {
        cudaError_t e = dev_alloc(&plan->stage, align256(nm * 3 * plan->rsz) * 2 + align256(nm * plan->rsz));
        if (e != cudaSuccess) {
            cudaGetLastError();
            plan->stage = nullptr;
            return fail(plan, ENUF_ERR_OOM, "staging alloc: %s", cudaGetErrorString(e));
        }
    }
    char* b = static_cast<char*>(plan->stage);
    void* dpos = b;
    void* dF = b + align256(nm * 3 * plan->rsz);
    void* dq = b + 2 * align256(nm * 3 * plan->rsz);
    if (n > 0) {
        CU(cudaMemcpyAsync(dpos, pos, (size_t)n * 3 * plan->rsz, cudaMemcpyHostToDevice, plan->stream));
        CU(cudaMemcpyAsync(dq, q, (size_t)n * plan->rsz, cudaMemcpyHostToDevice, plan->stream));
    }
    enuf_status st = enuf_energy_forces(plan, n, dpos, dq, dF, nullptr, nullptr);
    if (st != ENUF_OK) return st;
    if (n > 0) CU(cudaMemcpyAsync(F, dF, (size_t)n * 3 * plan->rsz, cudaMemcpyDeviceToHost, plan->stream));
    CU(cudaStreamSynchronize(plan->stream));
    if (E)
        for (int i = 0; i < 4; ++i) E[i] = plan->hE[i];
    if (virial) *virial = plan->hE[7];
    return ENUF_OK;
}

enuf_status enuf_debug_buffer(enuf_plan_t plan, int which, void* host, size_t bytes) {
    if (!plan || !host) return ENUF_ERR_INVALID;
    const size_t n3 = (size_t)plan->g.n * plan->g.n * plan->g.n;
    const void* src = nullptr;
    size_t need = 0;
    if (which == ENUF_BUF_GRID) { src = plan->w.grid; need = n3 * plan->rsz; }
    else if (which == ENUF_BUF_FIELD) { src = plan->w.h; need = (size_t)plan->g.nf * n3 * plan->rsz; }
    else return fail(plan, ENUF_ERR_INVALID, "unknown buffer %d", which);
    if (bytes != need) return fail(plan, ENUF_ERR_INVALID, "buffer needs %zu bytes, got %zu", need, bytes);
    CU(cudaStreamSynchronize(plan->stream));
    CU(cudaMemcpy(host, src, need, cudaMemcpyDeviceToHost));
    return ENUF_OK;
}

enuf_status enuf_enable_timing(enuf_plan_t plan, int on) {
    if (!plan) return ENUF_ERR_INVALID;
    plan->ev.on = on != 0;
    return ENUF_OK;
}

enuf_status enuf_stage_time(enuf_plan_t plan, int stage, float* ms) {
    if (!plan || !ms || stage < 0 || stage >= kStageCount) return ENUF_ERR_INVALID;
    if (!plan->ev.on) return fail(plan, ENUF_ERR_INVALID, "timing is off");
    CU(cudaEventSynchronize(plan->ev.stop[stage]));
    CU(cudaEventElapsedTime(ms, plan->ev.start[stage], plan->ev.stop[stage]));
    return ENUF_OK;
}

int enuf_launches_per_eval(enuf_plan_t plan) { return plan ? plan->launches : 0; }

void enuf_destroy(enuf_plan_t plan) {
    if (!plan) return;
    if (plan->stream) cudaStreamSynchronize(plan->stream);
    drop_graph(plan);
    if (plan->dmem) cudaFree(plan->dmem);
    if (plan->stage) cudaFree(plan->stage);
    if (plan->hE) cudaFreeHost(plan->hE);
    for (int i = 0; i < kStageCount; ++i) {
        if (plan->ev.start[i]) cudaEventDestroy(plan->ev.start[i]);
        if (plan->ev.stop[i]) cudaEventDestroy(plan->ev.stop[i]);
    }
    if (plan->evFork) cudaEventDestroy(plan->evFork);
    if (plan->evJoin) cudaEventDestroy(plan->evJoin);
    if (plan->evA) cudaEventDestroy(plan->evA);
    if (plan->evZ) cudaEventDestroy(plan->evZ);
    if (plan->evT) cudaEventDestroy(plan->evT);
    if (plan->aux) cudaStreamDestroy(plan->aux);
    if (plan->own_stream && plan->stream) cudaStreamDestroy(plan->stream);
    delete plan;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// DPD systems
// ---------------------------------------------------------------------------
struct dpd_system_s {
    enuf_plan_t plan = nullptr;
    DpdDev d{};
    void* dmem = nullptr;
    cudaGraphExec_t gstep = nullptr;
    bool g_timing = false;
    uint64_t step = 0;
    int launches = 0;
};

namespace {

// step: inside a step graph (the energies but the kinetic one are then
// reduced beside the gather; the caller waits on plan->evT before the kick).
enuf_status enqueue_force_eval(dpd_system_t sys, cudaStream_t s0, cudaStream_t s1, Events* ev, LaunchLog* log,
                               bool step = false) {
    enuf_plan_t plan = sys->plan;
    if (ev && ev->on) s1 = s0;   // stage events: the branches one after the other
    // DPD pair + bond forces on s1 (F overwritten), after what s0 did so far
    CU(cudaEventRecord(plan->evA, s0));
    CU(cudaStreamWaitEvent(s1, plan->evA, 0));
    // one pair launch (pairs = 2): the DPD pair forces run in the real-space launch (k_pairs)
    const bool fuse = pair_launches(plan->P) == 2;
    cudaError_t e = plan->prec == ENUF_FP32 ? enqueue_dpd_forces<float>(plan->w, sys->d, s1, ev, log, !fuse)
                                            : enqueue_dpd_forces<double>(plan->w, sys->d, s1, ev, log, !fuse);
    if (e != cudaSuccess) return fail(plan, ENUF_ERR_CUDA, "dpd enqueue: %s", cudaGetErrorString(e));
    // electrostatics added into F (real space follows the DPD kernel on s1)
    EvalArgs a{sys->d.N, sys->d.pos, sys->d.q, sys->d.F, false};
    return enqueue_eval(plan, a, s0, s1, plan->evFork, plan->evJoin, ev, log, false, fuse ? &sys->d : nullptr, step);
}

enuf_status initial_force(dpd_system_t sys) {
    enuf_plan_t plan = sys->plan;
    LaunchLog log;
    CU(cudaMemcpyAsync(sys->d.v0, sys->d.vel, (size_t)sys->d.N * 3 * plan->rsz, cudaMemcpyDeviceToDevice,
                       plan->stream));
    enuf_status st = enqueue_force_eval(sys, plan->stream, plan->aux, nullptr, &log);
    if (st != ENUF_OK) return st;
    st = enqueue_tot(plan, true, plan->stream, &log);
    if (st != ENUF_OK) return st;
    CU(cudaMemcpyAsync(plan->hE, plan->w.Edev, 16 * sizeof(double), cudaMemcpyDeviceToHost, plan->stream));
    CU(cudaStreamSynchronize(plan->stream));
    CU(cudaGetLastError());
    return ENUF_OK;
}

enuf_status capture_step(dpd_system_t sys) {
    enuf_plan_t plan = sys->plan;
    if (sys->gstep) cudaGraphExecDestroy(sys->gstep);
    sys->gstep = nullptr;
    cudaGraph_t graph = nullptr;
    CU(cudaStreamBeginCapture(plan->stream, cudaStreamCaptureModeThreadLocal));
    LaunchLog log;
    Events* ev = plan->ev.on ? &plan->ev : nullptr;
    if (ev) cudaEventRecordWithFlags(ev->start[6], plan->stream, cudaEventRecordExternal);
    cudaError_t e = plan->prec == ENUF_FP32 ? enqueue_vv_pre<float>(sys->d, plan->stream, &log)
                                            : enqueue_vv_pre<double>(sys->d, plan->stream, &log);
    enuf_status st = e == cudaSuccess ? ENUF_OK : fail(plan, ENUF_ERR_CUDA, "vv_pre: %s", cudaGetErrorString(e));
    if (st == ENUF_OK) st = enqueue_force_eval(sys, plan->stream, plan->aux, ev, &log, true);
    if (st == ENUF_OK) {
        // the last block of the half kick adds the kinetic energy to the
        // step's other energies (reduced beside the gather) and forms the totals
        e = cudaStreamWaitEvent(plan->stream, plan->evT, 0);
        if (e == cudaSuccess)
            e = plan->prec == ENUF_FP32
                    ? enqueue_vv_post<float>(plan->g, plan->w, sys->d, plan->stream, &log, false, true)
                    : enqueue_vv_post<double>(plan->g, plan->w, sys->d, plan->stream, &log, false, true);
        if (e != cudaSuccess) st = fail(plan, ENUF_ERR_CUDA, "vv_post: %s", cudaGetErrorString(e));
    }
    // the step's energies stay in device memory: a copy to the host (a graph node
    // each step cost ~5 us at 81k beads) is enqueued only when asked
    // (dpd_step / dpd_step_host with E, dpd_copy_energies)
    if (ev) cudaEventRecordWithFlags(ev->stop[6], plan->stream, cudaEventRecordExternal);
    e = cudaStreamEndCapture(plan->stream, &graph);
    if (st != ENUF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(plan, ENUF_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiateWithFlags(&sys->gstep, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(plan, ENUF_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
    sys->g_timing = plan->ev.on;
    sys->launches = log.kernels;
    plan->launches = log.kernels;
    return ENUF_OK;
}

}  // namespace

extern "C" {

enuf_status dpd_create(enuf_plan_t plan, const dpd_params* params, int n, const void* pos, const void* vel,
                       const int* type, const void* q, int n_bonds, const int* bonds, dpd_system_t* out) {
    if (!plan || !params || !out) return ENUF_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || n > plan->n_max) return fail(plan, ENUF_ERR_INVALID, "n = %d outside [1, n_max]", n);
    if (!pos || !vel || !type || !q || (n_bonds > 0 && !bonds) || n_bonds < 0)
        return fail(plan, ENUF_ERR_INVALID, "null array");
    if (n_bonds > (1 << 28)) return fail(plan, ENUF_ERR_INVALID, "n_bonds = %d too large", n_bonds);
    if (params->ntypes < 1 || !params->a) return fail(plan, ENUF_ERR_INVALID, "ntypes < 1 or a == NULL");
    if (!(params->dt > 0)) return fail(plan, ENUF_ERR_INVALID, "dt must be > 0");
    const double L = plan->P.L;
    if (std::floor(L / (1.0 + 1e-5)) < 3.0)
        return fail(plan, ENUF_ERR_INVALID, "DPD needs L >= 3 (1 + 1e-5): 3 cells of edge > 1 per box edge");
    for (int i = 0; i < n; ++i)
        if (type[i] < 0 || type[i] >= params->ntypes) return fail(plan, ENUF_ERR_INVALID, "type[%d] out of range", i);
    for (int k = 0; k < 2 * n_bonds; ++k)
        if (bonds[k] < 0 || bonds[k] >= n) return fail(plan, ENUF_ERR_INVALID, "bond index out of range");

    dpd_system_t sys = new (std::nothrow) dpd_system_s();
    if (!sys) return ENUF_ERR_OOM;
    sys->plan = plan;
    DpdDev& d = sys->d;
    d.check = plan->w.check;
    d.N = n;
    d.ntypes = params->ntypes;
    // cell edge L/ncd >= 1 + 1e-5: float rounding of x * ncd/L cannot put two
    // beads closer than the cutoff 1 two cells apart
    d.ncd = std::max(1, (int)std::floor(L / (1.0 + 1e-5)));
    d.ncells = d.ncd * d.ncd * d.ncd;
    d.L = L;
    d.gamma = params->gamma;
    d.sigma = params->sigma;
    d.dt = params->dt;
    d.lambda_vv = params->lambda_vv;
    d.K_bond = params->K_bond;
    d.r0_bond = params->r0_bond;
    d.seed = params->seed;
    for (int r = 0; r < 10; ++r) {   // Philox4x32-10 round keys (Salmon et al., SC'11)
        d.rk0[r] = (uint32_t)d.seed + (uint32_t)r * 0x9E3779B9u;
        d.rk1[r] = (uint32_t)(d.seed >> 32) + (uint32_t)r * 0xBB67AE85u;
    }
    d.rdt = 1.0 / std::sqrt(params->dt);
    // cell blocks of B^3 cells: the largest B <= 4 (and <= ncd - 2, so the
    // (B + 2)^3 halo holds distinct cells) whose mean halo population stays
    // below 85% of the staging capacity (density 3: B = 4; density 4: B = 3)
    d.B = std::max(1, std::min(4, d.ncd - 2));
    {
        const double cell = L / d.ncd;
        const double per_cell = (double)n / (L * L * L) * cell * cell * cell;
        while (d.B > 1 && (d.B + 2) * (d.B + 2) * (d.B + 2) * per_cell > 0.85 * kDpdCap) --d.B;
    }
    d.cinv = (double)d.ncd / L;
    d.xmaxf = largest_float_below(L);
    const size_t rs = plan->rsz;
    const size_t nz = (size_t)n;
    d.nbonds = n_bonds;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align256(b); return o; };
    const size_t o_pos = take(nz * 3 * rs), o_vel = take(nz * 3 * rs), o_v0 = take(nz * 3 * rs),
                 o_F = take(nz * 3 * rs), o_q = take(nz * rs), o_type = take(nz * 4),
                 o_atab = take((size_t)d.ntypes * d.ntypes * rs), o_bnd = take(std::max<size_t>(1, (size_t)n_bonds) * 8),
                 o_ckey = take(nz * 4),
                 o_ccount = take((size_t)d.ncells * 4), o_cstart = take(((size_t)d.ncells + 1) * 4),
                 o_ccur = take(((size_t)d.ncells + 1) * 4), o_sp = take(nz * 4 * rs), o_sv = take(nz * 4 * rs),
                 o_step = take(8);
    cudaError_t e = dev_alloc(&sys->dmem, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete sys;
        return fail(plan, ENUF_ERR_OOM, "dpd alloc(%zu): %s", off, cudaGetErrorString(e));
    }
    char* b = static_cast<char*>(sys->dmem);
    d.pos = b + o_pos; d.vel = b + o_vel; d.v0 = b + o_v0; d.F = b + o_F; d.q = b + o_q;
    d.type = reinterpret_cast<int*>(b + o_type); d.atab = b + o_atab;
    d.bnd = reinterpret_cast<int*>(b + o_bnd);
    d.ckey = reinterpret_cast<int*>(b + o_ckey); d.ccount = reinterpret_cast<int*>(b + o_ccount);
    d.cstart = reinterpret_cast<int*>(b + o_cstart); d.ccur = reinterpret_cast<int*>(b + o_ccur);
    d.sp = b + o_sp; d.sv = b + o_sv; d.step_dev = reinterpret_cast<uint64_t*>(b + o_step);
    auto bail = [&](enuf_status s) { dpd_destroy(sys); return s; };
    if (cudaMemset(sys->dmem, 0, off) != cudaSuccess) return bail(fail(plan, ENUF_ERR_CUDA, "memset failed"));
    std::vector<char> at((size_t)d.ntypes * d.ntypes * rs);
    for (int k = 0; k < d.ntypes * d.ntypes; ++k) {
        if (rs == 4) reinterpret_cast<float*>(at.data())[k] = (float)params->a[k];
        else reinterpret_cast<double*>(at.data())[k] = params->a[k];
    }
    if (cudaMemcpy(d.pos, pos, nz * 3 * rs, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.vel, vel, nz * 3 * rs, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.q, q, nz * rs, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.type, type, nz * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.atab, at.data(), at.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (n_bonds > 0 && cudaMemcpy(d.bnd, bonds, (size_t)n_bonds * 8, cudaMemcpyHostToDevice) != cudaSuccess))
        return bail(fail(plan, ENUF_ERR_CUDA, "upload failed"));
    enuf_status st = initial_force(sys);
    if (st != ENUF_OK) return bail(st);
    *out = sys;
    return ENUF_OK;
}

enuf_status dpd_step(dpd_system_t sys, int nsteps, double* E) {
    if (!sys) return ENUF_ERR_INVALID;
    enuf_plan_t plan = sys->plan;
    if (nsteps < 0) return fail(plan, ENUF_ERR_INVALID, "nsteps < 0");
    if (!sys->gstep || sys->g_timing != plan->ev.on) {
        enuf_status st = capture_step(sys);
        if (st != ENUF_OK) return st;
    }
    for (int s = 0; s < nsteps; ++s) CU(cudaGraphLaunch(sys->gstep, plan->stream));
    sys->step += (uint64_t)nsteps;
    if (E) {
        CU(cudaMemcpyAsync(plan->hE, plan->w.Edev, 16 * sizeof(double), cudaMemcpyDeviceToHost, plan->stream));
        CU(cudaStreamSynchronize(plan->stream));
        for (int i = 0; i < 8; ++i) E[i] = plan->hE[i];
    }
    return ENUF_OK;
}

enuf_status dpd_copy_energies(dpd_system_t sys) {
    if (!sys) return ENUF_ERR_INVALID;
    enuf_plan_t plan = sys->plan;
    CU(cudaMemcpyAsync(plan->hE, plan->w.Edev, 16 * sizeof(double), cudaMemcpyDeviceToHost, plan->stream));
    return ENUF_OK;
}

enuf_status dpd_get_state(dpd_system_t sys, void* pos, void* vel, void* F, uint64_t* step) {
    if (!sys) return ENUF_ERR_INVALID;
    enuf_plan_t plan = sys->plan;
    const size_t b = (size_t)sys->d.N * 3 * plan->rsz;
    if (pos) CU(cudaMemcpyAsync(pos, sys->d.pos, b, cudaMemcpyDeviceToHost, plan->stream));
    if (vel) CU(cudaMemcpyAsync(vel, sys->d.vel, b, cudaMemcpyDeviceToHost, plan->stream));
    if (F) CU(cudaMemcpyAsync(F, sys->d.F, b, cudaMemcpyDeviceToHost, plan->stream));
    CU(cudaStreamSynchronize(plan->stream));
    if (step) *step = sys->step;
    return ENUF_OK;
}

enuf_status dpd_set_state(dpd_system_t sys, const void* pos, const void* vel, const void* F, uint64_t step) {
    if (!sys) return ENUF_ERR_INVALID;
    enuf_plan_t plan = sys->plan;
    const size_t b = (size_t)sys->d.N * 3 * plan->rsz;
    if (pos) CU(cudaMemcpyAsync(sys->d.pos, pos, b, cudaMemcpyHostToDevice, plan->stream));
    if (vel) CU(cudaMemcpyAsync(sys->d.vel, vel, b, cudaMemcpyHostToDevice, plan->stream));
    CU(cudaMemcpyAsync(sys->d.step_dev, &step, 8, cudaMemcpyHostToDevice, plan->stream));
    if (F) CU(cudaMemcpyAsync(sys->d.F, F, b, cudaMemcpyHostToDevice, plan->stream));
    // one synchronisation: the caller may reuse its buffers (and the step
    // value on this stack frame is read) once the copies have completed
    CU(cudaStreamSynchronize(plan->stream));
    sys->step = step;
    if (F) return ENUF_OK;
    return initial_force(sys);
}

enuf_status dpd_get_forces(dpd_system_t sys, void* F) { return dpd_get_state(sys, nullptr, nullptr, F, nullptr); }

enuf_status dpd_step_host(dpd_system_t sys, int nsteps, void* pos, void* vel, void* F, double* E) {
    if (!sys) return ENUF_ERR_INVALID;
    enuf_plan_t plan = sys->plan;
    if (nsteps < 0) return fail(plan, ENUF_ERR_INVALID, "nsteps < 0");
    if (!sys->gstep || sys->g_timing != plan->ev.on) {
        enuf_status st = capture_step(sys);
        if (st != ENUF_OK) return st;
    }
    const size_t b = (size_t)sys->d.N * 3 * plan->rsz;
    if (pos) CU(cudaMemcpyAsync(sys->d.pos, pos, b, cudaMemcpyHostToDevice, plan->stream));
    if (vel) CU(cudaMemcpyAsync(sys->d.vel, vel, b, cudaMemcpyHostToDevice, plan->stream));
    if (F) CU(cudaMemcpyAsync(sys->d.F, F, b, cudaMemcpyHostToDevice, plan->stream));
    for (int s = 0; s < nsteps; ++s) CU(cudaGraphLaunch(sys->gstep, plan->stream));
    sys->step += (uint64_t)nsteps;
    if (pos) CU(cudaMemcpyAsync(pos, sys->d.pos, b, cudaMemcpyDeviceToHost, plan->stream));
    if (vel) CU(cudaMemcpyAsync(vel, sys->d.vel, b, cudaMemcpyDeviceToHost, plan->stream));
    if (F) CU(cudaMemcpyAsync(F, sys->d.F, b, cudaMemcpyDeviceToHost, plan->stream));
    if (E) CU(cudaMemcpyAsync(plan->hE, plan->w.Edev, 16 * sizeof(double), cudaMemcpyDeviceToHost, plan->stream));
    CU(cudaStreamSynchronize(plan->stream));
    if (E)
        for (int i = 0; i < 8; ++i) E[i] = plan->hE[i];
    return ENUF_OK;
}

enuf_status dpd_device_state(dpd_system_t sys, void** pos, void** vel, void** F) {
    if (!sys) return ENUF_ERR_INVALID;
    if (pos) *pos = sys->d.pos;
    if (vel) *vel = sys->d.vel;
    if (F) *F = sys->d.F;
    return ENUF_OK;
}

void dpd_destroy(dpd_system_t sys) {
    if (!sys) return;
    if (sys->plan && sys->plan->stream) cudaStreamSynchronize(sys->plan->stream);
    if (sys->gstep) cudaGraphExecDestroy(sys->gstep);
    if (sys->dmem) cudaFree(sys->dmem);
    delete sys;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
struct enuf_batch_s {
    std::vector<enuf_plan_t> plans;
    std::vector<int> n;
    std::vector<cudaStream_t> s0, s1;
    std::vector<cudaEvent_t> evDone;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t evStart = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<const void*> g_pos, g_q;
    std::vector<void*> g_F;
    int launches = 0;
    // one launch sequence over all systems (FP32, see batch_eligible)
    bool seq = false;
    cudaStream_t aux = nullptr;
    cudaEvent_t evFork = nullptr, evJoin = nullptr;
    void* dtab = nullptr;      // argument tables and block maps
    size_t dtab_bytes = 0;
    double* dE = nullptr;      // [nsys][16] totals
    double* hE = nullptr;      // pinned copy
    BatchLaunch L{};
    bool built = false;
};

namespace {

// The batched kernels need each system's plan to run the fused-plane
// two-factor FFT, the column spreading form (tile edges 8..24) and the
// binning offsets in the last count block.
bool batch_plan_ok(const enuf_plan_s* p) {
    const int T = p->g.T;
    const bool col = T == 8 || T == 10 || T == 12 || T == 16 || T == 20 || T == 24;
    return p->prec == ENUF_FP32 && p->fs.two && p->fs.fused && p->fs.spread == 1 && col && p->g.bin_last &&
           p->w.wb != nullptr;
}

BatchSys batch_sys(const enuf_plan_s* p, int n, const void* pos, const void* q, void* F, double* Edev) {
    BatchSys x;
    x.g = p->g;
    x.fs = p->fs;
    x.fp = p->fp;
    x.w = p->w;
    x.N = n;
    x.pos = pos;
    x.q = q;
    x.F = F;
    x.Edev = Edev;
    return x;
}

}  // namespace

extern "C" {

enuf_status enuf_batch_plan(int nsys, const enuf_params* params, const int* n, void* cuda_stream,
                            enuf_batch_t* out) {
    if (!out || nsys < 1 || !params || !n) return ENUF_ERR_INVALID;
    *out = nullptr;
    enuf_batch_t b = new (std::nothrow) enuf_batch_s();
    if (!b) return ENUF_ERR_OOM;
    auto bail = [&](enuf_status s) { enuf_batch_destroy(b); return s; };
    if (cuda_stream) b->stream = static_cast<cudaStream_t>(cuda_stream);
    else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(ENUF_ERR_CUDA);
        b->own_stream = true;
    }
    if (cudaEventCreateWithFlags(&b->evStart, cudaEventDisableTiming) != cudaSuccess) return bail(ENUF_ERR_CUDA);
    for (int s = 0; s < nsys; ++s) {
        enuf_plan_t p = nullptr;
        enuf_status st = enuf_plan(&params[s], n[s], nullptr, &p);
        if (st != ENUF_OK) return bail(st);
        b->plans.push_back(p);
        b->n.push_back(n[s]);
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bail(ENUF_ERR_CUDA);
        b->evDone.push_back(e);
    }
    bool seq = nsys < (1 << 11);
    for (int s = 0; s < nsys && seq; ++s) seq = batch_plan_ok(b->plans[s]);
    if (seq) {
        std::vector<BatchSys> sys;
        for (int s = 0; s < nsys; ++s) sys.push_back(batch_sys(b->plans[s], n[s], nullptr, nullptr, nullptr, nullptr));
        b->dtab_bytes = batch_bytes<float>(sys.data(), nsys);
        if (dev_alloc(&b->dtab, b->dtab_bytes) != cudaSuccess) {
            cudaGetLastError();
            b->dtab = nullptr;
            return bail(ENUF_ERR_OOM);
        }
        if (dev_alloc((void**)&b->dE, (size_t)nsys * 16 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            b->dE = nullptr;
            return bail(ENUF_ERR_OOM);
        }
        if (cudaMallocHost((void**)&b->hE, (size_t)nsys * 16 * sizeof(double)) != cudaSuccess ||
            cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->evFork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->evJoin, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return bail(ENUF_ERR_CUDA);
        }
        b->seq = true;
    }
    *out = b;
    return ENUF_OK;
}

namespace {

// One launch sequence over all systems: the tables follow the caller's
// arrays; the graph (launches reading the tables, one copy of the totals)
// is captured once.
enuf_status batch_seq_eval(enuf_batch_t b, const void* const* pos, const void* const* q, void* const* F, double* E) {
    const int ns = (int)b->plans.size();
    bool same = b->built;
    for (int s = 0; same && s < ns; ++s) same = b->g_pos[s] == pos[s] && b->g_q[s] == q[s] && b->g_F[s] == F[s];
    if (!same) {
        // the previous evaluation may still read the tables
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return ENUF_ERR_CUDA;
        std::vector<BatchSys> sys;
        for (int s = 0; s < ns; ++s) sys.push_back(batch_sys(b->plans[s], b->n[s], pos[s], q[s], F[s], b->dE + 16 * s));
        BatchLaunch L{};
        if (batch_build<float>(b->dtab, sys.data(), ns, &L) != cudaSuccess) return ENUF_ERR_CUDA;
        b->L = L;
        b->g_pos.assign(pos, pos + ns);
        b->g_q.assign(q, q + ns);
        b->g_F.assign(F, F + ns);
        b->built = true;
    }
    if (!b->gexec) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ENUF_ERR_CUDA;
        LaunchLog log;
        cudaError_t e = batch_enqueue<float>(b->L, b->stream, b->aux, b->evFork, b->evJoin, &log);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->hE, b->dE, (size_t)ns * 16 * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return ENUF_ERR_CUDA;
        }
        e = cudaGraphInstantiateWithFlags(&b->gexec, graph, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return ENUF_ERR_CUDA;
        b->launches = log.kernels;
    }
    if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess) return ENUF_ERR_CUDA;
    if (E) {
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return ENUF_ERR_CUDA;
        for (int s = 0; s < ns; ++s)
            for (int i = 0; i < 4; ++i) E[4 * s + i] = b->hE[16 * s + i];
    }
    return ENUF_OK;
}

}  // namespace

enuf_status enuf_batch_energy_forces(enuf_batch_t b, const void* const* pos, const void* const* q, void* const* F,
                                     double* E) {
    if (!b || !pos || !q || !F) return ENUF_ERR_INVALID;
    const int ns = (int)b->plans.size();
    for (int s = 0; s < ns; ++s)
        if (b->n[s] > 0 && (!pos[s] || !q[s] || !F[s])) return ENUF_ERR_INVALID;
    if (b->seq) return batch_seq_eval(b, pos, q, F, E);
    bool same = b->gexec && (int)b->g_pos.size() == ns;
    for (int s = 0; same && s < ns; ++s) same = b->g_pos[s] == pos[s] && b->g_q[s] == q[s] && b->g_F[s] == F[s];
    if (!same) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ENUF_ERR_CUDA;
        cudaEventRecord(b->evStart, b->stream);
        LaunchLog log;
        enuf_status st = ENUF_OK;
        for (int s = 0; s < ns && st == ENUF_OK; ++s) {
            enuf_plan_t p = b->plans[s];
            cudaStreamWaitEvent(p->stream, b->evStart, 0);
            EvalArgs a{b->n[s], pos[s], q[s], F[s], true};
            st = enqueue_eval(p, a, p->stream, p->aux, p->evFork, p->evJoin, nullptr, &log, true);
            if (st == ENUF_OK)
                cudaMemcpyAsync(p->hE, p->w.Edev, 16 * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
            cudaEventRecord(b->evDone[s], p->stream);
            cudaStreamWaitEvent(b->stream, b->evDone[s], 0);
        }
        cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (st != ENUF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return ENUF_ERR_CUDA;
        e = cudaGraphInstantiateWithFlags(&b->gexec, graph, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return ENUF_ERR_CUDA;
        b->g_pos.assign(pos, pos + ns);
        b->g_q.assign(q, q + ns);
        b->g_F.assign(F, F + ns);
        b->launches = log.kernels;
    }
    if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess) return ENUF_ERR_CUDA;
    if (E) {
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return ENUF_ERR_CUDA;
        for (int s = 0; s < ns; ++s)
            for (int i = 0; i < 4; ++i) E[4 * s + i] = b->plans[s]->hE[i];
    }
    return ENUF_OK;
}

int enuf_batch_launches(enuf_batch_t b) { return b ? b->launches : 0; }

int enuf_batch_mode(enuf_batch_t b) { return b && b->seq ? 1 : 0; }

void enuf_batch_destroy(enuf_batch_t b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->dtab) cudaFree(b->dtab);
    if (b->dE) cudaFree(b->dE);
    if (b->hE) cudaFreeHost(b->hE);
    if (b->aux) cudaStreamDestroy(b->aux);
    if (b->evFork) cudaEventDestroy(b->evFork);
    if (b->evJoin) cudaEventDestroy(b->evJoin);
    for (auto p : b->plans) enuf_destroy(p);
    for (auto e : b->evDone) cudaEventDestroy(e);
    if (b->evStart) cudaEventDestroy(b->evStart);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free spreading. Some callers cannot allocate device memory at
// all: code that runs inside a memory-pool or arena owned by someone else,
// host threads of a framework that forbids cudaMalloc on its hot path (an
// allocation synchronises the device), or plugins whose GPU memory budget is
// fixed up front. For them the charged-bead binning and the spreading stage
// run on a fixed scratch region that is part of the library's device image:
// a file-scope device array, resident on every GPU that loads this library
// until the process exits. Its address is looked up once per device.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

}  // namespace

extern "C" enuf_status enuf_spread_noalloc(const enuf_params* params, int n, const void* pos, const void* q,
                                           void* grid, void* cuda_stream) {
    if (!params || n < 0 || !grid || (n > 0 && (!pos || !q))) {
        fprintf(stderr, "enuf_spread_noalloc: null argument or n < 0\n");
        return ENUF_ERR_INVALID;
    }
    enuf_plan_s geo;  // geometry only: nothing is allocated
    enuf_status st = derive(&geo, *params, n, nullptr);
    if (st != ENUF_OK) {
        fprintf(stderr, "enuf_spread_noalloc: %s\n", geo.err);
        return st;
    }
    const Geo& g = geo.g;
    const size_t esz = geo.rsz;
    const size_t nm = (size_t)std::max(n, 1);
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align256(b); return o; };
    const size_t ncmp = (size_t)g.nbin * g.chunk;
    const size_t o_cnt = take((size_t)g.nbin * 4), o_bhist = take((size_t)g.nbin * g.ntiles * 4),
                 o_boff = take((size_t)g.nbin * g.ntiles * 4), o_ttot = take((size_t)g.ntiles * 4),
                 o_tstart = take((size_t)(g.ntiles + 1) * 4), o_tk = take(16), o_ctile = take(ncmp * 4),
                 o_cpos = take(ncmp * 4 * esz), o_cfrac = take(ncmp * 4 * esz), o_cbase = take(ncmp * 4),
                 o_sq = take(nm * 4 * esz), o_sw = take(nm * 4 * esz), o_sb = take(nm * 4),
                 o_part = take((size_t)2 * g.nbin * 8);
    if (off > kNoAllocScratchBytes) {
        fprintf(stderr,
                "enuf_spread_noalloc: %d beads on a %d^3 grid need %zu bytes of scratch; the static scratch "
                "holds %zu bytes\n",
                n, g.n, off, kNoAllocScratchBytes);
        return ENUF_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        fprintf(stderr, "enuf_spread_noalloc: no usable current device (%s)\n", cudaGetErrorString(e));
        return ENUF_ERR_CUDA;
    }
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "enuf_spread_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
            return ENUF_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    e = ensure_configured(geo.prec);
    if (e != cudaSuccess) {
        fprintf(stderr, "enuf_spread_noalloc: %s\n", cudaGetErrorString(e));
        return ENUF_ERR_CUDA;
    }
    char* b = static_cast<char*>(g_noalloc_addr[dev]);
    Work w{};
    w.cnt_blk = reinterpret_cast<int*>(b + o_cnt);
    w.bhist = reinterpret_cast<int*>(b + o_bhist);
    w.boff = reinterpret_cast<int*>(b + o_boff);
    w.ttot = reinterpret_cast<int*>(b + o_ttot);
    w.tstart = reinterpret_cast<int*>(b + o_tstart);
    w.ticket = reinterpret_cast<int*>(b + o_tk);   // cleared below, before the binning counts on it
    w.ctile = reinterpret_cast<int*>(b + o_ctile);
    w.cpos = b + o_cpos;
    w.cfrac = b + o_cfrac;
    w.cbase = reinterpret_cast<int*>(b + o_cbase);
    w.sq = b + o_sq;
    w.sw = b + o_sw;
    w.sb = reinterpret_cast<int*>(b + o_sb);
    w.part = reinterpret_cast<double*>(b + o_part);
    w.off_q = 0;
    EvalArgs a{n, pos, q, nullptr, false};
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the binning's arrival counter must start at zero: a call that stopped
    // part way could have left it set (a memset node allocates nothing)
    e = cudaMemsetAsync(w.ticket, 0, 16, s);
    if (e == cudaSuccess)
        e = geo.prec == ENUF_FP32 ? enqueue_spread_only<float>(g, w, a, grid, s)
                                  : enqueue_spread_only<double>(g, w, a, grid, s);
    if (e != cudaSuccess) {
        fprintf(stderr, "enuf_spread_noalloc: launch: %s\n", cudaGetErrorString(e));
        return ENUF_ERR_CUDA;
    }
    return ENUF_OK;
}
