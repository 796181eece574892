// enuf_enqueue.cuh -- launch sequences of one ENUF evaluation and one DPD
// step. Two streams: s0 carries binning -> spread -> FFT passes -> gather, s1
// carries the DPD pair forces and the real-space electrostatics, which only
// depend on the binning and write F; the branches join before the gather.
// Every sequence is stream-ordered and capturable into a CUDA graph.
#pragma once
#include <algorithm>
#include <utility>

#include "enuf_batch.cuh"
#include "enuf_fft2.cuh"
#include "enuf_kernels.cuh"

namespace enuf {

constexpr int kBinThreads = 1024;

inline void rec(Events* ev, int stage, bool start, cudaStream_t s) {
    if (ev && ev->on)
        cudaEventRecordWithFlags(start ? ev->start[stage] : ev->stop[stage], s, cudaEventRecordExternal);
}

// Programmatic dependent launch where pdl is set: the launch of the kernel is
// prepared while the previous kernel of the stream runs; every kernel opens
// with griddepcontrol.wait, so it touches no memory before that kernel has
// completed. pdl is off for a kernel whose stream predecessor is not a kernel
// (an event wait, an event record, the start of a graph).
//
// Priority: the reciprocal chain (binning, spreading, FFT passes, gather,
// integrator, totals) is the critical path of a step; its kernels launch at
// the device's greatest priority and the DPD / real-space branch at the
// lowest, so the block scheduler gives the chain its CTAs first and the other
// branch fills the gaps (graphs are instantiated with node priorities).
inline int launch_priority(bool critical) {
    static const int greatest = [] {
        int least = 0, great = 0;
        cudaDeviceGetStreamPriorityRange(&least, &great);
        return great;
    }();
    return critical ? greatest : 0;
}

template <typename... P, typename... A>
inline void launch(bool pdl, bool critical, void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                   A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = launch_priority(critical);
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 2 : 1;
    cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

inline bool pdl_ok(const Events* ev) { return !(ev && ev->on); }

// Totals inputs of a plan (dpd: include the DPD and kinetic partials); the
// ticket index selects the arrival counter of the reducing kernel.
inline TotalsArgs totals_args(const Geo& g, const Work& w, bool dpd, int ticket) {
    TotalsArgs t;
    t.part = w.part;
    t.off_q = w.off_q;
    t.nq = g.nbin;
    t.off_real = w.off_real;
    t.nreal = w.nblk_real;
    t.off_recip = w.off_recip;
    t.nrecip = w.nblk_conv;
    t.off_dpd = w.off_dpd;
    t.ndpd = dpd ? w.nblk_dpd : 0;
    t.off_kin = w.off_kin;
    t.nkin = dpd ? w.nblk_kin : 0;
    t.Edev = w.Edev;
    t.ticket = w.ticket + ticket;
    t.pre = nullptr;
    return t;
}
inline TotalsArgs no_totals() {
    TotalsArgs t{};
    t.Edev = nullptr;
    return t;
}

template <typename R>
cudaError_t configure_kernels(int max_smem) {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (r != cudaSuccess) e = r;
    };
    set((const void*)k_bin_count<R>);
    // the count kernel may hold a whole SM's shared memory (its chunk list and
    // the tile histogram; see the plan's chunk rule)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)k_bin_count<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBinSmem);
    set((const void*)k_bin_scatter<R>);
    set((const void*)k_spread<R>);
    set((const void*)k_fft_x<R>);
    set((const void*)k_fft_y<R>);
    set((const void*)k_fft_z<R>);
    set((const void*)k_fft_iy<R>);
    set((const void*)k_fft_ix<R>);
    if constexpr (sizeof(R) == 4) {
        set((const void*)k_fft_x<R, true>);
        set((const void*)k_fft_y<R, true>);
        set((const void*)k_fft_z<R, true>);
        set((const void*)k_fft_iy<R, true>);
        set((const void*)k_fft_ix<R, true>);
        set((const void*)k_fft_xy<R, true>);
        set((const void*)k_fft_yx<R, true>);
    }
    set((const void*)k_spread_col<R, 8, false>);
    set((const void*)k_spread_col<R, 8, true>);
    set((const void*)k_spread_col<R, 10, false>);
    set((const void*)k_spread_col<R, 10, true>);
    set((const void*)k_spread_col<R, 12, false>);
    set((const void*)k_spread_col<R, 12, true>);
    set((const void*)k_spread_col<R, 16, false>);
    set((const void*)k_spread_col<R, 16, true>);
    set((const void*)k_spread_col<R, 20, false>);
    set((const void*)k_spread_col<R, 20, true>);
    set((const void*)k_spread_col<R, 24, false>);
    set((const void*)k_spread_col<R, 24, true>);
    set((const void*)k_fft_xy<R>);
    set((const void*)k_fft_yx<R>);
    // the FFT passes prefer the largest shared-memory carve-out (several CTAs per SM)
    auto carve = [&](const void* f) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (r != cudaSuccess) e = r;
    };
    if constexpr (sizeof(R) == 4) {
        carve((const void*)k2_fft_x<R>);
        carve((const void*)k2_fft_y<R>);
        carve((const void*)k2_fft_z<R>);
        carve((const void*)k2_fft_zp<R>);
        carve((const void*)k2_fft_iy<R>);
        carve((const void*)k2_fft_ix<R>);
        set((const void*)k2_fft_x<R>);
        set((const void*)k2_fft_y<R>);
        set((const void*)k2_fft_z<R>);
        set((const void*)k2_fft_zp<R>);
        set((const void*)k2_fft_iy<R>);
        set((const void*)k2_fft_ix<R>);
        set((const void*)k2_fft_xy<R>);
        set((const void*)k2_fft_yx<R>);
        set((const void*)k_spread_brick<R, false>);
        set((const void*)k_spread_brick<R, true>);
        set((const void*)k_spread_sc<16, 8>);
        set((const void*)k_spread_sc<20, 8>);
        set((const void*)k_spread_sc<24, 8>);
        set((const void*)kb_bin_count<R>);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)kb_bin_count<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kBinSmem);
        set((const void*)kb_bin_scatter<R>);
        set((const void*)kb_real<R>);
        set((const void*)kb_spread_col<R, 8>);
        set((const void*)kb_spread_col<R, 10>);
        set((const void*)kb_spread_col<R, 12>);
        set((const void*)kb_spread_col<R, 16>);
        set((const void*)kb_spread_col<R, 20>);
        set((const void*)kb_spread_col<R, 24>);
        set((const void*)kb_fft_xy<R>);
        set((const void*)kb_fft_z<R>);
        set((const void*)kb_fft_yx<R>);
    }
    set((const void*)k_real<R>);
    set((const void*)k_dpd<R>);
    set((const void*)k_pairs<R>);
    return e;
}

template <typename R>
int spread_smem(const Geo& g) {
    return kSpreadCap * (int)sizeof(typename V4<R>::T) + spread_tile_slots(g.T) * (int)sizeof(R) +
           (kSpreadThreads / 32) * 3 * kMaxTaps * ((int)sizeof(R) + 4) + kSpreadCap * 4 + kSpreadCap * 8;
}

// a1: compaction + coordinates + tile histograms, tile offsets, tile scan, scatter.
// Blocks of the weights kernel: enough words per thread for the plan's capacity,
// at most four CTAs per SM.
inline int bin_weight_blocks(const Geo& g) {
    const long long words = (long long)g.nbin * g.chunk * 6 * g.p;
    return (int)std::max(1LL, std::min((long long)4 * 152, (words + 255) / 256));
}

template <typename R>
void enqueue_bin(const Geo& g, const Work& w, int N, const R* pos, const R* q, R* Fzero, cudaStream_t s, bool pdl) {
    using V = typename V4<R>::T;
    launch(false, true, k_bin_count<R>, g.nbin, kBinThreads, (g.ntiles + g.chunk) * sizeof(int), s, g, N, pos, q,
           w.cnt_blk, w.bhist, w.ctile, static_cast<V*>(w.cpos), static_cast<V*>(w.cfrac), w.cbase, Fzero,
           w.part + w.off_q, w.ticket, w.boff, w.tstart);
    if (!g.bin_last) {
        launch(pdl, true, k_tile_offsets, (g.ntiles + 255) / 256, 256, 0, s, g, (const int*)w.bhist, w.boff, w.ttot);
        launch(pdl, true, k_scan, 1, 1024, 0, s, w.ttot, w.tstart, g.ntiles, (int*)nullptr, 0);
    }
    launch(pdl, true, k_bin_scatter<R>, g.nbin, kBinThreads, g.ntiles * sizeof(int), s, g, (const int*)w.cnt_blk,
           (const int*)w.ctile, static_cast<const V*>(w.cpos), static_cast<const V*>(w.cfrac), (const int*)w.cbase,
           (const int*)w.boff, (const int*)w.tstart, static_cast<V*>(w.sq), static_cast<V*>(w.sw), w.sb);
    if (w.wb)
        launch(pdl, true, k_bin_weights<R>, bin_weight_blocks(g), 256, 0, s, g, (const int*)w.tstart,
               static_cast<const V*>(w.sw), static_cast<R*>(w.wb));
}

// Kernels enqueue_bin launches.
inline int bin_kernels(const Geo& g, const Work& w) { return (g.bin_last ? 2 : 4) + (w.wb ? 1 : 0); }

// Spreading: for the common tile edges the column-stationary kernel (FP32)
// or its slab form (FP64, where the FP64 instruction count decides), the
// work-item kernel with shared-memory atomics otherwise (or without weights).
template <typename R, int T>
inline void launch_col(const Geo& g, const Work& w, R* grid, cudaStream_t s, bool pdl) {
    using V = typename V4<R>::T;
    constexpr bool SLAB = sizeof(R) == 8;
    launch(pdl, true, k_spread_col<R, T, SLAB>, g.ntiles, spread2_threads<SLAB>(T), col_smem<R>(T, SLAB), s, g,
           (const int*)w.tstart, static_cast<const V*>(w.sq), (const int*)w.sb, static_cast<const R*>(w.wb), grid);
}

template <typename R>
inline void enqueue_spread(const Geo& g, const Work& w, R* grid, cudaStream_t s, bool pdl) {
    using V = typename V4<R>::T;
    if (w.wb) {
        switch (g.T) {
            case 8: launch_col<R, 8>(g, w, grid, s, pdl); return;
            case 10: launch_col<R, 10>(g, w, grid, s, pdl); return;
            case 12: launch_col<R, 12>(g, w, grid, s, pdl); return;
            case 16: launch_col<R, 16>(g, w, grid, s, pdl); return;
            case 20: launch_col<R, 20>(g, w, grid, s, pdl); return;
            case 24: launch_col<R, 24>(g, w, grid, s, pdl); return;
            default: break;
        }
    }
    launch(pdl, true, k_spread<R>, g.ntiles, kSpreadThreads, spread_smem<R>(g), s, g, (const int*)w.tstart,
           static_cast<const V*>(w.sq), static_cast<const V*>(w.sw), (const int*)w.sb, grid);
}

// The FFT passes of one evaluation (fused plane passes or five line passes);
// CR selects the kernels compiled with the composite radices.
// Footprint spreading on bricks (FP32): into the grid (spread = 2), or fused
// with the forward x pass into spec1 (spread = 3).
template <typename R>
void enqueue_spread_brick(const Geo& g, const FftShape& fs, const FftPlanDev& fp, const Work& w, cudaStream_t s,
                          bool pdl) {
    using V = typename V4<R>::T;
    using C = typename Cx<R>::T;
    auto k = fs.spread == 3 ? k_spread_brick<R, true> : k_spread_brick<R, false>;
    launch(pdl, true, k, fs.brick_grid, fs.brick_threads, fs.brick_smem, s, g, fp, fs.brick_x, (const int*)w.tstart,
           static_cast<const V*>(w.sq), (const int*)w.sb, static_cast<const R*>(w.wb), static_cast<R*>(w.grid),
           static_cast<const C*>(w.tw), static_cast<C*>(w.spec1), fs.brick_lp);
}

// Scatter-form spreading (FP32, spread = 4): one CTA per region of edge sc_E.
inline void enqueue_spread_sc(const Geo& g, const FftShape& fs, const Work& w, cudaStream_t s, bool pdl) {
    const int regions = (g.n / fs.sc_E) * (g.n / fs.sc_E) * (g.n / fs.sc_E);
    auto k = fs.sc_E == 16 ? k_spread_sc<16, 8> : (fs.sc_E == 20 ? k_spread_sc<20, 8> : k_spread_sc<24, 8>);
    launch(pdl, true, k, regions, kScThreads, sc_smem(fs.sc_E), s, g, (const int*)w.tstart,
           static_cast<const float4*>(w.sq), (const int*)w.sb, static_cast<const float*>(w.wb),
           static_cast<float*>(w.grid));
}

// The same passes on the two-factor kernels (FP32 grids with n = f1 f2); with
// the spreading fused with the x pass (spread = 3) the x pass is already done.
// evZ (or nullptr) is recorded right after the z pass, whose blocks write the
// reciprocal energy and virial partials (the kernel after it then launches
// without programmatic dependent launch: its stream predecessor is the record).
template <typename R>
void enqueue_fft2(const Geo& g, const FftShape& fs, const FftPlanDev& fp, const Work& w, cudaStream_t s0, bool pdl,
                  LaunchLog* log, cudaEvent_t evZ) {
    using C = typename Cx<R>::T;
    const C* tw = static_cast<const C*>(w.tw);
    if (fs.fused) {
        launch(pdl, true, k2_fft_xy<R>, g.n, fs.t_xy, fs.smem_xy, s0, g, fp, static_cast<const R*>(w.grid), tw,
               static_cast<C*>(w.spec2));
        launch(pdl, true, k2_fft_z<R>, fs.grid_z, fs.tz, fs.smem_z, s0, g, fp, static_cast<const C*>(w.spec2), tw,
               (const double*)w.tab, (const double*)w.tabv, static_cast<const R*>(w.tabr), static_cast<C*>(w.spec3),
               w.part + w.off_recip, fs.lz, 1);
        if (evZ) cudaEventRecord(evZ, s0);
        launch(pdl && !evZ, true, k2_fft_yx<R>, g.nf * g.n, fs.t_yx, fs.smem_yx, s0, g, fp,
               static_cast<const C*>(w.spec3), tw, static_cast<R*>(w.h));
        log->kernels += 4;
    } else {
        if (fs.spread != 3) {
            launch(pdl, true, k2_fft_x<R>, fs.grid_x, fs.tx, fs.smem_x, s0, g, fp, static_cast<const R*>(w.grid), tw,
                   static_cast<C*>(w.spec1), fs.lx);
            log->kernels += 1;
        }
        launch(pdl, true, k2_fft_y<R>, dim3(g.nc + 1, fs.grid_y_z), fs.ty, fs.smem_y, s0, g, fp,
               static_cast<const C*>(w.spec1), tw, static_cast<C*>(w.spec2), fs.ly);
        launch(pdl, true, k2_fft_zp<R>, fs.grid_z, fs.tz, fs.smem_z, s0, g, fp, static_cast<const C*>(w.spec2), tw,
               (const double*)w.tab, (const double*)w.tabv, static_cast<const R*>(w.tabr), static_cast<C*>(w.spec3),
               w.part + w.off_recip, fs.lz);
        if (evZ) cudaEventRecord(evZ, s0);
        launch(pdl && !evZ, true, k2_fft_iy<R>, fs.grid_iy, fs.tiy, fs.smem_iy, s0, g, fp,
               static_cast<const C*>(w.spec3), tw, static_cast<C*>(w.spec4), fs.liy);
        launch(pdl, true, k2_fft_ix<R>, fs.grid_ix, fs.tix, fs.smem_ix, s0, g, fp, static_cast<const C*>(w.spec4),
               tw, static_cast<R*>(w.h), fs.lix);
        log->kernels += 5;   // the spreading kernel and four passes
    }
}

template <typename R, bool CR>
void enqueue_fft(const Geo& g, const FftShape& fs, const FftPlanDev& fp, const Work& w, cudaStream_t s0, bool pdl,
                 LaunchLog* log, cudaEvent_t evZ) {
    using C = typename Cx<R>::T;
    const C* tw = static_cast<const C*>(w.tw);
    if (fs.fused) {   // whole z-planes in shared memory: x+y, z (+convolve), y+x
        launch(pdl, true, k_fft_xy<R, CR>, g.n, fs.t_xy, fs.smem_xy, s0, g, fp, static_cast<const R*>(w.grid),
               tw, static_cast<C*>(w.spec2));
        launch(pdl, true, k_fft_z<R, CR>, fs.grid_z, fs.tz, fs.smem_z, s0, g, fp, static_cast<const C*>(w.spec2),
               tw, (const double*)w.tab, (const double*)w.tabv, static_cast<const R*>(w.tabr),
               static_cast<C*>(w.spec3), w.part + w.off_recip, fs.lz, 1);
        if (evZ) cudaEventRecord(evZ, s0);
        launch(pdl && !evZ, true, k_fft_yx<R, CR>, g.nf * g.n, fs.t_yx, fs.smem_yx, s0, g, fp,
               static_cast<const C*>(w.spec3), tw, static_cast<R*>(w.h));
        log->kernels += 4;
    } else {
        launch(pdl, true, k_fft_x<R, CR>, fs.grid_x, fs.tx, fs.smem_x, s0, g, fp, static_cast<const R*>(w.grid),
               tw, static_cast<C*>(w.spec1), fs.lx);
        launch(pdl, true, k_fft_y<R, CR>, dim3(g.nc + 1, fs.grid_y_z), fs.ty, fs.smem_y, s0, g, fp,
               static_cast<const C*>(w.spec1), tw, static_cast<C*>(w.spec2), fs.ly);
        launch(pdl, true, k_fft_z<R, CR>, fs.grid_z, fs.tz, fs.smem_z, s0, g, fp, static_cast<const C*>(w.spec2),
               tw, (const double*)w.tab, (const double*)w.tabv, static_cast<const R*>(w.tabr),
               static_cast<C*>(w.spec3), w.part + w.off_recip, fs.lz, 0);
        if (evZ) cudaEventRecord(evZ, s0);
        launch(pdl && !evZ, true, k_fft_iy<R, CR>, fs.grid_iy, fs.tiy, fs.smem_iy, s0, g, fp,
               static_cast<const C*>(w.spec3), tw, static_cast<C*>(w.spec4), fs.liy);
        launch(pdl, true, k_fft_ix<R, CR>, fs.grid_ix, fs.tix, fs.smem_ix, s0, g, fp, static_cast<const C*>(w.spec4),
               tw, static_cast<R*>(w.h), fs.lix);
        log->kernels += 6;
    }
}

// the gather with its tap loops unrolled for the common window widths
template <typename R>
auto gather_kernel(int taps) {
    switch (taps) {
        case 6: return k_gather<R, 6>;
        case 8: return k_gather<R, 8>;
        case 10: return k_gather<R, 10>;
        case 12: return k_gather<R, 12>;
        default: return k_gather<R, 0>;
    }
}

template <typename R>
cudaError_t enqueue_enuf(const Geo& g, const FftShape& fs, const FftPlanDev& fp, const Work& w,
                         const EvalArgs& a, cudaStream_t s0, cudaStream_t s1, cudaEvent_t evFork,
                         cudaEvent_t evJoin, Events* ev, LaunchLog* log, bool fuse_totals, const DpdDev* dpd,
                         cudaEvent_t evZ, cudaEvent_t evT) {
    using C = typename Cx<R>::T;
    using V = typename V4<R>::T;
    const R* pos = static_cast<const R*>(a.pos);
    const R* q = static_cast<const R*>(a.q);
    R* F = static_cast<R*>(a.F);
    V* sq = static_cast<V*>(w.sq);
    V* sw = static_cast<V*>(w.sw);
    const bool pdl = pdl_ok(ev);
    // with per-stage events the two branches run one after the other, so that
    // each stage's events time its kernels alone
    if (ev && ev->on) s1 = s0;
    rec(ev, 0, true, s0);
    enqueue_bin<R>(g, w, a.N, pos, q, a.zeroF ? F : nullptr, s0, pdl);
    rec(ev, 0, false, s0);
    log->kernels += bin_kernels(g, w);

    // real-space branch
    cudaEventRecord(evFork, s0);
    cudaStreamWaitEvent(s1, evFork, 0);
    rec(ev, 4, true, s1);
    const int real_smem = real_smem_bytes<R>();
    if (dpd) {   // DPD pairs and real-space pairs in one launch
        const DpdDev& d = *dpd;
        launch(false, false, k_pairs<R>, w.nblk_dpd + w.nblk_real, kRealThreads,
               std::max(real_smem, dpd_smem_bytes<R>()), s1, d, d.B, static_cast<const V*>(d.sp),
               static_cast<const V*>(d.sv), (const int*)d.cstart, static_cast<const R*>(d.atab),
               static_cast<const R*>(d.pos), (const int*)d.bnd, (const uint64_t*)d.step_dev, static_cast<R*>(d.F),
               w.part + w.off_dpd, w.nblk_dpd, g, (const int*)w.tstart, (const V*)sq, (const V*)sw,
               w.part + w.off_real);
    } else {
        launch(false, false, k_real<R>, w.nblk_real, kRealThreads, real_smem, s1, g, (const int*)w.tstart,
               (const V*)sq, (const V*)sw, F, w.part + w.off_real);
    }
    rec(ev, 4, false, s1);
    cudaEventRecord(evJoin, s1);
    log->kernels += 1;

    // reciprocal branch
    rec(ev, 1, true, s0);
    if constexpr (sizeof(R) == 4) {
        if (fs.spread == 4)
            enqueue_spread_sc(g, fs, w, s0, pdl);
        else if (fs.spread > 1)
            enqueue_spread_brick<R>(g, fs, fp, w, s0, pdl);
        else
            enqueue_spread<R>(g, w, static_cast<R*>(w.grid), s0, pdl);
    } else {
        enqueue_spread<R>(g, w, static_cast<R*>(w.grid), s0, pdl);
    }
    rec(ev, 1, false, s0);
    rec(ev, 2, true, s0);
    // a DPD step records evZ after the z pass: the side stream then reduces the
    // step's energies but the kinetic one while the last FFT pass and the gather run
    const cudaEvent_t ez = evZ && evT ? evZ : nullptr;
    if constexpr (sizeof(R) == 4) {
        if (fs.two)
            enqueue_fft2<R>(g, fs, fp, w, s0, pdl, log, ez);
        else if (fs.composite)
            enqueue_fft<R, true>(g, fs, fp, w, s0, pdl, log, ez);
        else
            enqueue_fft<R, false>(g, fs, fp, w, s0, pdl, log, ez);
    } else {
        enqueue_fft<R, false>(g, fs, fp, w, s0, pdl, log, ez);
    }
    rec(ev, 2, false, s0);

    if (ez) {   // a DPD step: its energies but the kinetic one, beside the last pass and the gather
        cudaStreamWaitEvent(s1, evZ, 0);
        TotalsArgs t = totals_args(g, w, true, 0);
        t.pre = w.part + w.off_pre;
        launch(false, false, k_totals_pre, 8, 256, 0, s1, t);
        cudaEventRecord(evT, s1);
        log->kernels += 1;
    }

    cudaStreamWaitEvent(s0, evJoin, 0);
    rec(ev, 3, true, s0);
    // with fuse_totals the gather's last block also reduces the energies
    launch(false, true, gather_kernel<R>(2 * g.p), w.nblk_gather, kGatherThreads, 0, s0, g, (const int*)w.tstart,
           (const V*)sq, (const V*)sw, (const int*)w.sb, static_cast<const R*>(w.wb), static_cast<const R*>(w.h), F,
           fuse_totals ? totals_args(g, w, false, 1) : no_totals());
    rec(ev, 3, false, s0);
    log->kernels += 1;
    return cudaGetLastError();
}

template <typename R>
cudaError_t enqueue_totals(const Geo& g, const Work& w, bool dpd, cudaStream_t s, LaunchLog* log, bool pdl) {
    launch(pdl, true, k_totals, 1, 1024, 0, s, g, totals_args(g, w, dpd, 3));
    log->kernels += 1;
    return cudaGetLastError();
}

template <typename R>
cudaError_t enqueue_dpd_forces(const Work& w, const DpdDev& d, cudaStream_t s, Events* ev, LaunchLog* log,
                               bool pair_kernel) {
    using V = typename V4<R>::T;
    const int blocks = (d.N + 255) / 256 > 0 ? (d.N + 255) / 256 : 1;
    const bool pdl = pdl_ok(ev);
    rec(ev, 7, true, s);
    // the cell count also zeroes F, which the pair kernel adds into
    launch(false, false, k_cell_count<R>, blocks, 256, 0, s, d.N, d.ncd, d.L, d.cinv, d.xmaxf, static_cast<const R*>(d.pos),
           d.ckey, d.ccount, static_cast<R*>(d.F));
    // the cell starts (and the scatter cursors): several CTAs without a
    // wait for up to kScanMbMax cells, else one CTA; k_cell_scatter then
    // clears the counts
    if (d.ncells <= kScanMbMax)
        launch(pdl, false, k_scan_mb, (d.ncells + kScanMbSpan - 1) / kScanMbSpan, 1024, 0, s,
               (const int*)d.ccount, d.cstart, d.ncells, d.ccur);
    else
        launch(pdl, false, k_scan, 1, 1024, 0, s, d.ccount, d.cstart, d.ncells, d.ccur, 0);
    launch(pdl, false, k_cell_scatter<R>, blocks, 256, 0, s, d.N, d.L, d.xmaxf, static_cast<const R*>(d.pos),
           static_cast<const R*>(d.v0), (const int*)d.type, (const int*)d.ckey, d.ccur, static_cast<V*>(d.sp),
           static_cast<V*>(d.sv), d.ccount, d.ncells);
    rec(ev, 7, false, s);
    log->kernels += 3;
    if (!pair_kernel) return cudaGetLastError();   // the pairs run in k_pairs with the real space
    rec(ev, 5, true, s);
    const int dpd_smem = dpd_smem_bytes<R>();
    launch(pdl, false, k_dpd<R>, w.nblk_dpd, kDpdThreads, dpd_smem, s, d, d.B, static_cast<const V*>(d.sp),
           static_cast<const V*>(d.sv), (const int*)d.cstart, static_cast<const R*>(d.atab),
           static_cast<const R*>(d.pos), (const int*)d.bnd, (const uint64_t*)d.step_dev, static_cast<R*>(d.F),
           w.part + w.off_dpd);
    rec(ev, 5, false, s);
    log->kernels += 1;
    return cudaGetLastError();
}

template <typename R>
cudaError_t enqueue_vv_pre(const DpdDev& d, cudaStream_t s, LaunchLog* log) {
    const int blocks = (3 * d.N + 255) / 256 > 0 ? (3 * d.N + 255) / 256 : 1;
    launch(false, true, k_vv_pre<R>, blocks, 256, 0, s, d.N, (R)d.lambda_vv, (R)d.dt, static_cast<R*>(d.pos),
           static_cast<R*>(d.vel), static_cast<R*>(d.v0), static_cast<const R*>(d.F), d.step_dev);
    log->kernels += 1;
    return cudaGetLastError();
}

// Step 6 of Table 2; the last block also reduces the step's energies (pre:
// all but the kinetic one were reduced by k_totals_pre).
template <typename R>
cudaError_t enqueue_vv_post(const Geo& g, const Work& w, const DpdDev& d, cudaStream_t s, LaunchLog* log, bool pdl,
                            bool pre) {
    TotalsArgs t = totals_args(g, w, true, 2);
    if (pre) t.pre = w.part + w.off_pre;
    launch(pdl, true, k_vv_post<R>, w.nblk_kin, 256, 0, s, g, d.N, (R)d.dt, static_cast<R*>(d.vel),
           static_cast<const R*>(d.F), w.part + w.off_kin, t);
    log->kernels += 1;
    return cudaGetLastError();
}

// Binning and spreading only, into a caller-provided grid (the allocation-free
// entry point runs this sequence on scratch it does not allocate).
template <typename R>
cudaError_t enqueue_spread_only(const Geo& g, const Work& w, const EvalArgs& a, void* grid_out, cudaStream_t s) {
    using V = typename V4<R>::T;
    enqueue_bin<R>(g, w, a.N, static_cast<const R*>(a.pos), static_cast<const R*>(a.q), nullptr, s, true);
    launch(true, true, k_spread<R>, g.ntiles, kSpreadThreads, spread_smem<R>(g), s, g, (const int*)w.tstart,
           static_cast<const V*>(w.sq), static_cast<const V*>(w.sw), (const int*)w.sb, static_cast<R*>(grid_out));
    return cudaGetLastError();
}

}  // namespace enuf

#include "enuf_batch_host.cuh"

namespace enuf {

#define ENUF_INSTANTIATE(R)                                                                                  \
    template cudaError_t configure_kernels<R>(int);                                                          \
    template int spread_smem<R>(const Geo&);                                                                 \
    template cudaError_t enqueue_enuf<R>(const Geo&, const FftShape&, const FftPlanDev&, const Work&,        \
                                         const EvalArgs&, cudaStream_t, cudaStream_t, cudaEvent_t,           \
                                         cudaEvent_t, Events*, LaunchLog*, bool, const DpdDev*,              \
                                         cudaEvent_t, cudaEvent_t);                                          \
    template cudaError_t enqueue_totals<R>(const Geo&, const Work&, bool, cudaStream_t, LaunchLog*, bool);   \
    template cudaError_t enqueue_dpd_forces<R>(const Work&, const DpdDev&, cudaStream_t, Events*,            \
                                               LaunchLog*, bool);                                            \
    template cudaError_t enqueue_vv_pre<R>(const DpdDev&, cudaStream_t, LaunchLog*);                         \
    template cudaError_t enqueue_vv_post<R>(const Geo&, const Work&, const DpdDev&, cudaStream_t, LaunchLog*,  \
                                            bool, bool);                                                     \
    template cudaError_t enqueue_spread_only<R>(const Geo&, const Work&, const EvalArgs&, void*, cudaStream_t);

}  // namespace enuf
