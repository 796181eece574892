// enuf_batch_host.cuh -- host side of the batched launch sequence: the
// argument tables and block maps of the batched kernels (enuf_batch.cuh),
// and the launches. Instantiated for float.
#pragma once
#include <vector>

namespace enuf {

namespace batch_detail {

inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Block map of one batched kernel: for each system its blocks, as
// (system << kBatchShift) | local block.
inline void append_blocks(std::vector<int>& cmap, int sys, int nblk) {
    for (int b = 0; b < nblk; ++b) cmap.push_back((sys << kBatchShift) | b);
}

inline int bin_count_smem(const Geo& g) { return (g.ntiles + g.chunk) * (int)sizeof(int); }

}  // namespace batch_detail

template <typename R>
size_t batch_bytes(const BatchSys* sys, int nsys) {
    using namespace batch_detail;
    size_t blocks = 0;
    for (int s = 0; s < nsys; ++s) {
        const BatchSys& x = sys[s];
        blocks += 2 * (size_t)x.g.nbin + bin_weight_blocks(x.g) + x.w.nblk_real + x.g.ntiles + x.g.n + x.fs.grid_z +
                  (size_t)x.g.nf * x.g.n + x.w.nblk_gather;
    }
    const size_t rec = sizeof(BinCountArgs<R>) + sizeof(BinScatterArgs<R>) + sizeof(BinWeightsArgs<R>) +
                       sizeof(RealArgs<R>) + sizeof(SpreadArgs<R>) + sizeof(FftXYArgs<R>) + sizeof(FftZArgs<R>) +
                       sizeof(FftYXArgs<R>) + sizeof(GatherArgs<R>);
    // argument tables (the spreading table once per tile-edge group at most) and block maps
    return al256(rec * nsys) + al256(sizeof(SpreadArgs<R>) * nsys) * 6 + al256(blocks * sizeof(int)) + 20 * 256;
}

template <typename R>
cudaError_t batch_build(void* dbuf, const BatchSys* sys, int nsys, BatchLaunch* out) {
    using namespace batch_detail;
    using V = typename V4<R>::T;
    using C = typename Cx<R>::T;
    if (nsys < 1 || nsys >= (1 << (31 - kBatchShift))) return cudaErrorInvalidValue;
    char* base = static_cast<char*>(dbuf);
    size_t off = 0;
    cudaError_t err = cudaSuccess;
    // one table (records of type A) and one block map per kernel
    auto put = [&](BatchKernel& k, const void* recs, size_t rbytes, const std::vector<int>& cmap) {
        k.tab = base + off;
        off += al256(rbytes);
        k.cmap = reinterpret_cast<int*>(base + off);
        off += al256(cmap.size() * sizeof(int));
        k.blocks = (int)cmap.size();
        if (err == cudaSuccess) err = cudaMemcpy(k.tab, recs, rbytes, cudaMemcpyHostToDevice);
        if (err == cudaSuccess) err = cudaMemcpy(k.cmap, cmap.data(), cmap.size() * sizeof(int), cudaMemcpyHostToDevice);
    };
    BatchLaunch L;
    {
        std::vector<BinCountArgs<R>> a(nsys);
        std::vector<BinScatterArgs<R>> b(nsys);
        std::vector<BinWeightsArgs<R>> c(nsys);
        std::vector<int> ma, mb, mc;
        for (int s = 0; s < nsys; ++s) {
            const BatchSys& x = sys[s];
            const Geo& g = x.g;
            const Work& w = x.w;
            a[s] = BinCountArgs<R>{g, x.N, static_cast<const R*>(x.pos), static_cast<const R*>(x.q), w.cnt_blk, w.bhist,
                                   w.ctile, static_cast<V*>(w.cpos), static_cast<V*>(w.cfrac), w.cbase,
                                   static_cast<R*>(x.F), w.part + w.off_q, w.ticket, w.boff, w.tstart, g.nbin};
            b[s] = BinScatterArgs<R>{g, w.cnt_blk, w.ctile, static_cast<const V*>(w.cpos),
                                     static_cast<const V*>(w.cfrac), w.cbase, w.boff, w.tstart,
                                     static_cast<V*>(w.sq), static_cast<V*>(w.sw), w.sb, g.nbin};
            c[s] = BinWeightsArgs<R>{g, w.tstart, static_cast<const V*>(w.sw), static_cast<R*>(w.wb),
                                     bin_weight_blocks(g)};
            append_blocks(ma, s, g.nbin);
            append_blocks(mb, s, g.nbin);
            append_blocks(mc, s, c[s].nblk);
            L.bin_count.smem = std::max(L.bin_count.smem, bin_count_smem(g));
            L.bin_scatter.smem = std::max(L.bin_scatter.smem, g.ntiles * (int)sizeof(int));
        }
        put(L.bin_count, a.data(), a.size() * sizeof(a[0]), ma);
        put(L.bin_scatter, b.data(), b.size() * sizeof(b[0]), mb);
        put(L.bin_weights, c.data(), c.size() * sizeof(c[0]), mc);
        L.bin_count.threads = 1024;
        L.bin_scatter.threads = 1024;
        L.bin_weights.threads = 256;
    }
    {
        std::vector<RealArgs<R>> a(nsys);
        std::vector<int> m;
        for (int s = 0; s < nsys; ++s) {
            const BatchSys& x = sys[s];
            a[s] = RealArgs<R>{x.g, x.w.tstart, static_cast<const V*>(x.w.sq), static_cast<const V*>(x.w.sw),
                               static_cast<R*>(x.F), x.w.part + x.w.off_real, x.w.nblk_real};
            append_blocks(m, s, x.w.nblk_real);
        }
        put(L.real, a.data(), a.size() * sizeof(a[0]), m);
        L.real.threads = kRealThreads;
        L.real.smem = real_smem_bytes<R>();
    }
    {   // spreading: one launch per tile edge, the systems of that edge only
        static const int kT[6] = {8, 10, 12, 16, 20, 24};
        for (int ti = 0; ti < 6; ++ti) {
            std::vector<SpreadArgs<R>> a;
            std::vector<int> m;
            for (int s = 0; s < nsys; ++s) {
                const BatchSys& x = sys[s];
                if (x.g.T != kT[ti]) continue;
                const int row = (int)a.size();
                a.push_back(SpreadArgs<R>{x.g, x.w.tstart, static_cast<const V*>(x.w.sq), x.w.sb,
                                          static_cast<const R*>(x.w.wb), static_cast<R*>(x.w.grid), x.g.ntiles});
                append_blocks(m, row, x.g.ntiles);
            }
            if (a.empty()) continue;
            BatchKernel& k = L.spread[L.nspread++];
            put(k, a.data(), a.size() * sizeof(a[0]), m);
            k.T = kT[ti];
            k.threads = col_threads(kT[ti]);
            k.smem = col_smem<R>(kT[ti], false);
        }
    }
    {
        std::vector<FftXYArgs<R>> a(nsys);
        std::vector<FftZArgs<R>> b(nsys);
        std::vector<FftYXArgs<R>> c(nsys);
        std::vector<int> ma, mb, mc;
        for (int s = 0; s < nsys; ++s) {
            const BatchSys& x = sys[s];
            const Geo& g = x.g;
            const Work& w = x.w;
            const C* tw = static_cast<const C*>(w.tw);
            a[s] = FftXYArgs<R>{g, x.fp, static_cast<const R*>(w.grid), tw, static_cast<C*>(w.spec2), g.n};
            b[s] = FftZArgs<R>{g, x.fp, static_cast<const C*>(w.spec2), tw, (const double*)w.tab, (const double*)w.tabv,
                               static_cast<const R*>(w.tabr), static_cast<C*>(w.spec3), w.part + w.off_recip, x.fs.lz,
                               x.fs.grid_z};
            c[s] = FftYXArgs<R>{g, x.fp, static_cast<const C*>(w.spec3), tw, static_cast<R*>(w.h), g.nf * g.n};
            append_blocks(ma, s, g.n);
            append_blocks(mb, s, x.fs.grid_z);
            append_blocks(mc, s, g.nf * g.n);
            L.fft_xy.threads = std::max(L.fft_xy.threads, x.fs.t_xy);
            L.fft_xy.smem = std::max(L.fft_xy.smem, x.fs.smem_xy);
            L.fft_z.threads = std::max(L.fft_z.threads, x.fs.tz);
            L.fft_z.smem = std::max(L.fft_z.smem, x.fs.smem_z);
            L.fft_yx.threads = std::max(L.fft_yx.threads, x.fs.t_yx);
            L.fft_yx.smem = std::max(L.fft_yx.smem, x.fs.smem_yx);
        }
        put(L.fft_xy, a.data(), a.size() * sizeof(a[0]), ma);
        put(L.fft_z, b.data(), b.size() * sizeof(b[0]), mb);
        put(L.fft_yx, c.data(), c.size() * sizeof(c[0]), mc);
    }
    {
        std::vector<GatherArgs<R>> a(nsys);
        std::vector<int> m;
        for (int s = 0; s < nsys; ++s) {
            const BatchSys& x = sys[s];
            const Work& w = x.w;
            TotalsArgs t = totals_args(x.g, w, false, 1);
            t.Edev = x.Edev;
            // blocks in proportion to the system (a warp per charged bead, <= 1/8 of
            // the beads charged on average; the kernel strides over any excess)
            const int nb = std::max(1, std::min(w.nblk_gather, (x.N + 63) / 64));
            a[s] = GatherArgs<R>{x.g, w.tstart, static_cast<const V*>(w.sq), static_cast<const V*>(w.sw), w.sb,
                                 static_cast<const R*>(w.wb), static_cast<const R*>(w.h), static_cast<R*>(x.F), t, nb};
            append_blocks(m, s, nb);
        }
        put(L.gather, a.data(), a.size() * sizeof(a[0]), m);
        L.gather.threads = kGatherThreads;
        L.gather.smem = 0;
        L.gather.T = 2 * sys[0].g.p;   // the common tap count, or 0
        for (int s = 1; s < nsys; ++s)
            if (2 * sys[s].g.p != L.gather.T) L.gather.T = 0;
    }
    if (off > batch_bytes<R>(sys, nsys)) return cudaErrorInvalidValue;   // the tables outgrew their buffer
    *out = L;
    return err;
}

template <typename R>
cudaError_t batch_enqueue(const BatchLaunch& L, cudaStream_t s0, cudaStream_t s1, cudaEvent_t evFork, cudaEvent_t evJoin,
                          LaunchLog* log) {
    auto run = [&](bool pdl, bool critical, auto kern, const BatchKernel& k, auto* tab, cudaStream_t s) {
        launch(pdl, critical, kern, k.blocks, k.threads, k.smem, s, tab, (const int*)k.cmap);
        log->kernels += 1;
    };
    run(false, true, kb_bin_count<R>, L.bin_count, (const BinCountArgs<R>*)L.bin_count.tab, s0);
    run(true, true, kb_bin_scatter<R>, L.bin_scatter, (const BinScatterArgs<R>*)L.bin_scatter.tab, s0);
    run(true, true, kb_bin_weights<R>, L.bin_weights, (const BinWeightsArgs<R>*)L.bin_weights.tab, s0);
    cudaEventRecord(evFork, s0);
    cudaStreamWaitEvent(s1, evFork, 0);
    run(false, false, kb_real<R>, L.real, (const RealArgs<R>*)L.real.tab, s1);
    cudaEventRecord(evJoin, s1);
    for (int i = 0; i < L.nspread; ++i) {
        const BatchKernel& k = L.spread[i];
        const SpreadArgs<R>* tab = (const SpreadArgs<R>*)k.tab;
        const bool pdl = true;   // the predecessor is the binning's last kernel or the previous group
        switch (k.T) {
            case 8: run(pdl, true, kb_spread_col<R, 8>, k, tab, s0); break;
            case 10: run(pdl, true, kb_spread_col<R, 10>, k, tab, s0); break;
            case 12: run(pdl, true, kb_spread_col<R, 12>, k, tab, s0); break;
            case 16: run(pdl, true, kb_spread_col<R, 16>, k, tab, s0); break;
            case 20: run(pdl, true, kb_spread_col<R, 20>, k, tab, s0); break;
            case 24: run(pdl, true, kb_spread_col<R, 24>, k, tab, s0); break;
            default: return cudaErrorInvalidValue;
        }
    }
    run(true, true, kb_fft_xy<R>, L.fft_xy, (const FftXYArgs<R>*)L.fft_xy.tab, s0);
    run(true, true, kb_fft_z<R>, L.fft_z, (const FftZArgs<R>*)L.fft_z.tab, s0);
    run(true, true, kb_fft_yx<R>, L.fft_yx, (const FftYXArgs<R>*)L.fft_yx.tab, s0);
    cudaStreamWaitEvent(s0, evJoin, 0);
    const GatherArgs<R>* gtab = (const GatherArgs<R>*)L.gather.tab;
    switch (L.gather.T) {
        case 6: run(false, true, kb_gather<R, 6>, L.gather, gtab, s0); break;
        case 8: run(false, true, kb_gather<R, 8>, L.gather, gtab, s0); break;
        case 10: run(false, true, kb_gather<R, 10>, L.gather, gtab, s0); break;
        case 12: run(false, true, kb_gather<R, 12>, L.gather, gtab, s0); break;
        default: run(false, true, kb_gather<R, 0>, L.gather, gtab, s0); break;
    }
    return cudaGetLastError();
}

}  // namespace enuf
