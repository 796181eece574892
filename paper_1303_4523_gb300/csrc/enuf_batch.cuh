// enuf_batch.cuh -- one launch sequence for many systems (FP32).
//
// A batched launch runs one kernel of the evaluation (Table 2 step 4: bin,
// spread, the fused-plane FFT passes with the convolution, gather; and the
// real-space pairs) for every system of a batch at once. The grid is the
// concatenation of the systems' own grids: block b works for system
// cmap[b] >> kBatchShift as its block cmap[b] & kBatchLocal, with the
// system's arguments read from row (system) of a device table of argument
// records. Each system keeps its own plan (grid size, tile, FFT split,
// workspace, tables), so systems of different size and box run side by side
// in one kernel; a system's last-block reductions count its own blocks only.
#pragma once
#include "enuf_fft2.cuh"

namespace enuf {

constexpr int kBatchShift = 20;
constexpr int kBatchLocal = (1 << kBatchShift) - 1;

template <typename R>
struct BinCountArgs {
    Geo g;
    int N;
    const R* pos;
    const R* q;
    int* cnt_blk;
    int* bhist;
    int* ctile;
    typename V4<R>::T* cpos;
    typename V4<R>::T* cfrac;
    int* cbase;
    R* Fzero;
    double* qpart;
    int* ticket;
    int* boff;
    int* tstart;
    int nblk;
};
template <typename R>
__global__ void __launch_bounds__(1024) kb_bin_count(const BinCountArgs<R>* __restrict__ tab, const int* __restrict__ cmap) {
    pdl_enter();
    const int m = cmap[blockIdx.x];
    const BinCountArgs<R>& a = tab[m >> kBatchShift];
    k_bin_count_body<R>(a.g, a.N, a.pos, a.q, a.cnt_blk, a.bhist, a.ctile, a.cpos, a.cfrac, a.cbase, a.Fzero, a.qpart,
                        a.ticket, a.boff, a.tstart, Blk{m & kBatchLocal, a.nblk});
}

template <typename R>
struct BinScatterArgs {
    Geo g;
    const int* cnt_blk;
    const int* ctile;
    const typename V4<R>::T* cpos;
    const typename V4<R>::T* cfrac;
    const int* cbase;
    const int* boff;
    const int* tstart;
    typename V4<R>::T* sq;
    typename V4<R>::T* sw;
    int* sb;
    int nblk;
};
template <typename R>
__global__ void __launch_bounds__(1024) kb_bin_scatter(const BinScatterArgs<R>* __restrict__ tab,
                                                      const int* __restrict__ cmap) {
    pdl_enter();
    const int m = cmap[blockIdx.x];
    const BinScatterArgs<R>& a = tab[m >> kBatchShift];
    k_bin_scatter_body<R>(a.g, a.cnt_blk, a.ctile, a.cpos, a.cfrac, a.cbase, a.boff, a.tstart, a.sq, a.sw, a.sb,
                          Blk{m & kBatchLocal, a.nblk});
}

template <typename R>
struct BinWeightsArgs {
    Geo g;
    const int* tstart;
    const typename V4<R>::T* sw;
    R* wb;
    int nblk;
};
template <typename R>
__global__ void __launch_bounds__(256) kb_bin_weights(const BinWeightsArgs<R>* __restrict__ tab, const int* __restrict__ cmap) {
    pdl_enter();
    const int m = cmap[blockIdx.x];
    const BinWeightsArgs<R>& a = tab[m >> kBatchShift];
    k_bin_weights_body<R>(a.g, a.tstart, a.sw, a.wb, Blk{m & kBatchLocal, a.nblk});
}

template <typename R>
struct RealArgs {
    Geo g;
    const int* tstart;
    const typename V4<R>::T* sq;
    const typename V4<R>::T* sw;
    R* F;
    double* rpart;
    int nblk;
};
template <typename R>
__global__ void __launch_bounds__(kRealThreads) kb_real(const RealArgs<R>* __restrict__ tab, const int* __restrict__ cmap) {
    pdl_enter();
    const int m = cmap[blockIdx.x];
    const RealArgs<R>& a = tab[m >> kBatchShift];
    k_real_body<R>(a.g, a.tstart, a.sq, a.sw, a.F, a.rpart, Blk{m & kBatchLocal, a.nblk});
}

// the column spreading form of one tile edge T (systems grouped by T)
template <typename R>
struct SpreadArgs {
    Geo g;
    const int* tstart;
    const typename V4<R>::T* sq;
    const int* sb;
    const R* wb;
    R* grid;
    int nblk;
};
template <typename R, int T>
__global__ void __launch_bounds__(col_threads(T)) kb_spread_col(const SpreadArgs<R>* __restrict__ tab,
                                                               const int* __restrict__ cmap) {
    pdl_enter();
    const int m = cmap[blockIdx.x];
    const SpreadArgs<R>& a = tab[m >> kBatchShift];
    k_spread_col_body<R, T, false>(a.g, a.tstart, a.sq, a.sb, a.wb, a.grid, Blk{m & kBatchLocal, a.nblk});
}

template <typename R>
struct FftXYArgs {
    Geo g;
    FftPlanDev fp;
    const R* grid;
    const typename Cx<R>::T* twg;
    typename Cx<R>::T* spec2;
    int nblk;
};
// the batched plane passes run thousands of CTAs: two per SM (<= 64 registers)
template <typename R>
__global__ void __launch_bounds__(512, 2) kb_fft_xy(const FftXYArgs<R>* __restrict__ tab, const int* __restrict__ cmap) {
    pdl_enter();
    const int m = cmap[blockIdx.x];
    const FftXYArgs<R>& a = tab[m >> kBatchShift];
    k2_fft_xy_body<R>(a.g, a.fp, a.grid, a.twg, a.spec2, Blk{m & kBatchLocal, a.nblk});
}

template <typename R>
struct FftZArgs {
    Geo g;
    FftPlanDev fp;
    const typename Cx<R>::T* spec2;
    const typename Cx<R>::T* twg;
    const double* tab;
    const double* tabv;
    const R* tabr;
    typename Cx<R>::T* spec3;
    double* epart;
    int LB;
    int nblk;
};
template <typename R>
__global__ void __launch_bounds__(512) kb_fft_z(const FftZArgs<R>* __restrict__ tab, const int* __restrict__ cmap) {
    pdl_enter();
    const int m = cmap[blockIdx.x];
    const FftZArgs<R>& a = tab[m >> kBatchShift];
    k2_fft_z_body<R>(a.g, a.fp, a.spec2, a.twg, a.tab, a.tabv, a.tabr, a.spec3, a.epart, a.LB, 1,
                     Blk{m & kBatchLocal, a.nblk});
}

template <typename R>
struct FftYXArgs {
    Geo g;
    FftPlanDev fp;
    const typename Cx<R>::T* spec3;
    const typename Cx<R>::T* twg;
    R* h;
    int nblk;
};
template <typename R>
__global__ void __launch_bounds__(512, 2) kb_fft_yx(const FftYXArgs<R>* __restrict__ tab, const int* __restrict__ cmap) {
    pdl_enter();
    const int m = cmap[blockIdx.x];
    const FftYXArgs<R>& a = tab[m >> kBatchShift];
    k2_fft_yx_body<R>(a.g, a.fp, a.spec3, a.twg, a.h, Blk{m & kBatchLocal, a.nblk});
}

template <typename R>
struct GatherArgs {
    Geo g;
    const int* tstart;
    const typename V4<R>::T* sq;
    const typename V4<R>::T* sw;
    const int* sb;
    const R* wb;
    const R* h;
    R* F;
    TotalsArgs tot;
    int nblk;
};
// PT: the tap count 2p when every system of the batch has the same window, else 0
template <typename R, int PT>
__global__ void __launch_bounds__(kGatherThreads, 4) kb_gather(const GatherArgs<R>* __restrict__ tab,
                                                            const int* __restrict__ cmap) {
    pdl_enter();
    const int m = cmap[blockIdx.x];
    const GatherArgs<R>& a = tab[m >> kBatchShift];
    k_gather_body<R, PT>(a.g, a.tstart, a.sq, a.sw, a.sb, a.wb, a.h, a.F, a.tot, Blk{m & kBatchLocal, a.nblk});
}

}  // namespace enuf

