// enuf_kernels.cuh -- sm_103a kernels of the ENUF-DPD hot path, templated on
// the working precision R (float or double). Energies, virials and charge
// sums are always reduced in double.
//
// Stages (Table 2 step 4, Eq. 14-25 of the paper):
//   bin      : charged beads -> tile bins of the oversampled grid (no global atomics)
//   spread   : transposed NFFT part 1, output-stationary shared-memory tiles
//   fft_x/y  : forward R2C/C2C passes, pruned to |k_t| <= n_c
//   fft_z    : forward z, influence x deconvolution multiply, FP64 energy and
//              virial, -i k_a D F for a = x, y, z, inverse z (conjugated NFFT part 1)
//   fft_iy/ix: inverse passes to three real fields
//   gather   : conjugated NFFT part 2, warp per bead, F_i += kappa 2 q_i/L^2 * sum psi h
//   real     : erfc Ewald + Slater correction pairs (Eq. 31, 27-28) on the tile bins
//   dpd      : conservative, dissipative and random pair forces (Eq. 2-7) + bonds
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "enuf_fft.cuh"
#include "enuf_internal.h"

namespace enuf {

template <typename R> struct V4;
template <> struct V4<float> { using T = float4; };
template <> struct V4<double> { using T = double4_32a; };

__device__ __forceinline__ float int_as_real(int v, float) { return __int_as_float(v); }
__device__ __forceinline__ double int_as_real(int v, double) { return __longlong_as_double((long long)v); }
__device__ __forceinline__ int real_as_int(float v) { return __float_as_int(v); }
__device__ __forceinline__ int real_as_int(double v) { return (int)__double_as_longlong(v); }

// Programmatic dependent launch (sm_90 and later): every kernel first waits
// until the grid before it in the stream has completed and its writes are
// visible (griddepcontrol.wait, a no-op when it was launched without the
// programmatic attribute). Nothing touches global memory before the wait. No
// kernel triggers its dependents early: CTAs of the next grid parked in the
// wait would hold shared memory that the other stream's kernels need, so the
// next grid launches at completion, with its launch work already done.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Asynchronous 16-byte global -> shared copies (both addresses 16-byte aligned),
// grouped by commit; wait_prior waits for all groups but the most recent one.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
// nbytes (a multiple of 8) from global to shared memory by the whole block:
// 16-byte granules when both ends and the size allow, else 8-byte ones; the
// caller commits the group
__device__ __forceinline__ void cp_async_block(void* sdst, const void* gsrc, int nbytes) {
    char* d = static_cast<char*>(sdst);
    const char* src = static_cast<const char*>(gsrc);
    if (((reinterpret_cast<size_t>(d) | reinterpret_cast<size_t>(src) | (size_t)nbytes) & 15) == 0) {
        for (int e = threadIdx.x; e < nbytes / 16; e += blockDim.x) cp_async16(d + 16 * e, src + 16 * e);
    } else {
        for (int e = threadIdx.x; e < nbytes / 8; e += blockDim.x) cp_async8(d + 8 * e, src + 8 * e);
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The block a kernel body works on: its index and the number of blocks of
// its launch for this system. A single-system launch passes (blockIdx.x,
// gridDim.x); a batched launch over many systems passes the block's index
// within its system's share of the grid and that share's size.
struct Blk {
    int id, n;
};

__device__ __forceinline__ float r_exp(float x) { return expf(x); }
__device__ __forceinline__ double r_exp(double x) { return exp(x); }
__device__ __forceinline__ float r_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double r_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }
// 1/sqrt: the hardware approximation in float (2 ulp). In double, Newton's
// iteration for x^{-1/2}, y <- y + y (1/2 - (x/2) y^2), from the float value:
// the relative error e goes to ~(3/2) e^2 per step, 2^-21 -> 2^-41 -> rounding
// (within 2 ulp), in 3 multiplies and 4 fused multiply-adds on the FP64 units
// instead of a correctly rounded square root and quotient. Outside the normal
// float range of x the quotient is taken.
__device__ __forceinline__ float r_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double r_rsqrt(double x) {
    const float xf = (float)x;
    if (!(xf > 1e-30f && xf < 1e30f)) return 1.0 / sqrt(x);
    double y = (double)rsqrtf(xf);
    const double h = 0.5 * x;
    y = fma(y, fma(-h, y * y, 0.5), y);
    y = fma(y, fma(-h, y * y, 0.5), y);
    return y;
}

// ---------------------------------------------------------------------------
// Coordinates. Wrapping and grid coordinates are computed in double with the
// exact operation sequence of the definition (no fused multiply-add), so the
// integer decisions (grid base, tile, cell) are reproducible.
// ---------------------------------------------------------------------------
// q = floor(x / L) comes from a float quotient (off by at most one for
// |x| < 2^20 L) corrected in double until 0 <= x - L q < L: the same q and w
// as an FP64 division would give, without one (an FP64 division is a long
// sequence on this part's few FP64 units, and DPD positions drift out of the
// box, so most steps wrap many beads).
__device__ __forceinline__ double wrap_pos(double x, double L) {
    if (x >= 0.0 && x < L) return x;
    double q = (double)floorf(__fdiv_rn((float)x, (float)L));
    double w = __dsub_rn(x, __dmul_rn(L, q));
    if (w < 0.0) {
        q -= 1.0;
        w = __dsub_rn(x, __dmul_rn(L, q));
    } else if (w >= L) {
        q += 1.0;
        w = __dsub_rn(x, __dmul_rn(L, q));
    }
    if (w >= L || w < 0.0) w = 0.0;
    return w;
}

template <typename R>
__device__ __forceinline__ double wrap_to_real(R x, double L) {
    double w = wrap_pos((double)x, L);
    if (sizeof(R) == 4) w = (double)__double2float_rn(w);
    return w;
}

// Wrapped position in the working precision. Inside [0, L) the value is kept
// as is (decided in float for float: x <= xmaxf, the largest float below L);
// outside it goes through the FP64 wrap.
__device__ __forceinline__ float wrap_r(float x, double L, float xmaxf) {
    if (x >= 0.0f && x <= xmaxf) return x;
    return __double2float_rn(wrap_pos((double)x, L));
}
__device__ __forceinline__ double wrap_r(double x, double L, float) { return wrap_pos(x, L); }

// Grid coordinate u = x_w * (n/L) in [0, n): one FP64 product and one floor
// (n/L formed once on the host), u >= n wraps to 0.
__device__ __forceinline__ void grid_coord(double xw, double ratio, int n, int& base, double& frac) {
    double u = __dmul_rn(xw, ratio);
    if (u >= (double)n) u = __dsub_rn(u, (double)n);
    const double bb = floor(u);
    base = (int)bb;
    frac = __dsub_rn(u, bb);
}

// FP32 path: the same floor decided in float on a compensated product. With
// n/L = rhi + rlo (two floats), p = fl(x rhi) and t = fl(x rlo + (x rhi - p))
// represent u = p + t to ~1e-13 relative; floor(u) = floor(p), less one when
// p is an integer and t < 0.
__device__ __forceinline__ void grid_coord_f(float x, float rhi, float rlo, int n, int& base, float& frac) {
    float p = __fmul_rn(x, rhi);
    const float e = __fmaf_rn(x, rhi, -p);
    const float t = __fmaf_rn(x, rlo, e);
    if (p >= (float)n) p = __fsub_rn(p, (float)n);
    float b = floorf(p);
    if (p == b && t < 0.0f) b = __fsub_rn(b, 1.0f);
    frac = __fadd_rn(__fsub_rn(p, b), t);
    if (b < 0.0f) b = __fadd_rn(b, (float)n);
    base = (int)b;
}

// Grid base and fraction in the working precision.
__device__ __forceinline__ void grid_coord_r(float xw, const Geo& g, int& base, float& frac) {
    grid_coord_f(xw, g.rhi, g.rlo, g.n, base, frac);
}
__device__ __forceinline__ void grid_coord_r(double xw, const Geo& g, int& base, double& frac) {
    grid_coord(xw, g.ratio, g.n, base, frac);
}

// Minimum-image difference and squared distance. For float the sequence is
// fixed with explicit intrinsics (the same sequence decides the cutoff in the
// oracle's float mode).
__device__ __forceinline__ float min_image(float a, float b, float L, float hL) {
    float d = __fsub_rn(a, b);
    if (d > hL) d = __fsub_rn(d, L);
    else if (d < -hL) d = __fadd_rn(d, L);
    return d;
}
__device__ __forceinline__ double min_image(double a, double b, double L, double hL) {
    double d = a - b;
    if (d > hL) d -= L;
    else if (d < -hL) d += L;
    return d;
}
__device__ __forceinline__ float dist2(float x, float y, float z) {
    return __fmaf_rn(z, z, __fmaf_rn(y, y, __fmul_rn(x, x)));
}
__device__ __forceinline__ double dist2(double x, double y, double z) { return x * x + y * y + z * z; }

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Block sum of two doubles; result valid in thread 0. Uses 64 doubles of shared memory.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double red[2][32];
    // warps holding only zeros skip their shuffle tree (its adds run on the
    // few FP64 units); the branch is uniform over the warp
    if (__any_sync(0xffffffffu, a != 0.0 || b != 0.0)) {
        a = warp_sum(a);
        b = warp_sum(b);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { red[0][w] = a; red[1][w] = b; }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = l < nw ? red[0][l] : 0.0;
        b = l < nw ? red[1][l] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
}

struct Kahan {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double x) {
        const double y = x - c;
        const double t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Totals quantity qd (0-8) of the 9 (Sum q, Sum q^2, E_real, W_real, E_recip,
// W_recip, E_c, E_bond, E_kin): where its per-block partials sit.
__device__ __forceinline__ void totals_src(const TotalsArgs& t, int qd, int& off, int& cnt, int& stride) {
    if (qd < 2) { off = t.off_q + qd; cnt = t.nq; stride = 2; }
    else if (qd < 4) { off = t.off_real + (qd - 2); cnt = t.nreal; stride = 2; }
    else if (qd < 6) { off = t.off_recip + (qd - 4); cnt = t.nrecip; stride = 2; }
    else if (qd < 8) { off = t.off_dpd + (qd - 6); cnt = t.ndpd; stride = 2; }
    else { off = t.off_kin; cnt = t.nkin; stride = 1; }
}

// Kahan sum, per lane, of the partials i = first, first + step, ... of
// quantity qd (eight independent loads in flight; partials come from other
// blocks and kernels: loads bypass L1).
__device__ __forceinline__ double kahan_lane(const TotalsArgs& t, int qd, int first, int step) {
    int off, cnt, stride;
    totals_src(t, qd, off, cnt, stride);
    Kahan k;
    for (int i0 = first; i0 < cnt; i0 += 8 * step) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + step * u;
            v[u] = i < cnt ? __ldcg(&t.part[off + stride * i]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) k.add(v[u]);
    }
    return k.s;
}

// Final FP64 totals (Kahan over the per-block partials) by one block of any
// multiple of 32 threads: warp w reduces the quantities qd with qd mod (warps)
// = w among the 9 (with t.pre: quantities 0-7 are read from pre and the
// warps share the kinetic partials).
// Edev: [0] E_real [1] E_recip [2] E_self+E_neutral [3] E_elec [4] E_conservative
//       [5] E_bond [6] E_kinetic [7] virial_elec
static __device__ void totals_block(const Geo& g, const TotalsArgs& t) {
    __shared__ double vals[9];
    __shared__ double kin[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (t.pre) {
        if (threadIdx.x < 8) vals[threadIdx.x] = __ldcg(&t.pre[threadIdx.x]);
        const double v = warp_sum(kahan_lane(t, 8, threadIdx.x, blockDim.x));
        if (l == 0) kin[w] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int k = 0; k < nw; ++k) s += kin[k];
            vals[8] = s;
        }
    } else {
        for (int qd = w; qd < 9; qd += nw) {
            const double v = warp_sum(kahan_lane(t, qd, l, 32));
            if (l == 0) vals[qd] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double* Edev = t.Edev;
        // constants formed on the host: no FP64 division or square root here
        const double Q = vals[0], Q2 = vals[1];
        const double e_self = g.c_self * Q2;
        const double e_neut = g.c_neut * Q * Q;
        const double e_real = vals[2], e_recip = g.c_recip * vals[4];
        Edev[0] = e_real;
        Edev[1] = e_recip;
        Edev[2] = e_self + e_neut;
        Edev[3] = e_real + e_recip + e_self + e_neut;
        Edev[4] = vals[6];
        Edev[5] = vals[7];
        Edev[6] = vals[8];
        Edev[7] = vals[3] + g.c_recip * vals[5] + 3.0 * e_neut;
        for (int i = 8; i < 16; ++i) Edev[i] = 0.0;
    }
}

// Quantities 0-7 of a DPD step's totals, one block per quantity, launched on
// the side stream once the pair kernels and the reciprocal (z) pass have
// written their partials, so that it runs beside the gather; the step's
// closing totals then add the kinetic partials only (t.pre).
static __global__ void __launch_bounds__(256) k_totals_pre(TotalsArgs t) {
    pdl_enter();
    __shared__ double ws[8];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const double v = warp_sum(kahan_lane(t, blockIdx.x, threadIdx.x, blockDim.x));
    if (l == 0) ws[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += ws[k];
        t.pre[blockIdx.x] = s;
    }
}

// The last block of a kernel to finish (arrival counter) runs the totals;
// nblk: the blocks of the launch that count on this ticket.
__device__ __forceinline__ void totals_if_last(const Geo& g, const TotalsArgs& t, int nblk) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(t.ticket, 1) == nblk - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    totals_block(g, t);
    if (threadIdx.x == 0) *t.ticket = 0;
}


// Kahan-compensated accumulator (FP64).

// ---------------------------------------------------------------------------
// a1: binning of the charged beads into tiles of the oversampled grid.
// k_bin_count: each block compacts the charged beads of its chunk (warp
//   ballots into a shared list), computes their grid coordinates in FP64 on
//   dense warps, histograms their tiles in shared memory and stores each
//   compacted bead's record.
//   The last block to finish (arrival counter) walks the per-block counts of
//   every tile (coalesced), writes each block's offset inside the tile and
//   scans the tile totals into the tile starts.
// k_bin_scatter moves the records to their sorted slots; k_bin_weights
//   computes their window weights. Besides the arrival counter the only
//   atomics are shared-memory ones.
// ---------------------------------------------------------------------------
// Exclusive scan of count ints held in shared memory into out[0..count] (out[count] =
// total) by the whole block: contiguous chunks per thread, warp and block scans.
__device__ __forceinline__ void block_exclusive_scan(const int* data, int count, int* __restrict__ out) {
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nwarp = (blockDim.x + 31) >> 5;
    const int per = (count + blockDim.x - 1) / blockDim.x;
    const int i0 = tid * per, i1 = min(count, i0 + per);
    int sum = 0;
    for (int i = i0; i < i1; ++i) sum += data[i];
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int z = lane < nwarp ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        wsum[lane] = z;
    }
    __syncthreads();
    int run = (x - sum) + (w > 0 ? wsum[w - 1] : 0);
    for (int i = i0; i < i1; ++i) {
        out[i] = run;
        run += data[i];
    }
    if (tid == 0) out[count] = wsum[nwarp - 1];
}

template <typename R>
__device__ __forceinline__ void k_bin_count_body(Geo g, int N, const R* __restrict__ pos,
                                                   const R* __restrict__ q, int* __restrict__ cnt_blk,
                                                   int* __restrict__ bhist, int* __restrict__ ctile,
                                                   typename V4<R>::T* __restrict__ cpos,
                                                   typename V4<R>::T* __restrict__ cfrac, int* __restrict__ cbase,
                                                   R* __restrict__ Fzero, double* __restrict__ qpart,
                                                   int* __restrict__ ticket, int* __restrict__ boff,
                                                   int* __restrict__ tstart, Blk blk) {
    pdl_enter();
    extern __shared__ int sm_bin[];
    int* hist = sm_bin;                 // [ntiles]
    int* slist = sm_bin + g.ntiles;     // [chunk]
    __shared__ int scount;
    for (int t = threadIdx.x; t < g.ntiles; t += blockDim.x) hist[t] = 0;
    if (threadIdx.x == 0) scount = 0;
    __syncthreads();
    const int b = blk.id, lane = threadIdx.x & 31;
    const int i0 = b * g.chunk;   // the block's region of the compacted arrays
    double s1 = 0.0, s2 = 0.0;
    // the beads, in groups of 32 consecutive ones (one warp's coalesced load),
    // are dealt to the blocks round robin: charged beads that sit together in
    // the input order (chains, counterions, salt) are spread over all blocks
    // (at most chunk / 32 groups per block: chunk is a multiple of 32)
    const int nwarp = blockDim.x >> 5, warp = threadIdx.x >> 5;
    const int ngroups = (N + 31) >> 5;
    for (int gi = b + warp * (int)blk.n; gi < ngroups; gi += nwarp * (int)blk.n) {
        const int i = gi * 32 + lane;
        R qi = (R)0;
        if (i < N) {
            qi = q[i];
            if (Fzero) {
                Fzero[3 * i] = (R)0;
                Fzero[3 * i + 1] = (R)0;
                Fzero[3 * i + 2] = (R)0;
            }
        }
        const bool charged = qi != (R)0;
        const unsigned m = __ballot_sync(0xffffffffu, charged);
        int basei = 0;
        if (lane == 0 && m) basei = atomicAdd(&scount, __popc(m));
        basei = __shfl_sync(0xffffffffu, basei, 0);
        if (charged) slist[basei + __popc(m & ((1u << lane) - 1u))] = i;
    }
    __syncthreads();
    const int nc = scount;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
        if (!ENUF_GUARD(g.check, k < g.chunk, 1)) continue;   // the compacted list holds a chunk
        const int i = slist[k];
        R xw[3], fr[3];
        int bs[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            xw[t] = wrap_r(pos[3 * i + t], g.L, g.xmaxf);
            grid_coord_r(xw[t], g, bs[t], fr[t]);
        }
        const int tile = ((bs[2] / g.T) * g.ntd + bs[1] / g.T) * g.ntd + bs[0] / g.T;
        if (!ENUF_GUARD(g.check, (unsigned)tile < (unsigned)g.ntiles, 0)) continue;
        atomicAdd(&hist[tile], 1);
        const int o = i0 + k;
        typename V4<R>::T a, c;
        a.x = xw[0]; a.y = xw[1]; a.z = xw[2]; a.w = q[i];
        // charge sums over the compacted beads: only the block's first warps
        // hold nonzero partials, the rest skip the reduction tree
        s1 += (double)a.w;
        s2 += (double)a.w * (double)a.w;
        c.x = fr[0]; c.y = fr[1]; c.z = fr[2]; c.w = int_as_real(i, (R)0);
        ctile[o] = tile;
        cpos[o] = a;
        cfrac[o] = c;
        cbase[o] = bs[0] | (bs[1] << 10) | (bs[2] << 20);
    }
    if (threadIdx.x == 0) cnt_blk[b] = nc;
    block_sum2(s1, s2);
    if (threadIdx.x == 0) {
        qpart[2 * b] = s1;
        qpart[2 * b + 1] = s2;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < g.ntiles; t += blockDim.x) bhist[b * g.ntiles + t] = hist[t];
    // the last block to arrive turns the per-block histograms into per-block
    // offsets within each tile and the tile starts (exclusive scan of the totals)
    if (!g.bin_last) return;
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1) == (int)blk.n - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int t = threadIdx.x; t < g.ntiles; t += blockDim.x) {
        int run = 0;
        for (int b0 = 0; b0 < g.nbin; b0 += 8) {   // eight independent loads in flight
            int v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = b0 + u < g.nbin ? __ldcg(&bhist[(b0 + u) * g.ntiles + t]) : 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (b0 + u < g.nbin) boff[(b0 + u) * g.ntiles + t] = run;
                run += v[u];
            }
        }
        hist[t] = run;   // tile totals
    }
    __syncthreads();
    block_exclusive_scan(hist, g.ntiles, tstart);
    if (threadIdx.x == 0) *ticket = 0;
}

template <typename R>
__global__ void __launch_bounds__(1024) k_bin_count(Geo g, int N, const R* __restrict__ pos,
                                                   const R* __restrict__ q, int* __restrict__ cnt_blk,
                                                   int* __restrict__ bhist, int* __restrict__ ctile,
                                                   typename V4<R>::T* __restrict__ cpos,
                                                   typename V4<R>::T* __restrict__ cfrac, int* __restrict__ cbase,
                                                   R* __restrict__ Fzero, double* __restrict__ qpart,
                                                   int* __restrict__ ticket, int* __restrict__ boff,
                                                   int* __restrict__ tstart) {
    k_bin_count_body<R>(g, N, pos, q, cnt_blk, bhist, ctile, cpos, cfrac, cbase, Fzero, qpart, ticket, boff, tstart, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// One thread per tile: offsets of each block's beads inside the tile, and the tile total.

// Exclusive scan of in[0, count) into out[0, count], out[count] = total; one
// CTA of 1024 threads, 16 elements per thread and round (four 16-byte loads).
// aux, when given, receives a copy of out; zero_in clears the input.
static __global__ void __launch_bounds__(1024) k_scan(int* __restrict__ in, int* __restrict__ out, int count,
                                                      int* __restrict__ aux, int zero_in) {
    pdl_enter();
    constexpr int IPT = 16;
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int carry = 0;
    for (int base = 0; base < count; base += 1024 * IPT) {
        const int i0 = base + IPT * tid;
        int v[IPT];
        if (i0 + IPT <= count) {
#pragma unroll
            for (int k = 0; k < IPT; k += 4) {
                const int4 x = *reinterpret_cast<const int4*>(in + i0 + k);
                v[k] = x.x; v[k + 1] = x.y; v[k + 2] = x.z; v[k + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < IPT; ++k) v[k] = i0 + k < count ? in[i0 + k] : 0;
        }
        int sum = 0;
#pragma unroll
        for (int k = 0; k < IPT; ++k) sum += v[k];
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int z = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            wsum[lane] = z;
        }
        __syncthreads();
        int run = carry + (x - sum) + (w > 0 ? wsum[w - 1] : 0);
        const int total = wsum[31];
        if (i0 + IPT <= count) {
#pragma unroll
            for (int k = 0; k < IPT; k += 4) {
                int4 o4;
                o4.x = run; run += v[k];
                o4.y = run; run += v[k + 1];
                o4.z = run; run += v[k + 2];
                o4.w = run; run += v[k + 3];
                *reinterpret_cast<int4*>(out + i0 + k) = o4;
                if (aux) *reinterpret_cast<int4*>(aux + i0 + k) = o4;
                if (zero_in) *reinterpret_cast<int4*>(in + i0 + k) = make_int4(0, 0, 0, 0);
            }
        } else {
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const int idx = i0 + k;
                if (idx < count) {
                    out[idx] = run;
                    if (aux) aux[idx] = run;
                    if (zero_in) in[idx] = 0;
                }
                run += v[k];
            }
        }
        carry += total;
        __syncthreads();
    }
    if (tid == 0) {
        out[count] = carry;
        if (aux) aux[count] = carry;
    }
}

// Exclusive scan of in[0, count) into out[0, count] and aux (out[count] =
// total) by ceil(count / kScanMbSpan) CTAs of 1024 threads, 4 elements per
// thread: every CTA adds up all elements before its own span (16-byte loads)
// and scans its span, so no CTA waits on another (for counts where that
// redundant prefix read stays small; in must be 16-byte aligned and is not
// modified).
constexpr int kScanMbSpan = 4096;
constexpr int kScanMbMax = 16 * kScanMbSpan;
static __global__ void __launch_bounds__(1024) k_scan_mb(const int* __restrict__ in, int* __restrict__ out, int count,
                                                         int* __restrict__ aux) {
    pdl_enter();
    __shared__ int wsum[32];
    __shared__ int spre;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int base = blockIdx.x * kScanMbSpan;
    int pre = 0;
    for (int k = tid; k < base / 4; k += 1024) {
        const int4 x = reinterpret_cast<const int4*>(in)[k];
        pre += x.x + x.y + x.z + x.w;
    }
    pre = __reduce_add_sync(0xffffffffu, pre);
    if (lane == 0) wsum[w] = pre;
    __syncthreads();
    if (w == 0) {
        const int z = __reduce_add_sync(0xffffffffu, wsum[lane]);
        if (lane == 0) spre = z;
    }
    __syncthreads();
    const int i0 = base + 4 * tid;
    int v[4];
    if (i0 + 4 <= count) {
        const int4 x = *reinterpret_cast<const int4*>(in + i0);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = i0 + k < count ? in[i0 + k] : 0;
    }
    const int sum = v[0] + v[1] + v[2] + v[3];
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int z = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        wsum[lane] = z;
    }
    __syncthreads();
    int run = spre + (x - sum) + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (i0 + k < count) {
            out[i0 + k] = run;
            if (aux) aux[i0 + k] = run;
        }
        run += v[k];
    }
    if (tid == 0 && base + kScanMbSpan >= count) {
        out[count] = spre + wsum[31];
        if (aux) aux[count] = spre + wsum[31];
    }
}

// Separate tile offsets for large tile x block counts: one thread per tile
// walks the per-block counts (coalesced) and writes each block's offset inside
// the tile and the tile total (then k_scan gives the tile starts).
static __global__ void __launch_bounds__(256) k_tile_offsets(Geo g, const int* __restrict__ bhist, int* __restrict__ boff,
                                                      int* __restrict__ ttot) {
    pdl_enter();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ntiles) return;
    int run = 0;
    int b = 0;
    for (; b + 4 <= g.nbin; b += 4) {
        const int v0 = bhist[b * g.ntiles + t], v1 = bhist[(b + 1) * g.ntiles + t];
        const int v2 = bhist[(b + 2) * g.ntiles + t], v3 = bhist[(b + 3) * g.ntiles + t];
        boff[b * g.ntiles + t] = run;
        boff[(b + 1) * g.ntiles + t] = run + v0;
        boff[(b + 2) * g.ntiles + t] = run + v0 + v1;
        boff[(b + 3) * g.ntiles + t] = run + v0 + v1 + v2;
        run += v0 + v1 + v2 + v3;
    }
    for (; b < g.nbin; ++b) {
        const int v = bhist[b * g.ntiles + t];
        boff[b * g.ntiles + t] = run;
        run += v;
    }
    ttot[t] = run;
}

template <typename R>
__device__ __forceinline__ void k_bin_scatter_body(Geo g, const int* __restrict__ cnt_blk,
                                                     const int* __restrict__ ctile,
                                                     const typename V4<R>::T* __restrict__ cpos,
                                                     const typename V4<R>::T* __restrict__ cfrac,
                                                     const int* __restrict__ cbase, const int* __restrict__ boff,
                                                     const int* __restrict__ tstart,
                                                     typename V4<R>::T* __restrict__ sq,
                                                     typename V4<R>::T* __restrict__ sw, int* __restrict__ sb, Blk blk) {
    pdl_enter();
    extern __shared__ int cur[];   // [ntiles] running counts
    const int b = blk.id;
    for (int t = threadIdx.x; t < g.ntiles; t += blockDim.x) cur[t] = 0;
    __syncthreads();
    const int nc = cnt_blk[b];
    const int i0 = b * g.chunk;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
        const int o = i0 + k;
        const int t = ctile[o];
        if (!ENUF_GUARD(g.check, (unsigned)t < (unsigned)g.ntiles, 2)) continue;
        const int slot = tstart[t] + boff[b * g.ntiles + t] + atomicAdd(&cur[t], 1);
        if (!ENUF_GUARD(g.check, (unsigned)slot < (unsigned)g.nmax, 2)) continue;
        sq[slot] = cpos[o];
        sw[slot] = cfrac[o];
        sb[slot] = cbase[o];
    }
}

template <typename R>
__global__ void __launch_bounds__(1024) k_bin_scatter(Geo g, const int* __restrict__ cnt_blk,
                                                     const int* __restrict__ ctile,
                                                     const typename V4<R>::T* __restrict__ cpos,
                                                     const typename V4<R>::T* __restrict__ cfrac,
                                                     const int* __restrict__ cbase, const int* __restrict__ boff,
                                                     const int* __restrict__ tstart,
                                                     typename V4<R>::T* __restrict__ sq,
                                                     typename V4<R>::T* __restrict__ sw, int* __restrict__ sb) {
    k_bin_scatter_body<R>(g, cnt_blk, ctile, cpos, cfrac, cbase, boff, tstart, sq, sw, sb, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// Window weights of every sorted charged bead (Eq. 14), computed once and
// read by the spreading and gathering kernels: wb[s][d][a] = psi(u_sd - l_a)
// for the 2p taps a of dimension d. One thread per (bead, dimension) writes
// its 2p consecutive weights (16-byte stores when 2p is a multiple of 4 in
// FP32); all SMs (in FP64 the exponentials run on the FP64 units).
template <typename R>
__device__ __forceinline__ void k_bin_weights_body(Geo g, const int* __restrict__ tstart,
                                                    const typename V4<R>::T* __restrict__ sw, R* __restrict__ wb, Blk blk) {
    pdl_enter();
    const int nq = tstart[g.ntiles];
    const int P2 = 2 * g.p;
    const R rb = (R)g.rb, wn = (R)g.wnorm;
    const int tot = 3 * nq;   // (bead, dimension) pairs; nq <= n_max < 2^29
    for (int e = blk.id * blockDim.x + threadIdx.x; e < tot; e += blk.n * blockDim.x) {
        const int s = e / 3, d = e - 3 * s;
        const typename V4<R>::T fr = sw[s];
        const R f = d == 0 ? fr.x : (d == 1 ? fr.y : fr.z);
        R* out = wb + (size_t)e * P2;   // = wb + (s 3 + d) 2p
        bool done = false;
        if constexpr (sizeof(R) == 4) {
            if ((P2 & 3) == 0) {
                for (int a = 0; a < P2; a += 4) {
                    float w4[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const R u = f + (R)(g.p - 1 - (a + k));
                        w4[k] = wn * r_exp(-u * u * rb);
                    }
                    *reinterpret_cast<float4*>(out + a) = make_float4(w4[0], w4[1], w4[2], w4[3]);
                }
                done = true;
            }
        }
        if (!done) {
            for (int a = 0; a < P2; ++a) {
                const R u = f + (R)(g.p - 1 - a);
                out[a] = wn * r_exp(-u * u * rb);
            }
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_bin_weights(Geo g, const int* __restrict__ tstart,
                                                    const typename V4<R>::T* __restrict__ sw, R* __restrict__ wb) {
    k_bin_weights_body<R>(g, tstart, sw, wb, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// ---------------------------------------------------------------------------
// a2: spreading g(l) = sum_j q_j prod_t psi(u_jt - l_t)   (Eq. 14/19, first half)
// One CTA owns one T^3 tile of the grid: it visits the beads of the (up to)
// 27 neighbouring bins, deposits the taps that fall inside its tile into
// shared memory, and writes the finished tile once. No global atomics.
// ---------------------------------------------------------------------------
constexpr int kSpreadThreads = 256;
constexpr int kMaxTaps = 16;
constexpr int kSpreadCap = 512;   // beads staged in shared memory per round
// Shared slots of the work-item kernel's tile: T^3 rounded up to a multiple of
// 4, so that the regions after it (the int2 work items last) stay 16-byte
// aligned for odd T as well.
__host__ __device__ constexpr int spread_tile_slots(int T) { return (T * T * T + 3) & ~3; }

// Taps of a bead (base b, 2p taps from b - p + 1) that fall in the tile [o, o+T)
// of a periodic grid of n points, as a bit mask over the taps. With at least
// 3 tiles per dimension the window (2p <= 2T) meets tile tb - 1, tb or tb + 1
// of the bead's tile tb in one contiguous run, found arithmetically; otherwise
// the taps are tested one by one.
__device__ __forceinline__ unsigned tap_mask(int b, int o, int T, int n, int ntd, int p) {
    const int P2 = 2 * p;
    if (ntd >= 3) {
        const int tb = b / T, tc = o / T;
        int dt = tc - tb;
        if (dt > 1) dt -= ntd;
        else if (dt < -1) dt += ntd;
        if (dt < -1 || dt > 1) return 0u;
        const int ou = (tb + dt) * T;        // tile origin in the bead's unwrapped frame
        const int l0 = b - p + 1;
        const int a0 = max(0, ou - l0), a1 = min(P2, ou + T - l0);
        if (a1 <= a0) return 0u;
        return ((a1 - a0) >= 32 ? 0xffffffffu : ((1u << (a1 - a0)) - 1u)) << a0;
    }
    unsigned m = 0u;
    for (int a = 0; a < P2; ++a) {
        int l = b - p + 1 + a;
        l = l < 0 ? l + n : (l >= n ? l - n : l);
        if ((unsigned)(l - o) < (unsigned)T) m |= 1u << a;
    }
    return m;
}

// Slots [lo, lo + cnt) of the tile (lines o .. o + T - 1) that hold the taps in
// mask m != 0: contiguous taps on contiguous slots, else (taps or slots wrap
// around a grid of few tiles) the whole tile, whose other slots weigh 0.
__device__ __forceinline__ int tap_slots(unsigned m, int b, int o, int T, int n, int p) {
    const int t0 = __ffs(m) - 1, t1 = 31 - __clz(m), c = __popc(m);
    int s0 = b - p + 1 + t0 - o;   // in (-n - p, n + p)
    s0 += s0 < 0 ? n : 0;
    s0 -= s0 >= n ? n : 0;
    const bool run = c == t1 - t0 + 1 && s0 + c <= T;
    return run ? (s0 | c << 5) : (T << 5);
}

template <typename R>
__global__ void __launch_bounds__(kSpreadThreads, 5) k_spread(Geo g, const int* __restrict__ tstart,
                                                           const typename V4<R>::T* __restrict__ sq,
                                                           const typename V4<R>::T* __restrict__ sw,
                                                           const int* __restrict__ sb,
                                                           R* __restrict__ grid) {
    pdl_enter();
    using V = typename V4<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int T = g.T, T3 = T * T * T;
    constexpr int NW = kSpreadThreads / 32;
    V* stg = reinterpret_cast<V*>(smraw);                          // [cap] (fx, fy, fz, q)
    R* acc = reinterpret_cast<R*>(stg + kSpreadCap);                // [T^3], padded to spread_tile_slots(T)
    R* wts = acc + spread_tile_slots(T);                            // [NW][3][16]
    int* lix = reinterpret_cast<int*>(wts + NW * 3 * kMaxTaps);     // [NW][3][16]
    int* sbase = lix + NW * 3 * kMaxTaps;                           // [cap]
    int2* items = reinterpret_cast<int2*>(sbase + kSpreadCap);      // [cap] (bead | x mask, y mask | z mask)
    __shared__ int nb_start[27], nb_pre[28];
    __shared__ int nnb, nitems;

    const int tile = blockIdx.x;
    const int tx = tile % g.ntd, ty = (tile / g.ntd) % g.ntd, tz = tile / (g.ntd * g.ntd);
    const int o[3] = {tx * T, ty * T, tz * T};
    for (int e = threadIdx.x; e < T3; e += blockDim.x) acc[e] = (R)0;
    const int no = g.ntd >= 3 ? 3 : g.ntd;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {   // neighbouring bins (<= 27): starts and an exclusive prefix of their sizes
        const int cntn = no * no * no;
        int st = 0, c = 0;
        if (lane < cntn) {
            const int dx = lane % no, dy = (lane / no) % no, dz = lane / (no * no);
            const int nz = g.ntd >= 3 ? (tz + dz - 1 + g.ntd) % g.ntd : dz;
            const int ny = g.ntd >= 3 ? (ty + dy - 1 + g.ntd) % g.ntd : dy;
            const int nx = g.ntd >= 3 ? (tx + dx - 1 + g.ntd) % g.ntd : dx;
            const int nt = (nz * g.ntd + ny) * g.ntd + nx;
            st = tstart[nt];
            c = tstart[nt + 1] - st;
        }
        int x = c;
#pragma unroll
        for (int of = 1; of < 32; of <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, of);
            if (lane >= of) x += y;
        }
        if (lane < cntn) {
            nb_start[lane] = st;
            nb_pre[lane] = x - c;
        }
        if (lane == cntn - 1) {
            nb_pre[cntn] = x;
            nnb = cntn;
        }
    }
    __syncthreads();
    R* myw = wts + warp * 3 * kMaxTaps;
    int* myl = lix + warp * 3 * kMaxTaps;
    const int P2 = 2 * g.p;
    const int total = nb_pre[nnb];
    const R rb = (R)g.rb, wn = (R)g.wnorm;
    for (int cb = 0; cb < total; cb += kSpreadCap) {
        const int cn = min(kSpreadCap, total - cb);
        if (threadIdx.x == 0) nitems = 0;
        // stage this round's candidates: one thread per bead, its bin by binary search
        for (int idx = threadIdx.x; idx < cn; idx += blockDim.x) {
            const int f = cb + idx;
            int lo = 0, hi = nnb;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (nb_pre[mid] <= f) lo = mid; else hi = mid;
            }
            const int j = nb_start[lo] + f - nb_pre[lo];
            V v = sw[j];
            v.w = sq[j].w;
            stg[idx] = v;
            sbase[idx] = sb[j];
        }
        __syncthreads();
        // phase A: one lane per candidate; beads whose window meets this tile become work items
        for (int c0 = 0; c0 < cn; c0 += blockDim.x) {
            const int c = c0 + threadIdx.x;
            unsigned mx = 0u, my = 0u, mz = 0u;
            if (c < cn) {
                const int pb = sbase[c];
                mx = tap_mask(pb & 1023, o[0], T, g.n, g.ntd, g.p);
                if (mx) my = tap_mask((pb >> 10) & 1023, o[1], T, g.n, g.ntd, g.p);
                if (my) mz = tap_mask((pb >> 20) & 1023, o[2], T, g.n, g.ntd, g.p);
            }
            const bool keep = mz != 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            int basei = 0;
            if (lane == 0 && bal) basei = atomicAdd(&nitems, __popc(bal));
            basei = __shfl_sync(0xffffffffu, basei, 0);
            if (keep) items[basei + __popc(bal & ((1u << lane) - 1u))] = make_int2(c | (int)(mx << 16), (int)(my | (mz << 16)));
        }
        __syncthreads();
        const int ni = nitems;
        // phase B: one warp per work item
        for (int it = warp; it < ni; it += NW) {
            const int2 e = items[it];
            const int c = e.x & 0xffff;
            const unsigned msk[3] = {(unsigned)e.x >> 16, (unsigned)e.y & 0xffffu, (unsigned)e.y >> 16};
            const V wv = stg[c];
            const int pb = sbase[c];
            if (lane < P2) {
                const int base[3] = {pb & 1023, (pb >> 10) & 1023, (pb >> 20) & 1023};
                const R fr[3] = {wv.x, wv.y, wv.z};
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    if ((msk[t] >> lane) & 1u) {
                        const int slot = __popc(msk[t] & ((1u << lane) - 1u));
                        int l = base[t] - g.p + 1 + lane;
                        l = l < 0 ? l + g.n : (l >= g.n ? l - g.n : l);
                        const R d = fr[t] + (R)(g.p - 1 - lane);
                        myw[t * kMaxTaps + slot] = wn * r_exp(-d * d * rb);
                        myl[t * kMaxTaps + slot] = l - o[t];
                    }
                }
            }
            __syncwarp();
            const int cx = __popc(msk[0]), cy = __popc(msk[1]), cz = __popc(msk[2]);
            const int cxy = cx * cy;
            // xy -> (ix, iy) by a float reciprocal: xy < 256 and the true quotient of
            // xy + 1/2 is at least 1/32 away from an integer, far above the error
            const float icx = 1.0f / (float)cx;
            const R qj = wv.w;
            for (int xy = lane; xy < cxy; xy += 32) {
                const int iy = (int)(((float)xy + 0.5f) * icx);
                const int ix = xy - iy * cx;
                const R wxy = qj * myw[ix] * myw[kMaxTaps + iy];
                const int rowo = myl[kMaxTaps + iy] * T + myl[ix];
                for (int iz = 0; iz < cz; ++iz)
                    atomicAdd(&acc[myl[2 * kMaxTaps + iz] * T * T + rowo], wxy * myw[2 * kMaxTaps + iz]);
            }
            __syncwarp();
        }
        __syncthreads();
    }
    const int n = g.n;
    // write-back, one row of T <= 24 points per warp iteration
    int ly = warp, lz = 0;
    while (ly >= T) { ly -= T; ++lz; }
    while (lz < T) {
        if (lane < T) grid[((size_t)(o[2] + lz) * n + (o[1] + ly)) * n + (o[0] + lane)] = acc[(lz * T + ly) * T + lane];
        ly += NW;
        while (ly >= T) { ly -= T; ++lz; }
    }
}

// Column-stationary spreading for the common tile edges T (template): one CTA
// per T^3 tile; candidates are the charged beads of the 27 neighbouring bins;
// those whose window meets the tile become items; per batch of items the
// per-dimension weights restricted to the tile (T slots each, zero outside
// the item's taps, q folded into z) are laid out in shared memory from the
// per-bead weights; each thread owns one (x, y) column of the tile and adds
// w_x w_y w_z(z) for every item into T registers. No atomics; the tile is
// written once.
constexpr int kColCand = 512;    // candidates staged per round
constexpr int kColItems = 128;   // items per weight batch

//
// SLAB (the FP64 form): the same staging, but the tile is accumulated in
// shared memory and each of the 4 warps owns a slab of z-planes; per item a
// warp whose slab meets the item's z-range spreads the item's footprint
// (its slots in x and y, lanes over the footprint's columns) into its planes.
// The FP64 units are then spent on the item's taps only: the column form
// multiplies every column of the tile by every z-slot, zero or not, and on
// GB300's few FP64 units that was ~4x the instructions.
constexpr int kSlabThreads = 128;
__host__ __device__ constexpr int col_threads(int T) { return T * T <= 128 ? 128 : ((T * T + 31) / 32) * 32; }
template <bool SLAB>
__host__ __device__ constexpr int spread2_threads(int T) { return SLAB ? kSlabThreads : col_threads(T); }

template <typename R>
__host__ __device__ constexpr int col_smem(int T, bool slab = false) {
    return kColCand * (4 + 4 + 8 + (int)sizeof(R)) + kColItems * 3 * T * (int)sizeof(R) +
           (slab ? T * T * T * (int)sizeof(R) : 0);
}

template <typename R, int T, bool SLAB>
__device__ __forceinline__ void k_spread_col_body(Geo g, const int* __restrict__ tstart,
                                                                        const typename V4<R>::T* __restrict__ sq,
                                                                        const int* __restrict__ sb,
                                                                        const R* __restrict__ wb,
                                                                        R* __restrict__ grid, Blk blk) {
    pdl_enter();
    constexpr int NT = spread2_threads<SLAB>(T);
    constexpr int NW = NT / 32;
    constexpr int SZ = (T + NW - 1) / NW;   // SLAB: z-planes per warp
    extern __shared__ __align__(16) unsigned char smraw[];
    R* wt = reinterpret_cast<R*>(smraw);                        // [kColItems][3][T]
    R* cq = wt + kColItems * 3 * T;                             // [kColCand] charges
    int* cslot = reinterpret_cast<int*>(cq + kColCand);         // [kColCand] sorted slots
    int* cbase = cslot + kColCand;                              // [kColCand] packed bases
    int2* items = reinterpret_cast<int2*>(cbase + kColCand);    // [kColCand] (candidate, slot ranges)
    R* acc_s = reinterpret_cast<R*>(items + kColCand);          // SLAB: [T][T][T] tile
    __shared__ int nb_start[27], nb_pre[28];
    __shared__ int nnb, nitems;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blk.id;
    const int tx = tile % g.ntd, ty = (tile / g.ntd) % g.ntd, tz = tile / (g.ntd * g.ntd);
    const int o[3] = {tx * T, ty * T, tz * T};
    const int no = g.ntd >= 3 ? 3 : g.ntd;
    if (warp == 0) {   // neighbouring bins (<= 27): starts and an exclusive prefix of their sizes
        const int cntn = no * no * no;
        int st = 0, c = 0;
        if (lane < cntn) {
            const int dx = lane % no, dy = (lane / no) % no, dz = lane / (no * no);
            const int nz = g.ntd >= 3 ? (tz + dz - 1 + g.ntd) % g.ntd : dz;
            const int ny = g.ntd >= 3 ? (ty + dy - 1 + g.ntd) % g.ntd : dy;
            const int nx = g.ntd >= 3 ? (tx + dx - 1 + g.ntd) % g.ntd : dx;
            const int nt = (nz * g.ntd + ny) * g.ntd + nx;
            st = tstart[nt];
            c = tstart[nt + 1] - st;
        }
        int x = c;
#pragma unroll
        for (int of = 1; of < 32; of <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, of);
            if (lane >= of) x += y;
        }
        if (lane < cntn) {
            nb_start[lane] = st;
            nb_pre[lane] = x - c;
        }
        if (lane == cntn - 1) {
            nb_pre[cntn] = x;
            nnb = cntn;
        }
    }
    __syncthreads();
    const int P2 = 2 * g.p, n = g.n;
    const int cx = tid % T, cy = tid / T;   // this thread's column (tid < T^2)
    const bool owner = !SLAB && tid < T * T;
    R acc[SLAB ? 1 : T];
    const int z0w = warp * SZ, z1w = min(T, z0w + SZ);   // SLAB: this warp's planes
    if constexpr (SLAB) {
        for (int e = z0w * T * T + lane; e < z1w * T * T; e += 32) acc_s[e] = (R)0;
    } else {
#pragma unroll
        for (int z = 0; z < T; ++z) acc[z] = (R)0;
    }
    const int total = nb_pre[nnb];
    for (int cb = 0; cb < total; cb += kColCand) {
        const int cn = min(kColCand, total - cb);
        if (tid == 0) nitems = 0;
        for (int idx = tid; idx < cn; idx += NT) {   // stage: one thread per candidate
            const int f = cb + idx;
            int lo = 0, hi = nnb;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (nb_pre[mid] <= f) lo = mid; else hi = mid;
            }
            const int j = nb_start[lo] + f - nb_pre[lo];
            cslot[idx] = j;
            cbase[idx] = sb[j];
            cq[idx] = sq[j].w;
        }
        __syncthreads();
        for (int c0 = 0; c0 < cn; c0 += NT) {   // items: candidates whose window meets the tile
            const int c = c0 + tid;
            unsigned mx = 0u, my = 0u, mz = 0u;
            if (c < cn) {
                const int pb = cbase[c];
                mx = tap_mask(pb & 1023, o[0], T, n, g.ntd, g.p);
                if (mx) my = tap_mask((pb >> 10) & 1023, o[1], T, n, g.ntd, g.p);
                if (my) mz = tap_mask((pb >> 20) & 1023, o[2], T, n, g.ntd, g.p);
            }
            const bool keep = mz != 0u;
            int rg = 0;   // SLAB: slot ranges (lo | cnt << 5) of x, y, z at bits 0, 10, 20
            if (SLAB && keep) {
                const int pb = cbase[c];
                rg = tap_slots(mx, pb & 1023, o[0], T, n, g.p) | tap_slots(my, (pb >> 10) & 1023, o[1], T, n, g.p) << 10 |
                     tap_slots(mz, (pb >> 20) & 1023, o[2], T, n, g.p) << 20;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            int basei = 0;
            if (lane == 0 && bal) basei = atomicAdd(&nitems, __popc(bal));
            basei = __shfl_sync(0xffffffffu, basei, 0);
            const int at = basei + __popc(bal & ((1u << lane) - 1u));
            if (keep && ENUF_GUARD(g.check, at < kColCand, 3)) items[at] = make_int2(c, rg);
        }
        __syncthreads();
        const int ni = nitems;
        for (int ib = 0; ib < ni; ib += kColItems) {
            const int nb = min(kColItems, ni - ib);
            // weights restricted to the tile: slot s of dimension d holds the weight of the
            // tap on grid line o_d + s, or 0 when that line is outside the item's window
            for (int e = tid; e < nb * 3 * T; e += NT) {
                const int i = e / (3 * T), r = e - i * (3 * T);
                const int d = r / T, sl = r - d * T;
                const int c = items[ib + i].x;
                const int base = (cbase[c] >> (10 * d)) & 1023;
                int a = o[d] + sl - base + g.p - 1;
                if (a < 0) a += n;
                else if (a >= n) a -= n;
                R v = (R)0;
                if (a < P2) v = wb[(size_t)cslot[c] * 3 * P2 + d * P2 + a];
                if (d == 2) v *= cq[c];
                wt[e] = v;
            }
            __syncthreads();
            if constexpr (SLAB) {
                for (int i = 0; i < nb; ++i) {
                    const int rg = items[ib + i].y;
                    const int lz = (rg >> 20) & 31, hz = lz + ((rg >> 25) & 31);
                    const int za = max(lz, z0w), zb = min(hz, z1w);
                    if (za >= zb) continue;   // warp-uniform
                    const int lx = rg & 31, nx = (rg >> 5) & 31, ly = (rg >> 10) & 31, ny = (rg >> 15) & 31;
                    const R* wi = wt + i * 3 * T;
                    // xy -> (ix, iy) by a float reciprocal: xy < 576 and the true quotient of
                    // xy + 1/2 is at least 1/48 away from an integer, far above the error
                    const float inx = 1.0f / (float)nx;
                    for (int xy = lane; xy < nx * ny; xy += 32) {
                        const int iy = (int)(((float)xy + 0.5f) * inx);
                        const int x = lx + xy - iy * nx, y = ly + iy;
                        if (!ENUF_GUARD(g.check, x < T && y < T && zb <= T, 4)) continue;
                        const R w = wi[x] * wi[T + y];
                        R* a = acc_s + y * T + x;
                        for (int z = za; z < zb; ++z) a[z * T * T] += w * wi[2 * T + z];
                    }
                }
            } else if (owner) {
                for (int i = 0; i < nb; ++i) {
                    const R* wi = wt + i * 3 * T;
                    const R w = wi[cx] * wi[T + cy];
                    if (w != (R)0) {
#pragma unroll
                        for (int z = 0; z < T; ++z) acc[z] += w * wi[2 * T + z];
                    }
                }
            }
            __syncthreads();
        }
    }
    if constexpr (SLAB) {   // each warp writes its own planes, rows of T points
        const size_t n2 = (size_t)n * n;
        for (int e = z0w * T * T + lane; e < z1w * T * T; e += 32) {
            const int z = e / (T * T), r = e - z * T * T, y = r / T, x = r - y * T;
            grid[(size_t)(o[2] + z) * n2 + (size_t)(o[1] + y) * n + (o[0] + x)] = acc_s[e];
        }
    } else if (owner) {
        R* col = grid + ((size_t)o[2] * n + (o[1] + cy)) * n + (o[0] + cx);
        const size_t n2 = (size_t)n * n;
#pragma unroll
        for (int z = 0; z < T; ++z) col[z * n2] = acc[z];
    }
}

template <typename R, int T, bool SLAB>
__global__ void __launch_bounds__(spread2_threads<SLAB>(T)) k_spread_col(Geo g, const int* __restrict__ tstart,
                                                                        const typename V4<R>::T* __restrict__ sq,
                                                                        const int* __restrict__ sb,
                                                                        const R* __restrict__ wb,
                                                                        R* __restrict__ grid) {
    k_spread_col_body<R, T, SLAB>(g, tstart, sq, sb, wb, grid, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// ---------------------------------------------------------------------------
// a2, scatter form (FP32; large grids with few beads per grid point). One CTA
// owns a region of RT^3 tiles, edge E = RT T (a template constant), held in
// shared memory. Its candidates are the charged beads of the (RT + 2)^3 bins
// around it: a window of 2p <= T taps reaches no farther than the next tile.
// Warps test 32 candidates at a time against the region and append the beads
// whose window meets it to a shared list; the list is then spread bead by
// bead, a warp per bead: lanes over its (x, y) taps, a loop over the z taps
// inside the region, each product q w_x w_y w_z added to the region. Work is
// spent only on taps that land in the region (the column form multiplies
// every column of its tile by every z slot, which at ~100 grid points per
// charged bead is mostly zeros).
//
// The region accumulates in 32-bit fixed point with native integer shared
// atomics (a float add to shared memory is a compare-and-swap loop): scale
// S = 2^k with S B <= 2^30, B = sum over the region's beads of |q| w_max^3
// bounding every point (w_max = the window's peak, psi(0)). Each term is
// rounded to 1/S: at most B 2^-31 per term, below the float rounding of the
// larger terms; the region is written once, rows of E points as 16-byte
// stores, converted back to float.
// The host admits it when 2p = PT, E is a multiple of T, RT <= 2 divides the
// tiles per dimension ntd >= RT + 2, n % 4 = 0 and n >= 2 (E + T + PT): a
// window's offset from the region origin is then unique modulo n.
// ---------------------------------------------------------------------------
constexpr int kScThreads = 256;
constexpr int kScCap = 1024;   // listed beads per round = candidates per round

// x pitch of the region in shared memory: the 8 x taps x 4 y rows of one
// update land on 32 distinct banks when the pitch is 8 or 24 modulo 32
__host__ __device__ constexpr int sc_pitch(int E) { return (E % 32 == 8 || E % 32 == 24) ? E : sc_pitch(E + 4); }
__host__ __device__ constexpr int sc_smem(int E) { return E * E * sc_pitch(E) * (int)sizeof(int) + kScCap * 16; }

template <int E, int PT>
__global__ void __launch_bounds__(kScThreads) k_spread_sc(Geo g, const int* __restrict__ tstart,
                                                          const float4* __restrict__ sq, const int* __restrict__ sb,
                                                          const float* __restrict__ wb, float* __restrict__ grid) {
    pdl_enter();
    static_assert(E % 4 == 0 && PT >= 2 && PT <= 16, "region edge and window");
    constexpr int EP = sc_pitch(E);
    constexpr int BPR = 32 / PT;               // y taps per round of lanes
    constexpr int NR = (PT + BPR - 1) / BPR;   // rounds
    constexpr int NW = kScThreads / 32;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) int acc[];            // [E][E][EP] fixed point
    int4* items = reinterpret_cast<int4*>(acc + E * E * EP);   // [kScCap] (bead, offsets, q, -)
    __shared__ int nb_start[64], nb_pre[65];
    __shared__ int nitems;
    __shared__ float wsum[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = g.T, RT = E / T, nr = g.ntd / RT;
    const int rx = blockIdx.x % nr, ry = (blockIdx.x / nr) % nr, rz = blockIdx.x / (nr * nr);
    const int ox = rx * E, oy = ry * E, oz = rz * E;
    for (int e = tid; e < E * E * EP / 4; e += kScThreads) reinterpret_cast<int4*>(acc)[e] = make_int4(0, 0, 0, 0);
    const int nbd = RT + 2, nbins = nbd * nbd * nbd;   // <= 64
    if (warp == 0) {   // the bins, their bead ranges and an exclusive prefix of their sizes
        int run = 0;
        for (int k0 = 0; k0 < nbins; k0 += 32) {
            const int k = k0 + lane;
            int st = 0, cnt = 0;
            if (k < nbins) {
                const int dx = k % nbd, dy = (k / nbd) % nbd, dz = k / (nbd * nbd);
                const int bx = (rx * RT + dx - 1 + g.ntd) % g.ntd;
                const int by = (ry * RT + dy - 1 + g.ntd) % g.ntd;
                const int bz = (rz * RT + dz - 1 + g.ntd) % g.ntd;
                const int t = (bz * g.ntd + by) * g.ntd + bx;
                st = tstart[t];
                cnt = tstart[t + 1] - st;
            }
            int x = cnt;
#pragma unroll
            for (int of = 1; of < 32; of <<= 1) {
                const int y = __shfl_up_sync(FULL, x, of);
                if (lane >= of) x += y;
            }
            if (k < nbins) {
                nb_start[k] = st;
                nb_pre[k] = run + x - cnt;
            }
            run += __shfl_sync(FULL, x, 31);
        }
        if (lane == 0) {
            nb_pre[nbins] = run;
            nitems = 0;
        }
    }
    __syncthreads();
    const int p = g.p, n = g.n, hn = n >> 1;
    const int total = nb_pre[nbins];
    // Candidates [f0, f1) of the bins' concatenation, 32 per warp step: the beads
    // whose window meets the region, appended to the list (list) and/or their
    // |q| summed.
    auto scan = [&](int f0, int f1, bool list, float& qsum) {
        for (int fb = f0 + 32 * warp; fb < f1; fb += 32 * NW) {
            const int f = fb + lane;
            bool hit = false;
            int pk = 0, j = 0;
            if (f < f1) {
                // its bin: the last k with nb_pre[k] <= f (a non-empty bin)
                int k = 0;
#pragma unroll
                for (int st = 32; st > 0; st >>= 1)
                    if (k + st < nbins && nb_pre[k + st] <= f) k += st;
                j = nb_start[k] + f - nb_pre[k];
                const int pb = sb[j];
                int d0 = (pb & 1023) - p + 1 - ox, d1 = ((pb >> 10) & 1023) - p + 1 - oy;
                int d2 = ((pb >> 20) & 1023) - p + 1 - oz;
                d0 += d0 < -hn ? n : (d0 >= hn ? -n : 0);
                d1 += d1 < -hn ? n : (d1 >= hn ? -n : 0);
                d2 += d2 < -hn ? n : (d2 >= hn ? -n : 0);
                hit = d0 > -PT && d0 < E && d1 > -PT && d1 < E && d2 > -PT && d2 < E;
                pk = (d0 + PT) | (d1 + PT) << 8 | (d2 + PT) << 16;   // each in [1, E + PT) < 256
            }
            const float qj = hit ? sq[j].w : 0.f;
            qsum += fabsf(qj);
            if (list) {
                const unsigned m = __ballot_sync(FULL, hit);
                int at = 0;
                if (lane == 0 && m) at = atomicAdd(&nitems, __popc(m));
                at = __shfl_sync(FULL, at, 0) + __popc(m & ((1u << lane) - 1u));
                if (hit) items[at] = make_int4(j, pk, __float_as_int(qj), 0);
            }
        }
    };
    // Spread the listed beads, q pre-multiplied by the scale S.
    auto spread = [&](float S) {
        const int a = lane % PT, b = lane / PT;
        const bool lane_on = lane < BPR * PT;
        const int ni = nitems;
        for (int it = warp; it < ni; it += NW) {
            const int4 rec = items[it];
            const int dx = (rec.y & 255) - PT, dy = ((rec.y >> 8) & 255) - PT, dz = (rec.y >> 16) - PT;
            const float w = lane < 3 * PT ? wb[(size_t)rec.x * (3 * PT) + lane] : 0.f;   // x, y, z taps
            const float wxq = __shfl_sync(FULL, w, a) * (__int_as_float(rec.z) * S);
            const int x = dx + a;
            const bool vx = lane_on && (unsigned)x < (unsigned)E;
            float wxy[NR];
            int i0[NR];
            bool v[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int bb = b + r * BPR;
                const float wy = __shfl_sync(FULL, w, PT + (bb < PT ? bb : PT - 1));
                const int y = dy + bb;
                v[r] = vx && bb < PT && (unsigned)y < (unsigned)E;
                wxy[r] = wxq * wy;
                i0[r] = (dz * E + y) * EP + x;
            }
            const int clo = max(0, -dz), chi = min(PT, E - dz);   // z taps inside the region
#pragma unroll
            for (int r = 0; r < NR; ++r) i0[r] += clo * E * EP;
            for (int c = clo; c < chi; ++c) {
                const float wzc = __shfl_sync(FULL, w, 2 * PT + c);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (v[r]) atomicAdd(&acc[i0[r]], __float2int_rn(wxy[r] * wzc));
                    i0[r] += E * EP;
                }
            }
        }
    };
    // the scale from the sum of |q| over the region's beads: in the listing pass
    // when all candidates fit one round, else from a pass of its own
    const bool one_round = total <= kScCap;
    float qs = 0.f;
    scan(0, total, one_round, qs);
#pragma unroll
    for (int of = 16; of > 0; of >>= 1) qs += __shfl_xor_sync(FULL, qs, of);
    if (lane == 0) wsum[warp] = qs;
    __syncthreads();
    float B = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) B += wsum[w];
    const float wm = (float)g.wnorm;
    B *= wm * wm * wm;
    int ex = 0;
    frexpf(B, &ex);                                   // B < 2^ex
    const float S = B > 0.f ? ldexpf(1.f, min(126, 30 - ex)) : 1.f;   // S B < 2^30
    if (one_round) {
        spread(S);
    } else {
        for (int f0 = 0; f0 < total; f0 += kScCap) {
            __syncthreads();
            if (tid == 0) nitems = 0;
            __syncthreads();
            float dummy = 0.f;
            scan(f0, min(total, f0 + kScCap), true, dummy);
            __syncthreads();
            spread(S);
        }
    }
    __syncthreads();
    const float iS = 1.f / S;   // a power of two: exact
    constexpr int Q = E / 4;    // 16-byte pieces per row
    for (int e = tid; e < E * E * Q; e += kScThreads) {
        const int row = e / Q, cq = e - row * Q;
        const int z = row / E, y = row - z * E;
        const int4 v = *reinterpret_cast<const int4*>(acc + (z * E + y) * EP + 4 * cq);
        *reinterpret_cast<float4*>(grid + ((size_t)(oz + z) * n + (oy + y)) * n + ox + 4 * cq) =
            make_float4((float)v.x * iS, (float)v.y * iS, (float)v.z * iS, (float)v.w * iS);
    }
}

// ---------------------------------------------------------------------------
// a3: forward FFT pass along x (R2C, two real rows per complex line), keep
// k_x = 0..nc; output spec1[z][kx][y].
// ---------------------------------------------------------------------------
template <typename R, bool CR = false>
__global__ void __launch_bounds__(256) k_fft_x(Geo g, FftPlanDev fp, const R* __restrict__ grid,
                                              const typename Cx<R>::T* __restrict__ twg,
                                              typename Cx<R>::T* __restrict__ spec1, int LP) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc1 = g.nc + 1;
    C* tw = reinterpret_cast<C*>(smraw);
    const int ls = line_stride<C>(n);   // padded, swizzled lines (the split reads across lines)
    C* b0 = tw + n;
    C* b1 = b0 + LP * ls;
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const float rn = 1.0f / (float)n;
    const int row0 = blockIdx.x * 2 * LP;     // first real row (z*n + y), y even
    const int nrows = n * n;
    const int nl = min(LP, (nrows - row0) / 2);
    const float rnl = 1.0f / (float)max(nl, 1);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int c = qdiv(idx, n, rn), x = idx - c * n;
        C v;
        v.x = grid[(size_t)(row0 + 2 * c) * n + x];
        v.y = grid[(size_t)(row0 + 2 * c + 1) * n + x];
        b0[c * ls + swz<C>(x)] = v;
    }
    __syncthreads();
    C* res = fft_lines<R, false, CR>(b0, b1, tw, fp, nl, ls);
    // split the two real transforms: A = (Z_k + conj Z_{n-k})/2, B = -i (Z_k - conj Z_{n-k})/2
    for (int idx = threadIdx.x; idx < nl * nc1; idx += blockDim.x) {
        const int k = qdiv(idx, nl, rnl), c = idx - k * nl;
        const C z = res[c * ls + swz<C>(k)];
        const C zm = res[c * ls + swz<C>(k == 0 ? 0 : n - k)];
        C A, B;
        A.x = (R)0.5 * (z.x + zm.x);
        A.y = (R)0.5 * (z.y - zm.y);
        B.x = (R)0.5 * (z.y + zm.y);
        B.y = (R)0.5 * (zm.x - z.x);
        const int row = row0 + 2 * c;
        const int zz = qdiv(row, n, rn), y = row - zz * n;
        C* dst = spec1 + ((size_t)zz * nc1 + k) * n + y;
        dst[0] = A;
        dst[1] = B;
    }
}

// forward pass along y for lines (z, kx), keep |ky| <= nc; output spec2[kx][ky][z]
template <typename R, bool CR = false>
__global__ void __launch_bounds__(256) k_fft_y(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec1,
                                              const typename Cx<R>::T* __restrict__ twg,
                                              typename Cx<R>::T* __restrict__ spec2, int LB) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc1 = g.nc + 1, K = g.K;
    C* tw = reinterpret_cast<C*>(smraw);
    const int ls = line_stride<C>(n);   // padded, swizzled lines (the output reads across lines)
    C* b0 = tw + n;
    C* b1 = b0 + LB * ls;
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const float rn = 1.0f / (float)n;
    const int kx = blockIdx.x;
    const int z0 = blockIdx.y * LB;
    const int nl = min(LB, n - z0);
    const float rnl = 1.0f / (float)max(nl, 1);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int c = qdiv(idx, n, rn), y = idx - c * n;
        b0[c * ls + swz<C>(y)] = spec1[((size_t)(z0 + c) * nc1 + kx) * n + y];
    }
    __syncthreads();
    C* res = fft_lines<R, false, CR>(b0, b1, tw, fp, nl, ls);
    for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
        const int ki = qdiv(idx, nl, rnl), c = idx - ki * nl;
        const int ky = ki - g.nc;
        spec2[((size_t)kx * K + ki) * n + z0 + c] = res[c * ls + swz<C>(ky < 0 ? ky + n : ky)];
    }
}

// z pass: forward z; E += w D |F|^2, W += w D v |F|^2 (FP64, Kahan); the
// fields G_a = -i k_a D F (a = x, y, z; Eq. 24) or, in gradient mode, the one
// field G = D F; all fields of the CTA's lines inverse-transformed together;
// output spec3[a][z][kx][ky].
template <typename R, bool CR = false>
__global__ void __launch_bounds__(256) k_fft_z(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec2,
                                              const typename Cx<R>::T* __restrict__ twg,
                                              const double* __restrict__ tab, const double* __restrict__ tabv,
                                              const R* __restrict__ tabr, typename Cx<R>::T* __restrict__ spec3,
                                              double* __restrict__ epart, int LB, int plane_major) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, K = g.K, nf = g.nf;
    const int NL = (nc + 1) * K;
    const float rK = 1.0f / (float)K, rn = 1.0f / (float)n;
    C* tw = reinterpret_cast<C*>(smraw);
    const int ls = line_stride<C>(n);   // padded, swizzled lines (loads and stores go across lines)
    C* b0 = tw + n;               // [LB][ls] forward lines
    C* b1 = b0 + LB * ls;         // [LB][ls] scratch
    C* X = b1 + LB * ls;          // [nf][LB][ls] fields
    C* Y = X + nf * LB * ls;      // [nf][LB][ls] scratch
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const int l0 = blockIdx.x * LB;
    const int nl = min(LB, NL - l0);
    const float rnl = 1.0f / (float)max(nl, 1);
    if (plane_major) {   // spec2[z][l]: lines gathered across planes
        for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
            const int z = qdiv(idx, nl, rnl), c = idx - z * nl;
            b0[c * ls + swz<C>(z)] = spec2[(size_t)z * NL + l0 + c];
        }
    } else {             // spec2[l][z]: lines contiguous
        for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
            const int c = qdiv(idx, n, rn), z = idx - c * n;
            b0[c * ls + swz<C>(z)] = spec2[(size_t)l0 * n + idx];
        }
    }
    __syncthreads();
    C* Fh = fft_lines<R, false, CR>(b0, b1, tw, fp, nl, ls);
    // energy and virial of the kept modes (half space kx >= 0, kx > 0 counted twice)
    Kahan ke, kw;
    for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
        const int c = qdiv(idx, K, rK), kzi = idx - c * K;
        const int l = l0 + c;
        const int kx = qdiv(l, K, rK);
        const int kz = kzi - nc;
        const C f = Fh[c * ls + swz<C>(kz < 0 ? kz + n : kz)];
        const double a2 = (double)f.x * (double)f.x + (double)f.y * (double)f.y;
        const double wgt = kx == 0 ? 1.0 : 2.0;
        ke.add(wgt * tab[(size_t)l * K + kzi] * a2);
        kw.add(wgt * tabv[(size_t)l * K + kzi] * a2);
    }
    double se = ke.s, sv = kw.s;
    block_sum2(se, sv);
    if (threadIdx.x == 0) {
        epart[2 * blockIdx.x] = se;
        epart[2 * blockIdx.x + 1] = sv;
    }
    // fields: line a * nl + c of X
    const int per = nl * n;
    const float rper = 1.0f / (float)per;
    for (int idx = threadIdx.x; idx < nf * per; idx += blockDim.x) {
        const int a = qdiv(idx, per, rper), e = idx - a * per;
        const int c = qdiv(e, n, rn), m = e - c * n;
        const int kz = m <= n / 2 ? m : m - n;
        C v;
        v.x = (R)0;
        v.y = (R)0;
        if (kz >= -nc && kz <= nc) {
            const int l = l0 + c;
            const R d = tabr[(size_t)l * K + (kz + nc)];
            const C f = Fh[c * ls + swz<C>(m)];
            if (nf == 1) {
                v.x = d * f.x;     // D F
                v.y = d * f.y;
            } else {
                const int kx = qdiv(l, K, rK), ky = (l - kx * K) - nc;
                const int ka = a == 0 ? kx : (a == 1 ? ky : kz);
                const R s = (R)ka * d;
                v.x = s * f.y;     // -i k_a D F
                v.y = -s * f.x;
            }
        }
        X[(a * nl + c) * ls + swz<C>(m)] = v;
    }
    __syncthreads();
    C* res = fft_lines<R, true, CR>(X, Y, tw, fp, nf * nl, ls);
    for (int idx = threadIdx.x; idx < nf * per; idx += blockDim.x) {
        const int a = qdiv(idx, per, rper), e = idx - a * per;
        const int z = qdiv(e, nl, rnl), c = e - z * nl;
        spec3[((size_t)a * n + z) * NL + l0 + c] = res[(a * nl + c) * ls + swz<C>(z)];
    }
}

// Forward x and y passes of one z-plane in shared memory (small grids): the
// n real rows as n/2 complex lines (two rows each), FFT along x, split into
// the two half spectra kx = 0..nc, FFT of the nc + 1 columns along y, keep
// |ky| <= nc; output spec2[z][kx][ky] (plane-major).
template <typename R, bool CR = false>
__global__ void __launch_bounds__(512) k_fft_xy(Geo g, FftPlanDev fp, const R* __restrict__ grid,
                                               const typename Cx<R>::T* __restrict__ twg,
                                               typename Cx<R>::T* __restrict__ spec2) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1, K = g.K, h = n / 2;
    const float rn = 1.0f / (float)n, rh = 1.0f / (float)h, rK = 1.0f / (float)K;
    C* tw = reinterpret_cast<C*>(smraw);
    const int ls = line_stride<C>(n);   // padded, swizzled lines
    C* L0 = tw + n;        // [n/2][ls]
    C* L1 = L0 + h * ls;   // [n/2][ls]
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const int z = blockIdx.x;
    const R* gz = grid + (size_t)z * n * n;
    for (int idx = threadIdx.x; idx < h * n; idx += blockDim.x) {
        const int c = qdiv(idx, n, rn), x = idx - c * n;
        C v;
        v.x = gz[(size_t)(2 * c) * n + x];
        v.y = gz[(size_t)(2 * c + 1) * n + x];
        L0[c * ls + swz<C>(x)] = v;
    }
    __syncthreads();
    C* X = fft_lines<R, false, CR>(L0, L1, tw, fp, h, ls);
    C* P = X == L0 ? L1 : L0;   // [nc+1][ls] columns over y, then scratch
    C* S = P + nc1 * ls;        // 2 (nc + 1) = n/2: P and S fill the other buffer
    // split the two real transforms: A = (Z_k + conj Z_{n-k})/2, B = -i (Z_k - conj Z_{n-k})/2
    for (int idx = threadIdx.x; idx < nc1 * h; idx += blockDim.x) {
        const int k = qdiv(idx, h, rh), c = idx - k * h;
        const C zk = X[c * ls + swz<C>(k)];
        const C zm = X[c * ls + swz<C>(k == 0 ? 0 : n - k)];
        C A, B;
        A.x = (R)0.5 * (zk.x + zm.x);
        A.y = (R)0.5 * (zk.y - zm.y);
        B.x = (R)0.5 * (zk.y + zm.y);
        B.y = (R)0.5 * (zm.x - zk.x);
        P[k * ls + swz<C>(2 * c)] = A;
        P[k * ls + swz<C>(2 * c + 1)] = B;
    }
    __syncthreads();
    C* Y = fft_lines<R, false, CR>(P, S, tw, fp, nc1, ls);
    C* out = spec2 + (size_t)z * nc1 * K;
    for (int idx = threadIdx.x; idx < nc1 * K; idx += blockDim.x) {
        const int kx = qdiv(idx, K, rK), ki = idx - kx * K;
        const int ky = ki - nc;
        out[idx] = Y[kx * ls + swz<C>(ky < 0 ? ky + n : ky)];
    }
}

// Inverse y and x passes of one (field, z-plane) in shared memory (small
// grids): the plane spec3[a][z][kx][ky], zero-padded to n along y, inverse
// FFT of the nc + 1 columns, then two Hermitian rows per complex line
// (C2R) inverse along x; output h[a][z][y][x].
template <typename R, bool CR = false>
__global__ void __launch_bounds__(512) k_fft_yx(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec3,
                                               const typename Cx<R>::T* __restrict__ twg, R* __restrict__ h) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1, K = g.K, hn = n / 2;
    const float rn = 1.0f / (float)n;
    C* tw = reinterpret_cast<C*>(smraw);
    const int ls = line_stride<C>(n);   // padded, swizzled lines
    C* L0 = tw + n;         // [n/2][ls]: the nc + 1 columns and their scratch
    C* L1 = L0 + hn * ls;   // [n/2][ls]: the x lines
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const int az = blockIdx.x;   // a * n + z
    const C* in = spec3 + (size_t)az * nc1 * K;
    C* P = L0;                   // [nc+1][ls] columns over y
    C* S = L0 + nc1 * ls;
    for (int idx = threadIdx.x; idx < nc1 * n; idx += blockDim.x) {
        const int kx = qdiv(idx, n, rn), m = idx - kx * n;
        const int ky = m <= n / 2 ? m : m - n;
        C v;
        v.x = (R)0;
        v.y = (R)0;
        if (ky >= -nc && ky <= nc) v = in[kx * K + (ky + nc)];
        P[kx * ls + swz<C>(m)] = v;
    }
    __syncthreads();
    C* Yc = fft_lines<R, true, CR>(P, S, tw, fp, nc1, ls);   // [kx][y], in L0
    // x lines: row pair (2c, 2c+1) as A + i B with the Hermitian extension
    for (int idx = threadIdx.x; idx < hn * n; idx += blockDim.x) {
        const int c = qdiv(idx, n, rn), m = idx - c * n;
        C a, b;
        a.x = a.y = b.x = b.y = (R)0;
        if (m == 0) {
            a.x = Yc[swz<C>(2 * c)].x;
            b.x = Yc[swz<C>(2 * c + 1)].x;
        } else if (m <= nc) {
            a = Yc[m * ls + swz<C>(2 * c)];
            b = Yc[m * ls + swz<C>(2 * c + 1)];
        } else if (m >= n - nc) {
            a = Yc[(n - m) * ls + swz<C>(2 * c)];
            a.y = -a.y;
            b = Yc[(n - m) * ls + swz<C>(2 * c + 1)];
            b.y = -b.y;
        }
        C zz;
        zz.x = a.x - b.y;   // A + i B
        zz.y = a.y + b.x;
        L1[c * ls + swz<C>(m)] = zz;
    }
    __syncthreads();
    C* Xr = fft_lines<R, true, CR>(L1, L0, tw, fp, hn, ls);
    R* out = h + (size_t)az * n * n;
    for (int idx = threadIdx.x; idx < hn * n; idx += blockDim.x) {
        const int c = qdiv(idx, n, rn), x = idx - c * n;
        const C v = Xr[c * ls + swz<C>(x)];
        out[(size_t)(2 * c) * n + x] = v.x;
        out[(size_t)(2 * c + 1) * n + x] = v.y;
    }
}

// inverse pass along y for lines (a, z, kx): K inputs zero-padded to n; output spec4[a][z][y][kx]
template <typename R, bool CR = false>
__global__ void __launch_bounds__(256) k_fft_iy(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec3,
                                               const typename Cx<R>::T* __restrict__ twg,
                                               typename Cx<R>::T* __restrict__ spec4, int LB) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1, K = g.K;
    const int NLT = g.nf * n * nc1;
    const float rnc1 = 1.0f / (float)nc1;
    C* tw = reinterpret_cast<C*>(smraw);
    const int ls = line_stride<C>(n);   // padded, swizzled lines (the output reads across lines)
    C* b0 = tw + n;
    C* b1 = b0 + LB * ls;
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const float rn = 1.0f / (float)n;
    const int l0 = blockIdx.x * LB;
    const int nl = min(LB, NLT - l0);
    const float rnl = 1.0f / (float)max(nl, 1);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int c = qdiv(idx, n, rn), m = idx - c * n;
        const int ky = m <= n / 2 ? m : m - n;
        C v;
        v.x = (R)0;
        v.y = (R)0;
        if (ky >= -nc && ky <= nc) v = spec3[(size_t)(l0 + c) * K + (ky + nc)];
        b0[c * ls + swz<C>(m)] = v;
    }
    __syncthreads();
    C* res = fft_lines<R, true, CR>(b0, b1, tw, fp, nl, ls);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int y = qdiv(idx, nl, rnl), c = idx - y * nl;
        const int l = l0 + c;
        const int az = qdiv(l, nc1, rnc1), kx = l - az * nc1;
        spec4[((size_t)az * n + y) * nc1 + kx] = res[c * ls + swz<C>(y)];
    }
}

// inverse pass along x (C2R, two Hermitian rows per complex line); output h[a][z][y][x]
template <typename R, bool CR = false>
__global__ void __launch_bounds__(256) k_fft_ix(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec4,
                                               const typename Cx<R>::T* __restrict__ twg,
                                               R* __restrict__ h, int LP) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1;
    const int nrows = g.nf * n * n;
    C* tw = reinterpret_cast<C*>(smraw);
    const int ls = line_stride<C>(n);   // swizzled lines
    C* b0 = tw + n;
    C* b1 = b0 + LP * ls;
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const float rn = 1.0f / (float)n;
    const int row0 = blockIdx.x * 2 * LP;
    const int nl = min(LP, (nrows - row0) / 2);
    const float rnl = 1.0f / (float)max(nl, 1);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int c = qdiv(idx, n, rn), m = idx - c * n;
        const C* A = spec4 + (size_t)(row0 + 2 * c) * nc1;
        const C* B = A + nc1;
        C a, b;
        a.x = a.y = b.x = b.y = (R)0;
        if (m == 0) {
            a.x = A[0].x;
            b.x = B[0].x;
        } else if (m <= nc) {
            a = A[m];
            b = B[m];
        } else if (m >= n - nc) {
            a = A[n - m];
            a.y = -a.y;
            b = B[n - m];
            b.y = -b.y;
        }
        C z;
        z.x = a.x - b.y;   // A + i B
        z.y = a.y + b.x;
        b0[c * ls + swz<C>(m)] = z;
    }
    __syncthreads();
    C* res = fft_lines<R, true, CR>(b0, b1, tw, fp, nl, ls);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int c = qdiv(idx, n, rn), x = idx - c * n;
        const C v = res[c * ls + swz<C>(x)];
        h[(size_t)(row0 + 2 * c) * n + x] = v.x;
        h[(size_t)(row0 + 2 * c + 1) * n + x] = v.y;
    }
}

// ---------------------------------------------------------------------------
// a6: gather (conjugated NFFT part 2, Eq. 25). Warp per charged bead.
// ---------------------------------------------------------------------------
constexpr int kGatherThreads = 256;

// PT > 0: the window's tap count 2p fixed at compile time. The tap loops are
// then unrolled: the z taps' offsets and weights sit in registers and the
// 3 x 2p loads of a column are all in flight at once (the runtime-count loop
// waits on each tap's loads before the next: at 3M beads the gather was
// bound by that latency, not by DRAM).
template <typename R, int PT = 0>
__device__ __forceinline__ void k_gather_body(Geo g, const int* __restrict__ tstart,
                                                           const typename V4<R>::T* __restrict__ sq,
                                                           const typename V4<R>::T* __restrict__ sw,
                                                           const int* __restrict__ sb, const R* __restrict__ wb,
                                                           const R* __restrict__ h, R* __restrict__ F,
                                                           TotalsArgs tot, Blk blk) {
    pdl_enter();
    constexpr int NW = kGatherThreads / 32;
    __shared__ R wts[NW][3][kMaxTaps];
    __shared__ R dwts[NW][3][kMaxTaps];   // gradient mode: psi'(d) = -(2 d / b) psi(d)
    __shared__ int lix[NW][3][kMaxTaps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Nq = tstart[g.ntiles];
    const int n = g.n;
    const size_t n3 = (size_t)n * n * n;   // n <= 1024: one grid's offsets fit an int
    const R* __restrict__ h0 = h;
    const R* __restrict__ h1 = g.nf == 3 ? h + n3 : h;
    const R* __restrict__ h2 = g.nf == 3 ? h + 2 * n3 : h;
    const int P2 = 2 * g.p;
    const float iP2 = 1.0f / (float)P2;
    const R rb = (R)g.rb, wn = (R)g.wnorm;
    const R pref = (R)g.pref;
    const bool grad = g.nf == 1;
    // the whole grid sweeps the tile-sorted beads in order (bead s by warp s mod
    // the grid's warps): the fields' working set at any moment is a band of
    // neighbouring tiles, which stays in L2 (measured: giving each block a
    // contiguous run instead spread the working set over the whole grid and
    // read 2.4x the DRAM bytes at 3M beads)
    for (int s = blk.id * NW + warp; s < Nq; s += blk.n * NW) {
        const typename V4<R>::T wv = sw[s];
        const R qs = sq[s].w;
        const int pb = sb[s];
        if (lane < P2) {
            const int base[3] = {pb & 1023, (pb >> 10) & 1023, (pb >> 20) & 1023};
            const R fr[3] = {wv.x, wv.y, wv.z};
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                int l = base[t] - g.p + 1 + lane;
                l = l < 0 ? l + n : (l >= n ? l - n : l);
                lix[warp][t][lane] = t == 2 ? l * n * n : l;
                const R d = fr[t] + (R)(g.p - 1 - lane);   // n x - l
                const R w = wb ? wb[(size_t)s * 3 * P2 + t * P2 + lane] : wn * r_exp(-d * d * rb);
                wts[warp][t][lane] = w;
                if (grad) dwts[warp][t][lane] = (R)-2 * d * rb * w;
            }
        }
        __syncwarp();
        R ax = 0, ay = 0, az = 0;
        // lanes over the (x, y) taps, the z taps summed first and weighted by
        // the column's x-y weight once; ab -> (a, b) by a float reciprocal
        // (ab < 256, so the quotient of ab + 1/2 is 1/32 from an integer)
        if constexpr (PT > 0) {
            constexpr int NAB = PT * PT;
            constexpr int NRD = (NAB + 31) / 32;   // rounds of lanes over the (x, y) taps
            R wz[PT], dz[PT];
            int oz[PT];
#pragma unroll
            for (int c = 0; c < PT; ++c) {
                wz[c] = wts[warp][2][c];
                dz[c] = grad ? dwts[warp][2][c] : (R)0;
                oz[c] = lix[warp][2][c];
            }
            if (!grad && NRD <= 2) {
                // three fields, at most two rounds: every round's loads issued before
                // the sums (6 p loads in flight per lane)
                R hv[NRD][3][PT];
                bool on[NRD];
#pragma unroll
                for (int r = 0; r < NRD; ++r) {
                    const int ab = lane + 32 * r;
                    on[r] = NAB % 32 == 0 || ab < NAB;
                    const int b = on[r] ? ab / PT : 0, a = on[r] ? ab - b * PT : 0;
                    const int rowo = lix[warp][1][b] * n + lix[warp][0][a];
#pragma unroll
                    for (int c = 0; c < PT; ++c) {
                        int off = oz[c] + rowo;
                        if (!ENUF_GUARD(g.check, (size_t)off < n3, 5)) off = 0;
                        hv[r][0][c] = on[r] ? h0[off] : (R)0;
                        hv[r][1][c] = on[r] ? h1[off] : (R)0;
                        hv[r][2][c] = on[r] ? h2[off] : (R)0;
                    }
                }
#pragma unroll
                for (int r = 0; r < NRD; ++r) {
                    const int ab = lane + 32 * r;
                    const int b = on[r] ? ab / PT : 0, a = on[r] ? ab - b * PT : 0;
                    R s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
                    for (int c = 0; c < PT; ++c) {
                        s0 = fma(wz[c], hv[r][0][c], s0);
                        s1 = fma(wz[c], hv[r][1][c], s1);
                        s2 = fma(wz[c], hv[r][2][c], s2);
                    }
                    const R wab = on[r] ? wts[warp][0][a] * wts[warp][1][b] : (R)0;
                    ax = fma(wab, s0, ax);
                    ay = fma(wab, s1, ay);
                    az = fma(wab, s2, az);
                }
            } else {
#pragma unroll
                for (int r = 0; r < NRD; ++r) {
                    const int ab = lane + 32 * r;
                    if (NAB % 32 != 0 && ab >= NAB) break;
                    const int b = ab / PT, a = ab - b * PT;
                    const int rowo = lix[warp][1][b] * n + lix[warp][0][a];
                    const R wx = wts[warp][0][a], wy = wts[warp][1][b];
                    if (grad) {   // one field: sum_l grad Psi(n x - l) h(l)
                        R hv[PT];
#pragma unroll
                        for (int c = 0; c < PT; ++c) {
                            const int off = oz[c] + rowo;
                            hv[c] = ENUF_GUARD(g.check, (size_t)off < n3, 5) ? h0[off] : (R)0;
                        }
                        R s0 = 0, s1 = 0;
#pragma unroll
                        for (int c = 0; c < PT; ++c) {
                            s0 = fma(wz[c], hv[c], s0);
                            s1 = fma(dz[c], hv[c], s1);
                        }
                        ax = fma(dwts[warp][0][a] * wy, s0, ax);
                        ay = fma(wx * dwts[warp][1][b], s0, ay);
                        az = fma(wx * wy, s1, az);
                    } else {
                        R h0v[PT], h1v[PT], h2v[PT];
#pragma unroll
                        for (int c = 0; c < PT; ++c) {
                            int off = oz[c] + rowo;
                            if (!ENUF_GUARD(g.check, (size_t)off < n3, 5)) off = 0;
                            h0v[c] = h0[off];
                            h1v[c] = h1[off];
                            h2v[c] = h2[off];
                        }
                        R s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
                        for (int c = 0; c < PT; ++c) {
                            s0 = fma(wz[c], h0v[c], s0);
                            s1 = fma(wz[c], h1v[c], s1);
                            s2 = fma(wz[c], h2v[c], s2);
                        }
                        const R wab = wx * wy;
                        ax = fma(wab, s0, ax);
                        ay = fma(wab, s1, ay);
                        az = fma(wab, s2, az);
                    }
                }
            }
        } else if (grad) {   // one field: sum_l grad Psi(n x - l) h(l)
            for (int ab = lane; ab < P2 * P2; ab += 32) {
                const int b = (int)(((float)ab + 0.5f) * iP2);
                const int a = ab - b * P2;
                const int rowo = lix[warp][1][b] * n + lix[warp][0][a];
                R s0 = 0, s1 = 0;   // sum_z psi h, sum_z psi' h
                for (int c = 0; c < P2; ++c) {
                    const int off = lix[warp][2][c] + rowo;
                    if (!ENUF_GUARD(g.check, (size_t)off < n3, 5)) continue;
                    const R hv = h0[off];
                    s0 = fma(wts[warp][2][c], hv, s0);
                    s1 = fma(dwts[warp][2][c], hv, s1);
                }
                const R wx = wts[warp][0][a], wy = wts[warp][1][b];
                ax = fma(dwts[warp][0][a] * wy, s0, ax);
                ay = fma(wx * dwts[warp][1][b], s0, ay);
                az = fma(wx * wy, s1, az);
            }
        } else {
            for (int ab = lane; ab < P2 * P2; ab += 32) {
                const int b = (int)(((float)ab + 0.5f) * iP2);
                const int a = ab - b * P2;
                const int rowo = lix[warp][1][b] * n + lix[warp][0][a];
                R s0 = 0, s1 = 0, s2 = 0;   // sum_z psi h_a
                for (int c = 0; c < P2; ++c) {
                    const R w = wts[warp][2][c];
                    const int off = lix[warp][2][c] + rowo;   // z index pre-scaled by n^2
                    if (!ENUF_GUARD(g.check, (size_t)off < n3, 5)) continue;
                    s0 = fma(w, h0[off], s0);
                    s1 = fma(w, h1[off], s1);
                    s2 = fma(w, h2[off], s2);
                }
                const R wab = wts[warp][0][a] * wts[warp][1][b];
                ax = fma(wab, s0, ax);
                ay = fma(wab, s1, ay);
                az = fma(wab, s2, az);
            }
        }
        if constexpr (sizeof(R) == 8) {   // each lane's share as a global reduction (a warp
            const int i = real_as_int(wv.w);   // sum would run 15 adds on the FP64 units)
            const R f = pref * qs;
            atomicAdd(&F[3 * i], f * ax);
            atomicAdd(&F[3 * i + 1], f * ay);
            atomicAdd(&F[3 * i + 2], f * az);
        } else {
        ax = warp_sum_r(ax);
        ay = warp_sum_r(ay);
        az = warp_sum_r(az);
        if (lane == 0) {
            const int i = real_as_int(wv.w);
            const R f = pref * qs;
            F[3 * i] += f * ax;
            F[3 * i + 1] += f * ay;
            F[3 * i + 2] += f * az;
        }
        }
        __syncwarp();
    }
    if (tot.Edev) totals_if_last(g, tot, blk.n);
}

template <typename R, int PT = 0>
__global__ void __launch_bounds__(kGatherThreads) k_gather(Geo g, const int* __restrict__ tstart,
                                                           const typename V4<R>::T* __restrict__ sq,
                                                           const typename V4<R>::T* __restrict__ sw,
                                                           const int* __restrict__ sb, const R* __restrict__ wb,
                                                           const R* __restrict__ h, R* __restrict__ F,
                                                           TotalsArgs tot) {
    k_gather_body<R, PT>(g, tstart, sq, sw, sb, wb, h, F, tot, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// ---------------------------------------------------------------------------
// a7 (electrostatic part): real-space erfc + Slater-correction pairs on the
// tile bins (Eq. 31, corrected Eq. 32, Eq. 27-28). Warp per charged bead; lanes
// stride over the candidates of each contiguous run of tiles.
// ---------------------------------------------------------------------------
constexpr int kRealThreads = 256;
constexpr int kRealCap = 2048;     // staged beads (x, y, z, q)
constexpr int kRealHalo = 1024;    // halo tiles (stencil up to 9 x 9 x 9 + 1 for the prefix)
constexpr int kRealRound = 8;      // tiles staged together at most
// FP64 also stages a float copy of the positions for the cutoff pre-test
template <typename R> __host__ __device__ constexpr int real_cap() { return sizeof(R) == 8 ? 1536 : kRealCap; }
template <typename R>
constexpr int real_smem_bytes() {   // FP64 adds the float copy, the staged slots and the partner queue
    return (real_cap<R>() + (kRealThreads / 32) * 64) * (int)sizeof(typename V4<R>::T) + (2 * kRealHalo + 1) * 4 +
           (sizeof(R) == 8 ? real_cap<R>() * ((int)sizeof(float4) + 4) + (kRealThreads / 32) * 64 * 4 : 0);
}

// Kernel table: per interval [j h, (j + 1) h] of [0, r_c] the power-basis
// coefficients c_0..c_5 of the quintic Hermite interpolant of J in t = r/h - j
// (J, J', J'' matched at both ends); kKtStride64 / kKtStride32 values per
// interval (16-byte aligned rows: 6 doubles, or 6 floats padded to 8).
template <typename R>
__device__ __forceinline__ void kt_load(const R* __restrict__ kt, int j, R (&c)[6]) {
    if constexpr (sizeof(R) == 8) {
        const double2* a = reinterpret_cast<const double2*>(kt + kKtStride64 * j);
        const double2 a0 = __ldg(a), a1 = __ldg(a + 1), a2 = __ldg(a + 2);
        c[0] = a0.x; c[1] = a0.y; c[2] = a1.x; c[3] = a1.y; c[4] = a2.x; c[5] = a2.y;
    } else {
        const float4* a = reinterpret_cast<const float4*>(kt + kKtStride32 * j);
        const float4 a0 = __ldg(a), a1 = __ldg(a + 1);
        c[0] = a0.x; c[1] = a0.y; c[2] = a0.z; c[3] = a0.w; c[4] = a1.x; c[5] = a1.y;
    }
}

// Pair energy u(r) and radial force f(r) = -du/dr of the real-space sum,
// u = J(r)/r with J = erfc(alpha r) - (1 + beta r) e^{-2 beta r} (the
// Slater correction, beta > 0), or with the Slater form factor in k space
// J = B1 - I. With a table (kt != null: FP64, and the k-space form factor)
// J and dJ/dt come from one Horner pass over the interval's coefficients and
// f = (J - J' r)/r^2; otherwise erfc and exp are evaluated directly.
template <typename R>
__device__ __forceinline__ void real_pair(R r2, R al, R c2a, R be, bool slater, R& u, R& fr_over_r, R& f_r,
                                          const R* __restrict__ kt = nullptr, int kn = 0, R kinv = 0) {
    const R ir = r_rsqrt(r2);
    const R r = r2 * ir;
    if (kt) {
        const R x = r * kinv;
        int j = (int)x;
        j = j >= kn ? kn - 1 : j;   // x >= 0
        const R t = x - (R)j;
        R c[6];
        kt_load<R>(kt, j, c);
        R d = c[5];
        R p = fma(c[5], t, c[4]);
#pragma unroll
        for (int k = 3; k >= 0; --k) {
            d = fma(d, t, p);
            p = fma(p, t, c[k]);
        }
        // J = p, J' r = (dJ/dt) (1/h) r = d x
        const R ff = fma(-d, x, p) * ir * ir;
        u = p * ir;
        fr_over_r = ff * ir;
        f_r = ff * r;
        return;
    }
    const R ar = al * r;
    const R ec = r_erfc(ar);
    R uu = ec * ir;
    R ff = ec * ir * ir + c2a * r_exp(-ar * ar) * ir;
    if (slater) {
        const R br = be * r;
        const R e2 = r_exp((R)-2 * br);
        uu -= ((R)1 + br) * e2 * ir;
        ff -= ((R)1 + (R)2 * br + (R)2 * br * br) * e2 * ir * ir;
    }
    u = uu;
    fr_over_r = ff * ir;   // multiplies the displacement vector
    f_r = ff * r;          // virial term r f(r)
}

// One lane per queued pair (lanes < m).
// FP64 evaluates each pair once (Newton's third law: +f for bead i in the
// lane, -f to bead j, original index from its sorted slot, atomically): the
// pair arithmetic runs on the few FP64 units and halving it pays for the
// atomics. FP32 evaluates both directions (each bead only adds into its own
// force), measured faster there.
template <typename R> __host__ __device__ constexpr bool real_half() { return sizeof(R) == 8; }

template <typename R, typename V>
__device__ __forceinline__ void real_drain(const Geo& g, const V* qu, const int* quj, int m, int lane, R qi, R kap,
                                           R al, R c2a, R be, bool slater, const V* __restrict__ sw,
                                           R* __restrict__ F, R& fx, R& fy, R& fz, R& eacc, R& wacc) {
    constexpr bool HALF = real_half<R>();
    if (lane < m) {
        const V e = qu[lane];
        const R r2 = dist2(e.x, e.y, e.z);
        R u, fo, fr;
        real_pair<R>(r2, al, c2a, be, slater, u, fo, fr, static_cast<const R*>(g.ktab), g.kn, (R)g.kinv);
        const R qq = kap * qi * e.w;
        const R gx = qq * fo * e.x, gy = qq * fo * e.y, gz = qq * fo * e.z;
        fx += gx;
        fy += gy;
        fz += gz;
        if (HALF) {
            const int j = real_as_int(sw[quj[lane]].w);
            atomicAdd(&F[3 * j], -gx);
            atomicAdd(&F[3 * j + 1], -gy);
            atomicAdd(&F[3 * j + 2], -gz);
        }
        const R ws = HALF ? (R)1 : (R)0.5;   // energy and virial per pair
        eacc += ws * qq * u;
        wacc += ws * qq * fr;
    }
}

// Staged FP64: the queue holds the staged index of candidates that passed
// the float pre-test; the double displacement, the exact cutoff decision and
// the pair run here, on full warps (the sweep's candidates pass the float
// test on a few lanes at a time, and every FP64 instruction costs the whole
// warp's issue on GB300's FP64 units).
template <typename R, typename V>
__device__ __forceinline__ void real_drain_staged(const Geo& g, const V& pi, const V* stg, const int* stgslot,
                                                  const int* quj, int m, int lane, R L, R hL, R rc2, R kap, R al,
                                                  R c2a, R be, bool slater, const V* __restrict__ sw,
                                                  R* __restrict__ F, R& fx, R& fy, R& fz, R& eacc, R& wacc) {
    if (lane < m) {
        const int f = quj[lane];
        const V pj = stg[f];
        const R dx = min_image(pi.x, pj.x, L, hL);
        const R dy = min_image(pi.y, pj.y, L, hL);
        const R dz = min_image(pi.z, pj.z, L, hL);
        const R r2 = dist2(dx, dy, dz);
        if (r2 < rc2 && r2 > (R)0) {
            R u, fo, fr;
            real_pair<R>(r2, al, c2a, be, slater, u, fo, fr, static_cast<const R*>(g.ktab), g.kn, (R)g.kinv);
            const R qq = kap * pi.w * pj.w;
            const R gx = qq * fo * dx, gy = qq * fo * dy, gz = qq * fo * dz;
            fx += gx;
            fy += gy;
            fz += gz;
            const int j = real_as_int(sw[stgslot[f]].w);
            atomicAdd(&F[3 * j], -gx);
            atomicAdd(&F[3 * j + 1], -gy);
            atomicAdd(&F[3 * j + 2], -gz);
            eacc += qq * u;
            wacc += qq * fr;
        }
    }
}

// Halo of a tile: per dimension either the whole periodic row of tiles (when
// the stencil 2 rs + 1 covers it) or the tiles t - rs .. t + rs.
__device__ __forceinline__ void halo_dim(int t, int rs, int ntd, int& lo, int& cnt) {
    if (2 * rs + 1 >= ntd) { lo = 0; cnt = ntd; }
    else { lo = t - rs; cnt = 2 * rs + 1; }
}

// Beads [c0, c1) of one tile against the nh-tile halo (total beads), this
// warp's share being beads c0 + woff, c0 + woff + NW, ... STAGED: candidates
// from the shared-memory copy; else from global memory through the halo prefix.
template <typename R, bool STAGED>
__device__ __forceinline__ void real_beads(const Geo& g, int c0, int c1, int woff, int selfbase, int total, int nh,
                                           const typename V4<R>::T* stg, const float4* stgf, const int* stgslot,
                                           const int* hoff, const int* gst, const typename V4<R>::T* __restrict__ sq,
                                           const typename V4<R>::T* __restrict__ sw, typename V4<R>::T* qu, int* quj,
                                           R* __restrict__ F, R& eacc, R& wacc) {
    using V = typename V4<R>::T;
    constexpr int NW = kRealThreads / 32;
    // FP64: the cutoff test r^2 < r_c^2 runs on the float copy first; candidates
    // above a band that covers the float error (positions and L rounded to float,
    // |r2f - r2| <= ~1.5e-6 L r_c) are out, the rest are decided in double
    constexpr bool PRE = STAGED && sizeof(R) == 8;
    const float Lf = (float)g.L, hLf = (float)(0.5 * g.L);
    const float r2hi = (float)(g.rc * g.rc) * (1.0f + 1e-4f) + 4e-6f * (float)(g.L * g.rc) + 1e-6f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const R L = (R)g.L, hL = (R)(0.5 * g.L);
    const R rc2 = (R)(g.rc * g.rc);
    const R al = (R)g.alpha, c2a = (R)g.c2a, be = (R)g.beta, kap = (R)g.kappa;
    const bool slater = g.beta > 0.0;
    for (int s = c0 + woff; s < c1; s += NW) {
        const V pi = sq[s];
        const float4 pif = make_float4((float)pi.x, (float)pi.y, (float)pi.z, 0.f);
        const int self = selfbase + (s - c0);   // the bead's own index in the halo order
        R fx = 0, fy = 0, fz = 0;
        int cnt = 0;
        int hseg = 0;
        const int steps = (total + 31) / 32 + 1;   // the extra step drains the queue
        for (int it = 0; it < steps; ++it) {
            const bool last = it == steps - 1;
            if (!last) {
                const int f = it * 32 + lane;
                bool hit = false;
                R dx = 0, dy = 0, dz = 0, qj = 0;
                // FP64: each pair once, only candidates with a larger sorted slot;
                // FP32: every candidate but the bead itself
                int gs = -1;
                bool cand;
                if constexpr (real_half<R>()) {
                    if (f < total) {
                        if (STAGED) {
                            gs = stgslot[f];
                        } else {
                            while (hseg + 1 < nh && hoff[hseg + 1] <= f) ++hseg;
                            gs = gst[hseg] + f - hoff[hseg];
                        }
                    }
                    cand = gs > s;
                } else {
                    cand = f < total && f != self;
                    if (cand && !STAGED) {
                        while (hseg + 1 < nh && hoff[hseg + 1] <= f) ++hseg;
                        gs = gst[hseg] + f - hoff[hseg];
                    }
                }
                if (PRE && cand) {
                    const float4 b = stgf[f];
                    const float rx = min_image(pif.x, b.x, Lf, hLf);
                    const float ry = min_image(pif.y, b.y, Lf, hLf);
                    const float rz = min_image(pif.z, b.z, Lf, hLf);
                    cand = dist2(rx, ry, rz) <= r2hi;
                }
                if (PRE) {
                    hit = cand;   // decided exactly in the drain
                } else if (cand) {
                    V pj;
                    pj = STAGED ? stg[f] : sq[gs];
                    dx = min_image(pi.x, pj.x, L, hL);
                    dy = min_image(pi.y, pj.y, L, hL);
                    dz = min_image(pi.z, pj.z, L, hL);
                    const R r2 = dist2(dx, dy, dz);
                    hit = r2 < rc2 && r2 > (R)0;
                    qj = pj.w;
                }
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const int at = cnt + __popc(m & ((1u << lane) - 1u));
                    if (ENUF_GUARD(g.check, at < 64, 7)) {   // the warp's queue holds 64
                        if (PRE) {
                            quj[at] = f;
                        } else {
                            V e;
                            e.x = dx; e.y = dy; e.z = dz; e.w = qj;
                            qu[at] = e;
                            if (real_half<R>()) quj[at] = gs;
                        }
                    }
                }
                cnt += __popc(m);
            }
            if (cnt >= 32 || (last && cnt > 0)) {
                const int m = min(cnt, 32);
                __syncwarp();
                if constexpr (PRE)
                    real_drain_staged<R, V>(g, pi, stg, stgslot, quj, m, lane, L, hL, rc2, kap, al, c2a, be, slater,
                                            sw, F, fx, fy, fz, eacc, wacc);
                else
                    real_drain<R, V>(g, qu, quj, m, lane, pi.w, kap, al, c2a, be, slater, sw, F, fx, fy, fz, eacc,
                                     wacc);
                __syncwarp();
                if (lane < cnt - m) {
                    if (!PRE) qu[lane] = qu[m + lane];
                    if (real_half<R>()) quj[lane] = quj[m + lane];
                }
                __syncwarp();
                cnt -= m;
            }
        }
        if constexpr (sizeof(R) == 8) {   // each lane's share as a global reduction: a warp
            const int i = real_as_int(sw[s].w);   // sum would run 15 adds on the FP64 units
            atomicAdd(&F[3 * i], fx);
            atomicAdd(&F[3 * i + 1], fy);
            atomicAdd(&F[3 * i + 2], fz);
        } else {
        fx = warp_sum_r(fx);
        fy = warp_sum_r(fy);
        fz = warp_sum_r(fz);
        if (lane == 0) {   // a global reduction: other warps (as partners, or the DPD
            const int i = real_as_int(sw[s].w);   // blocks of a fused pair launch) add into F too
            atomicAdd(&F[3 * i], fx);
            atomicAdd(&F[3 * i + 1], fy);
            atomicAdd(&F[3 * i + 2], fz);
        }
        }
    }
}

// Real-space erfc + Slater-correction pairs (Eq. 31, corrected Eq. 32,
// Eq. 27-28). One CTA per grid tile: the beads of the tiles within r_c (the
// stencil) are staged in shared memory with coalesced loads; one warp per
// bead of the central tile runs over the staged candidates; accepted pairs
// are compacted in a per-warp queue so the pair arithmetic (erfc and exp in
// FP32, the tabulated kernel in FP64) runs on full warps.
template <typename R>
__device__ __forceinline__ void k_real_body(Geo g, const int* __restrict__ tstart,
                                                       const typename V4<R>::T* __restrict__ sq,
                                                       const typename V4<R>::T* __restrict__ sw,
                                                       R* __restrict__ F, double* __restrict__ rpart, Blk blk) {
    pdl_enter();
    using V = typename V4<R>::T;
    constexpr int NW = kRealThreads / 32;
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int CAP = real_cap<R>();
    V* stg = reinterpret_cast<V*>(smraw);                       // [CAP]
    V* queue = stg + CAP;                                       // [NW][64]
    float4* stgf = reinterpret_cast<float4*>(queue + NW * 64);  // [CAP] float positions (FP64 only)
    int* hoff = reinterpret_cast<int*>(stgf + (sizeof(R) == 8 ? CAP : 0));   // [kRealHalo + 1]
    int* gst = hoff + kRealHalo + 1;                            // [kRealHalo]
    int* stgslot = gst + kRealHalo;                             // [CAP] sorted slot of each staged bead (FP64)
    int* quj = stgslot + CAP;                                   // [NW][64] partner slots (FP64)
    __shared__ int wtot[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    V* qu = queue + warp * 64;
    R eacc = 0, wacc = 0;
    // Rounds of up to kRealRound tiles of this block's sequence whose halos fit
    // the staging buffer together: each tile's halo is staged into its own
    // segment, then the warps take the round's beads in turn across the tiles
    // (a tile holds a few beads at large sizes, fewer than the warps), with no
    // barrier between tiles. A tile whose halo alone does not fit runs by
    // itself from global memory.
    __shared__ int r_c0[kRealRound], r_c1[kRealRound], r_seg[kRealRound], r_self[kRealRound], r_tot[kRealRound];
    __shared__ int r_cnt, r_used, r_next;
    int tile = blk.id;
    while (tile < g.ntiles) {
        if (tid == 0) {
            r_cnt = 0;
            r_used = 0;
        }
        __syncthreads();
        int t = tile;
        while (t < g.ntiles) {
            const int tx = t % g.ntd, ty = (t / g.ntd) % g.ntd, tz = t / (g.ntd * g.ntd);
            int xlo, xc, ylo, yc, zlo, zc;
            halo_dim(tx, g.rs, g.ntd, xlo, xc);
            halo_dim(ty, g.rs, g.ntd, ylo, yc);
            halo_dim(tz, g.rs, g.ntd, zlo, zc);
            const int nh = xc * yc * zc;   // <= kRealHalo by construction of the plan
            if (!ENUF_GUARD(g.check, nh <= kRealHalo, 6)) {   // uniform over the block
                t += blk.n;
                continue;
            }
            // halo tile ranges and their exclusive prefix (block scan, <= 4 per thread)
            int cnt4[4], sum = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int h = 4 * tid + k;
                cnt4[k] = 0;
                if (h < nh) {
                    const int hx = h % xc, hy = (h / xc) % yc, hz = h / (xc * yc);
                    const int ax = (xlo + hx + g.ntd) % g.ntd, ay = (ylo + hy + g.ntd) % g.ntd,
                              az = (zlo + hz + g.ntd) % g.ntd;
                    const int tt = (az * g.ntd + ay) * g.ntd + ax;
                    const int st = tstart[tt];
                    gst[h] = st;
                    cnt4[k] = tstart[tt + 1] - st;
                }
                sum += cnt4[k];
            }
            int x = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wtot[warp] = x;
            __syncthreads();
            int run = x - sum;
            for (int w = 0; w < warp; ++w) run += wtot[w];
            int total = 0;
            for (int w = 0; w < NW; ++w) total += wtot[w];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int h = 4 * tid + k;
                if (h < nh) hoff[h] = run;
                run += cnt4[k];
            }
            if (tid == 0) hoff[nh] = total;
            __syncthreads();
            const int used = r_used, cnt = r_cnt;
            const int c0 = tstart[t], c1 = tstart[t + 1];
            const int hc = (((tz - zlo + g.ntd) % g.ntd) * yc + (ty - ylo + g.ntd) % g.ntd) * xc +
                           (tx - xlo + g.ntd) % g.ntd;
            if (total > CAP) {
                if (cnt == 0) {   // this tile alone, candidates from global memory
                    real_beads<R, false>(g, c0, c1, warp, hoff[hc], total, nh, stg, stgf, stgslot, hoff, gst, sq,
                                         sw, qu, quj + warp * 64, F, eacc, wacc);
                    t += blk.n;
                }
                break;   // an oversized halo closes the round
            }
            if (used + total > CAP) break;   // staged with the next round
            for (int f = tid; f < total; f += blockDim.x) {
                int lo = 0, hi = nh;   // last h with hoff[h] <= f
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (hoff[mid] <= f) lo = mid; else hi = mid;
                }
                const int gsl = gst[lo] + f - hoff[lo];
                const V v = sq[gsl];
                stg[used + f] = v;
                if (real_half<R>()) stgslot[used + f] = gsl;
                if (sizeof(R) == 8) stgf[used + f] = make_float4((float)v.x, (float)v.y, (float)v.z, 0.f);
            }
            if (tid == 0) {
                r_c0[cnt] = c0;
                r_c1[cnt] = c1;
                r_seg[cnt] = used;
                r_self[cnt] = hoff[hc];
                r_tot[cnt] = total;
                r_cnt = cnt + 1;
                r_used = used + total;
            }
            __syncthreads();   // hoff, gst and the counters are read again for the next tile
            t += blk.n;
            if (r_cnt == kRealRound) break;
        }
        if (tid == 0) r_next = t;
        __syncthreads();
        // the round's beads, warps in turn across its tiles
        const int cnt = r_cnt;
        int before = 0;
        for (int k = 0; k < cnt; ++k) {
            const int c0 = r_c0[k], c1 = r_c1[k], seg = r_seg[k];
            const int woff = ((warp - before) % NW + NW) % NW;
            real_beads<R, true>(g, c0, c1, woff, r_self[k], r_tot[k], 0, stg + seg, stgf + seg, stgslot + seg, hoff,
                                gst, sq, sw, qu, quj + warp * 64, F, eacc, wacc);
            before += c1 - c0;
        }
        tile = r_next;
        __syncthreads();
    }
    double e = (double)eacc, w = (double)wacc;
    block_sum2(e, w);
    if (threadIdx.x == 0) {
        rpart[2 * blk.id] = e;
        rpart[2 * blk.id + 1] = w;
    }
}

template <typename R>
__global__ void __launch_bounds__(kRealThreads) k_real(Geo g, const int* __restrict__ tstart,
                                                       const typename V4<R>::T* __restrict__ sq,
                                                       const typename V4<R>::T* __restrict__ sw,
                                                       R* __restrict__ F, double* __restrict__ rpart) {
    k_real_body<R>(g, tstart, sq, sw, F, rpart, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// ---------------------------------------------------------------------------
// DPD: cell list of all beads (edge >= 1) by a counting sort.
// ---------------------------------------------------------------------------
// Cells of edge L/ncd > 1 (the plan keeps a relative margin so that rounding
// of x * ncd/L cannot separate two beads closer than 1 by two cells).
template <typename R>
__global__ void k_cell_count(int N, int ncd, double L, double inv, float xmaxf, const R* __restrict__ pos,
                             int* __restrict__ ckey, int* __restrict__ ccount, R* __restrict__ F) {
    pdl_enter();
    const R rinv = (R)inv;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        F[3 * i] = (R)0;   // the pair kernel adds into F
        F[3 * i + 1] = (R)0;
        F[3 * i + 2] = (R)0;
        int c[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            int v = (int)(wrap_r(pos[3 * i + t], L, xmaxf) * rinv);
            c[t] = v < 0 ? 0 : (v >= ncd ? ncd - 1 : v);
        }
        const int cell = (c[2] * ncd + c[1]) * ncd + c[0];
        ckey[i] = cell;
        atomicAdd(&ccount[cell], 1);
    }
}

// Also clears the cell counts for the next step's k_cell_count (the scan has
// read them).
template <typename R>
__global__ void k_cell_scatter(int N, double L, float xmaxf, const R* __restrict__ pos, const R* __restrict__ v0,
                               const int* __restrict__ type, const int* __restrict__ ckey,
                               int* __restrict__ ccur, typename V4<R>::T* __restrict__ sp,
                               typename V4<R>::T* __restrict__ sv, int* __restrict__ ccount, int ncells) {
    pdl_enter();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) ccount[c] = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int slot = atomicAdd(&ccur[ckey[i]], 1);
        typename V4<R>::T a, b;
        a.x = wrap_r(pos[3 * i], L, xmaxf);
        a.y = wrap_r(pos[3 * i + 1], L, xmaxf);
        a.z = wrap_r(pos[3 * i + 2], L, xmaxf);
        a.w = int_as_real(i, (R)0);
        b.x = v0[3 * i];
        b.y = v0[3 * i + 1];
        b.z = v0[3 * i + 2];
        b.w = int_as_real(type[i], (R)0);
        sp[slot] = a;
        sv[slot] = b;
    }
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products,
// key bumped by the Weyl constants between rounds. theta_ij draws word 0 of
// the counter (min(i,j), max(i,j), step_lo, step_hi) under key = seed. Within
// a launch the key and the step are fixed: the round keys come from the host
// (DpdDev::rk0/rk1, read as launch constants) and the first round's product
// of the counter word step_lo is formed once per thread (PhiloxStep); a draw
// then costs one wide multiply for word 0 in the first round, two per round
// after it, and one in the last (whose other outputs are not used).
struct PhiloxStep {
    uint32_t lo1, hi1;   // 0xCD9E8D57 * step_lo
    uint32_t x2;         // step_hi ^ round key 1 of round 0
};
__device__ __forceinline__ PhiloxStep philox_step(const DpdDev& d, uint64_t step) {
    const uint64_t p = (uint64_t)0xCD9E8D57u * (uint32_t)step;
    PhiloxStep ps;
    ps.lo1 = (uint32_t)p;
    ps.hi1 = (uint32_t)(p >> 32);
    ps.x2 = (uint32_t)(step >> 32) ^ d.rk1[0];
    return ps;
}
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, const PhiloxStep& ps, const DpdDev& d) {
    // round 0: the product of word 2 is the launch's
    const uint64_t p00 = (uint64_t)0xD2511F53u * c0;
    uint32_t n0 = ps.hi1 ^ c1 ^ d.rk0[0];
    uint32_t n1 = ps.lo1;
    uint32_t n2 = (uint32_t)(p00 >> 32) ^ ps.x2;
    uint32_t n3 = (uint32_t)p00;
#pragma unroll
    for (int r = 1; r < 9; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * n0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * n2;
        const uint32_t m0 = (uint32_t)(p1 >> 32) ^ n1 ^ d.rk0[r];
        const uint32_t m2 = (uint32_t)(p0 >> 32) ^ n3 ^ d.rk1[r];
        n1 = (uint32_t)p1;
        n3 = (uint32_t)p0;
        n0 = m0;
        n2 = m2;
    }
    // round 9: word 0 only
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * n2;
    return (uint32_t)(p1 >> 32) ^ n1 ^ d.rk0[9];
}

// theta_ij of Eq. 5: uniform on [-sqrt3, sqrt3].
template <typename R>
__device__ __forceinline__ R dpd_theta(const PhiloxStep& ps, const DpdDev& d, int i, int j) {
    const uint32_t w = philox_word0((uint32_t)min(i, j), (uint32_t)max(i, j), ps, d);
    // sqrt3 (2 u - 1) with u = (w + 1/2) 2^-32
    return fma((R)w, (R)(2.0 * 1.7320508075688772935 * 2.3283064365386962890625e-10),
               (R)(1.7320508075688772935 * (2.3283064365386962890625e-10 - 1.0)));
}

// DPD pair forces (Eq. 2-7, R_c = 1) + bonds (Sec. 2), added into F (which
// the caller zeroes): F[i] += F^C + F^D + F^R/sqrt(dt) + F^S. One CTA per B^3
// block of cells; the beads of the (B+2)^3 halo cells are staged in shared
// memory in halo-cell order (a warp per halo row: the H cells of a row along
// x are one contiguous run of the staged order). Every pair is evaluated once
// (Newton's third law; theta_ij is symmetric): a bead's partners are the
// beads of its forward half shell -- the beads after it in its own cell and
// the 13 neighbouring cells lexicographically after it, which in the staged
// copy are 5 contiguous runs of slots. One lane per central bead walks its
// runs (dpd_beads); the pairs within r = 1 go to a per-warp ring of pairs and
// the pair arithmetic (Philox draw, weights, dissipation) runs on full warps.
// The forces go out by global reductions, +f to i and -f to j (executed in
// L2: shared-memory float adds are compare-and-swap loops on this part, and
// in FP64 each of their iterations costs an add on the few FP64 units). The
// harmonic bonds run as one thread per bond into F. A block whose halo holds
// more beads than the staging capacity sweeps the global cell list instead,
// one warp per central cell (dpd_cells).
//
// The staged copies are unwrapped: the halo cells that lie across a box
// face are shifted by L, so the plain difference of two staged positions is
// the minimum image of every pair within r = 1 (cell edge >= 1) and no pair
// needs the wrap test. FP64: the cutoff test r^2 < 1 is taken on a float copy
// of the staged positions first and redone in double only inside a band
// around 1 (and near 0) that covers the float error, so the decision is the
// double one.
constexpr int kDpdThreads = 256;
// kDpdCap (staged beads per block) is in enuf_internal.h: the host sizes the
// cell blocks against it
constexpr int kDpdMaxB = 4;      // cells per block edge
constexpr int kDpdSegU = 14;     // unstaged half shell: single cells
constexpr int kDpdU = 4;         // bead sweep: candidates per lane and iteration
constexpr int kDpdQ = 256;       // bead sweep: pair ring per warp (>= 31 + 32 kDpdU, a power of 2)
static_assert(kDpdQ >= 31 + 32 * kDpdU && (kDpdQ & (kDpdQ - 1)) == 0, "pair ring");

template <typename R>
constexpr int dpd_smem_bytes() {
    return 2 * kDpdCap * (int)sizeof(typename V4<R>::T) + (sizeof(R) == 8 ? kDpdCap * (int)sizeof(float4) : 0) +
           (kDpdThreads / 32) * kDpdQ * 8;
}

// One warp-wide batch of up to 32 queued pairs (valid lanes) of the global
// cell list (wrapped positions: minimum image), all lanes call. The queue
// holds runs of one i (dpd_cells loops over i inside a candidate chunk): in
// FP32 the +f of a run is summed in the warp first, then added once; in FP64
// it goes per pair (the segmented sum would run on the few FP64 units).
template <typename R, typename V>
__device__ __forceinline__ void dpd_pairs(const bool valid, const int2 e, const V* __restrict__ P,
                                          const V* __restrict__ Pv, R* __restrict__ F,
                                          const R* __restrict__ atab, int ntypes, R L, R hL, R gam, R srdt,
                                          const PhiloxStep& ps, const DpdDev& d, R& ec) {
    const int lane = threadIdx.x & 31;
    R fx = 0, fy = 0, fz = 0;
    int key = -1, oi = 0;
    if (valid) {
        const V pi = P[e.x], vi = Pv[e.x];
        const V pj = P[e.y], vj = Pv[e.y];
        const R rx = min_image(pi.x, pj.x, L, hL);
        const R ry = min_image(pi.y, pj.y, L, hL);
        const R rz = min_image(pi.z, pj.z, L, hL);
        const R r2 = dist2(rx, ry, rz);
        const R ir = r_rsqrt(r2);
        const R r = r2 * ir;
        const R w = (R)1 - r;
        const int i = real_as_int(pi.w), j = real_as_int(pj.w);
        const int ti = real_as_int(vi.w), tj = real_as_int(vj.w);
        const R a = atab[ti * ntypes + tj];
        const R vd = (vi.x - vj.x) * rx + (vi.y - vj.y) * ry + (vi.z - vj.z) * rz;   // r_ij . v_ij
        const R th = dpd_theta<R>(ps, d, i, j);
        // Eq. 3-5 with w^D = (w^R)^2 = w^2: |F| = w (a - gamma w (r.v)/r + sigma theta/sqrt(dt))
        const R wi = w * ir;
        const R fm = wi * fma(-gam * wi, vd, fma(srdt, th, a));
        fx = fm * rx;
        fy = fm * ry;
        fz = fm * rz;
        // -f to bead j: a global reduction (executed in L2, no compare-and-swap loop)
        atomicAdd(&F[3 * j], -fx);
        atomicAdd(&F[3 * j + 1], -fy);
        atomicAdd(&F[3 * j + 2], -fz);
        ec = fma(a * w, w, ec);   // a w^2; halved once per block
        key = e.x;
        oi = i;
    }
    if constexpr (sizeof(R) == 8) {
        // FP64: +f to bead i per pair as well (the segmented sum below would
        // run its adds and double shuffles on the few FP64 units)
        if (key >= 0) {
            atomicAdd(&F[3 * oi], fx);
            atomicAdd(&F[3 * oi + 1], fy);
            atomicAdd(&F[3 * oi + 2], fz);
        }
        (void)lane;
        return;
    }
    // runs of equal i: sum each run into its first lane (segmented suffix sums)
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned after = lane == 31 ? 0u : heads & (0xffffffffu << (lane + 1));
    const int end = after ? __ffs(after) - 1 : 32;
    // levels up to the longest run of the batch (typically 2-3 of 5)
    const int longest = __reduce_max_sync(0xffffffffu, head ? end - lane : 0);
    for (int o = 1; o < longest; o <<= 1) {
        const R ax = __shfl_down_sync(0xffffffffu, fx, o);
        const R ay = __shfl_down_sync(0xffffffffu, fy, o);
        const R az = __shfl_down_sync(0xffffffffu, fz, o);
        if (lane + o < end) {
            fx += ax;
            fy += ay;
            fz += az;
        }
    }
    if (head && key >= 0) {
        atomicAdd(&F[3 * oi], fx);
        atomicAdd(&F[3 * oi + 1], fy);
        atomicAdd(&F[3 * oi + 2], fz);
    }
}

// The exact cutoff decision 0 < r^2 < 1 in the working precision (WRAP:
// minimum image of wrapped positions; else the unwrapped staged frame).
template <typename R, typename V, bool WRAP>
__device__ __forceinline__ bool dpd_within(const V& pi, const V& pj, R L, R hL) {
    const R rx = WRAP ? min_image(pi.x, pj.x, L, hL) : pi.x - pj.x;
    const R ry = WRAP ? min_image(pi.y, pj.y, L, hL) : pi.y - pj.y;
    const R rz = WRAP ? min_image(pi.z, pj.z, L, hL) : pi.z - pj.z;
    const R r2 = dist2(rx, ry, rz);
    return r2 < (R)1 && r2 > (R)0;
}

struct DpdBand {   // float pre-test of the FP64 path: r2f > hi: out; lo0 < r2f < lo: in; else exact
    float L, hL, lo0, lo, hi;
};

// All central cells of one block on the global cell list (a block whose halo
// overflows the staging capacity), one warp per cell: lanes over the
// candidates of the cell's half shell (its own cell, the next along x and the
// 12 cells of the rows after it, each looked up wrapped), a loop over the
// cell's beads; positions are wrapped, so pairs take the minimum image.
template <typename R>
__device__ __forceinline__ void dpd_cells(const DpdDev& d, int H, int B3, const int* chalo, const int* hoff,
                                          const int* gst, const typename V4<R>::T* __restrict__ P,
                                          const typename V4<R>::T* __restrict__ Pv, int2* queue,
                                          const R* __restrict__ atab, uint64_t step, R* __restrict__ F, R& ec) {
    using V = typename V4<R>::T;
    constexpr int NW = kDpdThreads / 32;
    constexpr int nseg = kDpdSegU;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const R L = (R)d.L, hL = (R)(0.5 * d.L);
    const R gam = (R)d.gamma, srdt = (R)(d.sigma * d.rdt);
    const PhiloxStep ps = philox_step(d, step);
    int cnt = 0;   // queued pairs of this warp, carried across its cells
    for (int cc = warp; cc < B3; cc += NW) {
        const int h = chalo[cc];
        if (h < 0) continue;
        const int cb = gst[h];
        const int nself = hoff[h + 1] - hoff[h];
        if (nself == 0) continue;
        // lane s < nseg: cell s of the half shell as (start slot, length)
        int sst = 0, sln = 0;
        if (lane < nseg) {
            int hc;
            if (lane == 0) hc = h;
            else if (lane == 1) hc = h + 1;
            else if (lane < 5) hc = h + H + (lane - 3);
            else hc = h + H * H + ((lane - 5) / 3 - 1) * H + ((lane - 5) % 3 - 1);
            sst = gst[hc];
            sln = hoff[hc + 1] - hoff[hc];
        }
        int x = sln;   // inclusive prefix of the cell counts
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int soff = x - sln;          // cell s starts at map position soff
        const int delta = sst - soff;      // slot = map position + delta
        const int mc = __shfl_sync(0xffffffffu, x, nseg - 1);
        // lanes over the map (one candidate j per lane per chunk), loop over the
        // cell's beads i (broadcast loads); queue runs are then runs of one i
        for (int jb = 0; jb < mc; jb += 32) {
            const int jf = jb + lane;
            int s = 0;
            for (int k = 1; k < nseg; ++k) s += jf >= __shfl_sync(0xffffffffu, soff, k) ? 1 : 0;
            const int j = jf + __shfl_sync(0xffffffffu, delta, s);
            const bool vj = jf < mc;
            V pj;
            if (vj) pj = P[j];
            for (int ii = 0; ii < nself; ++ii) {
                const int me = cb + ii;
                // forward only within the cell itself (run 0)
                bool hit = false;
                if (vj && (s != 0 || j > me)) hit = dpd_within<R, V, true>(P[me], pj, L, hL);
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit && ENUF_GUARD(d.check, cnt + __popc(m & ((1u << lane) - 1u)) < 64, 9))
                    queue[cnt + __popc(m & ((1u << lane) - 1u))] = make_int2(me, j);
                cnt += __popc(m);
                if (cnt >= 32) {
                    __syncwarp();
                    dpd_pairs<R, V>(true, queue[lane], P, Pv, F, atab, d.ntypes, L, hL, gam, srdt, ps, d, ec);
                    __syncwarp();
                    if (lane < cnt - 32) queue[lane] = queue[32 + lane];
                    __syncwarp();
                    cnt -= 32;
                }
            }
        }
    }
    __syncwarp();
    if (cnt > 0) dpd_pairs<R, V>(lane < cnt, queue[lane], P, Pv, F, atab, d.ntypes, L, hL, gam, srdt, ps, d, ec);
}

// One warp-wide batch of up to 32 queued pairs (i, j) whose i are mostly
// distinct (the bead sweep below queues one pair per lane and candidate):
// +f to i and -f to j, each by one global reduction per component.
template <typename R, typename V>
__device__ __forceinline__ void dpd_pairs_red(const bool valid, const int2 e, const V* __restrict__ P,
                                              const V* __restrict__ Pv, R* __restrict__ F,
                                              const R* __restrict__ atab, int ntypes, R gam, R srdt,
                                              const PhiloxStep& ps, const DpdDev& d, R& ec) {
    if (!valid) return;
    const V pi = P[e.x], vi = Pv[e.x];
    const V pj = P[e.y], vj = Pv[e.y];
    const R rx = pi.x - pj.x, ry = pi.y - pj.y, rz = pi.z - pj.z;   // unwrapped staged frame
    const R r2 = dist2(rx, ry, rz);
    const R ir = r_rsqrt(r2);
    const R w = (R)1 - r2 * ir;
    const int i = real_as_int(pi.w), j = real_as_int(pj.w);
    const R a = atab[real_as_int(vi.w) * ntypes + real_as_int(vj.w)];
    const R vd = (vi.x - vj.x) * rx + (vi.y - vj.y) * ry + (vi.z - vj.z) * rz;   // r_ij . v_ij
    const R th = dpd_theta<R>(ps, d, i, j);
    // Eq. 3-5 with w^D = (w^R)^2 = w^2: |F| = w (a - gamma w (r.v)/r + sigma theta/sqrt(dt))
    const R wi = w * ir;
    const R fm = wi * fma(-gam * wi, vd, fma(srdt, th, a));
    const R fx = fm * rx, fy = fm * ry, fz = fm * rz;
    atomicAdd(&F[3 * i], fx);
    atomicAdd(&F[3 * i + 1], fy);
    atomicAdd(&F[3 * i + 2], fz);
    atomicAdd(&F[3 * j], -fx);
    atomicAdd(&F[3 * j + 1], -fy);
    atomicAdd(&F[3 * j + 2], -fz);
    ec = fma(a * w, w, ec);   // a w^2; halved once per block
}

// The staged pair sweep with one lane per central bead: lane f of the block's
// central beads (cpre: prefix of the central cells' counts) walks the forward
// half shell of its cell -- the rest of its own cell and the next cell along
// x (run 0: slots after its own), the row (0, +1, -1..1) (run 1) and the
// three rows (+1, -1..1, -1..1) (runs 2-4), each a contiguous run of staged
// slots -- one candidate per iteration. A warp tests 32 beads' candidates at
// once; the pairs within r = 1 go to the warp's queue and are evaluated on
// full warps. Against one warp per cell (lanes over candidates, a loop over
// the cell's beads) this has no per-cell prefix of run lengths, no chunk
// remainders and one test per candidate.
template <typename R>
__device__ __forceinline__ void dpd_beads(const DpdDev& d, int H, int B3, const int* chalo, const int* cpre,
                                          const int* hoff, const typename V4<R>::T* __restrict__ P,
                                          const typename V4<R>::T* __restrict__ Pv, const float4* Pf,
                                          const DpdBand band, int2* queue, const R* __restrict__ atab,
                                          uint64_t step, R* __restrict__ F, R& ec) {
    using V = typename V4<R>::T;
    constexpr int NW = kDpdThreads / 32;
    constexpr bool PRE = sizeof(R) == 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const R L = (R)d.L, hL = (R)(0.5 * d.L);
    const R gam = (R)d.gamma, srdt = (R)(d.sigma * d.rdt);
    const PhiloxStep ps = philox_step(d, step);
    const int nc = cpre[B3];
    int cnt = 0, qh = 0;   // queued pairs of this warp, ring head
    for (int base = warp * 32; base < nc; base += NW * 32) {
        const int f = base + lane;
        const bool own = f < nc;
        int i = 0, h = 0;
        if (own) {
            int lo = 0, hi = B3;   // the central cell holding bead f
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (cpre[mid] <= f) lo = mid; else hi = mid;
            }
            h = chalo[lo];
            i = hoff[h] + f - cpre[lo];
        }
        V pi;
        float4 pif;
        if (own) {
            pi = P[i];
            if constexpr (PRE) pif = Pf[i];
        }
        // the five runs one after the other (uniform over the warp); within a
        // run, lane-local candidate t of the run, as long as the warp's longest
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            int j0 = 0, len = 0;
            if (own) {
                const int o = k == 0 ? 0 : (k == 1 ? H - 1 : H * H + (k - 3) * H - 1);
                j0 = k == 0 ? i + 1 : hoff[h + o];
                len = hoff[h + o + (k == 0 ? 2 : 3)] - j0;
            }
            const int mlen = __reduce_max_sync(0xffffffffu, len);
            // kDpdU candidates per lane and iteration: their loads and tests
            // are independent, then one ballot and append each
            for (int t = 0; t < mlen; t += kDpdU) {
                bool hit[kDpdU];
#pragma unroll
                for (int u = 0; u < kDpdU; ++u) {
                    hit[u] = false;
                    if (t + u < len) {
                        const int j = j0 + t + u;
                        if constexpr (PRE) {
                            const float4 b = Pf[j];
                            const float r2 = dist2(pif.x - b.x, pif.y - b.y, pif.z - b.z);
                            if (r2 <= band.hi)
                                hit[u] = (r2 < band.lo && r2 > band.lo0) || dpd_within<R, V, false>(pi, P[j], L, hL);
                        } else {
                            hit[u] = dpd_within<R, V, false>(pi, P[j], L, hL);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kDpdU; ++u) {
                    const unsigned m = __ballot_sync(0xffffffffu, hit[u]);
                    if (hit[u]) queue[(qh + cnt + __popc(m & ((1u << lane) - 1u))) & (kDpdQ - 1)] = make_int2(i, j0 + t + u);
                    cnt += __popc(m);
                }
                while (cnt >= 32) {
                    __syncwarp();
                    dpd_pairs_red<R, V>(true, queue[(qh + lane) & (kDpdQ - 1)], P, Pv, F, atab, d.ntypes, gam, srdt,
                                        ps, d, ec);
                    qh += 32;
                    cnt -= 32;
                }
            }
        }
    }
    __syncwarp();
    if (cnt > 0)
        dpd_pairs_red<R, V>(lane < cnt, queue[(qh + lane) & (kDpdQ - 1)], P, Pv, F, atab, d.ntypes, gam, srdt, ps, d,
                            ec);
}

template <typename R>
__device__ __forceinline__ void k_dpd_body(DpdDev d, int B, const typename V4<R>::T* __restrict__ sp, const typename V4<R>::T* __restrict__ sv,
          const int* __restrict__ cstart, const R* __restrict__ atab, const R* __restrict__ pos,
          const int* __restrict__ bnd, const uint64_t* __restrict__ stepp, R* __restrict__ F,
          double* __restrict__ dpart, Blk bk) {
    pdl_enter();
    using V = typename V4<R>::T;
    constexpr bool F64 = sizeof(R) == 8;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* spos = reinterpret_cast<V*>(smraw);                                  // [kDpdCap]
    V* svel = spos + kDpdCap;                                               // [kDpdCap]
    float4* spf = reinterpret_cast<float4*>(svel + kDpdCap);                // [kDpdCap] (FP64 only)
    int2* queues = reinterpret_cast<int2*>(spf + (F64 ? kDpdCap : 0));      // [NW][kDpdQ]
    constexpr int HMAX = (kDpdMaxB + 2) * (kDpdMaxB + 2) * (kDpdMaxB + 2);
    __shared__ int hoff[HMAX + 1], gst[HMAX];
    __shared__ int chalo[kDpdMaxB * kDpdMaxB * kDpdMaxB];
    __shared__ int cpre[kDpdMaxB * kDpdMaxB * kDpdMaxB + 1];   // prefix of the central cells' counts
    __shared__ unsigned char hsh[HMAX];   // per halo cell: 2 bits per axis, 1: -L, 2: +L
    const uint64_t step = *stepp;
    const int ncd = d.ncd, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int2* queue = queues + warp * kDpdQ;
    const int H = B + 2, H3 = H * H * H, B3 = B * B * B;
    if (!ENUF_GUARD(d.check, H3 <= HMAX && B3 <= kDpdMaxB * kDpdMaxB * kDpdMaxB, 8)) return;
    const int nblk = (ncd + B - 1) / B;
    const R L = (R)d.L, hL = (R)(0.5 * d.L);
    R ec = 0, eb = 0;
    // harmonic bonds (Sec. 2): one thread per bond, +f to i and -f to j
    {
        const R Kb = (R)d.K_bond, r0b = (R)d.r0_bond, iL = (R)(1.0 / d.L);
        for (int k = bk.id * blockDim.x + tid; k < d.nbonds; k += bk.n * blockDim.x) {
            const int i = bnd[2 * k], j = bnd[2 * k + 1];
            R dd[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                // minimum image of the raw (unwrapped) difference; a bond is far
                // shorter than L/2, so d/L is never near a half-integer
                const R dx = pos[3 * i + t] - pos[3 * j + t];
                dd[t] = dx - L * rint(dx * iL);
            }
            const R r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
            const R ir = r2 > (R)0 ? r_rsqrt(r2) : (R)0;
            const R dr = r2 * ir - r0b;   // r - r0
            eb = fma(Kb * dr, dr, eb);    // K (r - r0)^2; halved once per block
            if (r2 > (R)0) {
                const R fm = -Kb * dr * ir;
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    atomicAdd(&F[3 * i + t], fm * dd[t]);
                    atomicAdd(&F[3 * j + t], -fm * dd[t]);
                }
            }
        }
    }
    // float band of the FP64 cutoff test: the staged float positions (in
    // [-1 - L/3, 4L/3]) carry at most (4L/3 + 1) 2^-24 each, so for r2 near 1
    // |r2f - r2| <= 7e-7 (L + 1) + 3e-7
    DpdBand band;
    band.L = (float)d.L;
    band.hL = (float)(0.5 * d.L);
    const float eps = 1e-4f + 4e-6f * (float)d.L;
    band.lo0 = eps;
    band.lo = 1.0f - eps;
    band.hi = 1.0f + eps;
    for (int blk = bk.id; blk < nblk * nblk * nblk; blk += bk.n) {
        const int bx = blk % nblk, by = (blk / nblk) % nblk, bz = blk / (nblk * nblk);
        const int c0x = bx * B, c0y = by * B, c0z = bz * B;
        if (tid < H3) {   // halo cell ranges (H^3 <= 216 cells)
            const int hx = tid % H, hy = (tid / H) % H, hz = tid / (H * H);
            const int ux = c0x - 1 + hx, uy = c0y - 1 + hy, uz = c0z - 1 + hz;   // unwrapped
            const int cx = (ux + ncd) % ncd, cy = (uy + ncd) % ncd, cz = (uz + ncd) % ncd;
            const int c = (cz * ncd + cy) * ncd + cx;
            const int st = cstart[c];
            gst[tid] = st;
            hoff[tid] = cstart[c + 1] - st;
            auto code = [&](int u) { return u < 0 ? 1 : (u >= ncd ? 2 : 0); };
            hsh[tid] = (unsigned char)(code(ux) | code(uy) << 2 | code(uz) << 4);
        }
        if (tid < B3) {   // central cells of this block (clipped at the box edge)
            const int ix = tid % B, iy = (tid / B) % B, iz = tid / (B * B);
            const bool ok = c0x + ix < ncd && c0y + iy < ncd && c0z + iz < ncd;
            chalo[tid] = ok ? ((iz + 1) * H + (iy + 1)) * H + (ix + 1) : -1;
        }
        __syncthreads();
        if (warp == 0) {   // exclusive prefix of the halo counts (<= 7 per lane)
            const int per = (H3 + 31) / 32;
            int v[7], sum = 0;
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                const int h = lane * per + k;
                v[k] = (k < per && h < H3) ? hoff[h] : 0;
                sum += v[k];
            }
            int x = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            int run = x - sum;
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                const int h = lane * per + k;
                if (k < per && h < H3) hoff[h] = run;
                run += v[k];
            }
            if (lane == 31) hoff[H3] = x;
        }
        __syncthreads();
        const int total = hoff[H3];
        const bool staged = total <= kDpdCap;
        if (staged && warp == 0) {   // central cells' bead counts, exclusive prefix (B3 <= 64)
            const int c0 = 2 * lane, c1 = 2 * lane + 1;
            const int h0 = c0 < B3 ? chalo[c0] : -1, h1 = c1 < B3 ? chalo[c1] : -1;
            const int n0 = h0 >= 0 ? hoff[h0 + 1] - hoff[h0] : 0;
            const int n1 = h1 >= 0 ? hoff[h1 + 1] - hoff[h1] : 0;
            int x = n0 + n1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const int ex = x - n0 - n1;
            if (c0 < B3) cpre[c0] = ex;
            if (c1 < B3) cpre[c1] = ex + n0;
            if (lane == 31) cpre[B3] = x;
        }
        if (staged) {
            // a warp per halo row (H cells along x, contiguous in the staged
            // order); a lane finds its bead's cell among the row's H
            for (int r = warp; r < H * H; r += kDpdThreads / 32)
            for (int f = hoff[r * H] + lane; f < hoff[r * H + H]; f += 32) {
                int lo = r * H;
#pragma unroll
                for (int q = 1; q < kDpdMaxB + 2; ++q) lo += (q < H && f >= hoff[r * H + q]) ? 1 : 0;
                const int j = gst[lo] + f - hoff[lo];
                V p = sp[j];
                // the halo is H <= ncd distinct cells: shift the cells across
                // the box faces into one frame (cell edge >= 1, so beads of
                // adjacent halo cells are within r = 1 only as this image)
                const int sc = hsh[lo];
                if (sc) {
                    auto sh = [&](int c) { return c == 1 ? -L : (c == 2 ? L : (R)0); };
                    p.x += sh(sc & 3);
                    p.y += sh((sc >> 2) & 3);
                    p.z += sh(sc >> 4);
                }
                spos[f] = p;
                svel[f] = sv[j];
                if (F64) spf[f] = make_float4((float)p.x, (float)p.y, (float)p.z, 0.f);
            }
        }
        __syncthreads();
        if (staged)
            dpd_beads<R>(d, H, B3, chalo, cpre, hoff, spos, svel, spf, band, queue, atab, step, F, ec);
        else
            dpd_cells<R>(d, H, B3, chalo, hoff, gst, sp, sv, queue, atab, step, F, ec);
        __syncthreads();
    }
    double e1 = 0.5 * (double)ec, e2 = 0.5 * (double)eb;
    block_sum2(e1, e2);
    if (threadIdx.x == 0) {
        dpart[2 * bk.id] = e1;
        dpart[2 * bk.id + 1] = e2;
    }
}

template <typename R>
__global__ void __launch_bounds__(kDpdThreads, sizeof(R) == 4 ? 4 : 2)
    k_dpd(DpdDev d, int B, const typename V4<R>::T* __restrict__ sp, const typename V4<R>::T* __restrict__ sv,
          const int* __restrict__ cstart, const R* __restrict__ atab, const R* __restrict__ pos,
          const int* __restrict__ bnd, const uint64_t* __restrict__ stepp, R* __restrict__ F,
          double* __restrict__ dpart) {
    k_dpd_body<R>(d, B, sp, sv, cstart, atab, pos, bnd, stepp, F, dpart, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// The DPD pair forces and the real-space electrostatic pairs in one launch
// (horizontal fusion): blocks [0, nd) run the DPD body over the all-bead cell
// list, the others the real-space body over the charged-bead tiles. Both add
// into F (global reductions and per-bead sums) and write their own block
// partials; launched once both cell structures exist.
template <typename R>
__global__ void __launch_bounds__(kDpdThreads, sizeof(R) == 4 ? 4 : 2)
    k_pairs(DpdDev d, int B, const typename V4<R>::T* __restrict__ sp, const typename V4<R>::T* __restrict__ sv,
            const int* __restrict__ cstart, const R* __restrict__ atab, const R* __restrict__ pos,
            const int* __restrict__ bnd, const uint64_t* __restrict__ stepp, R* __restrict__ F,
            double* __restrict__ dpart, int nd, Geo g, const int* __restrict__ tstart,
            const typename V4<R>::T* __restrict__ sq, const typename V4<R>::T* __restrict__ sw,
            double* __restrict__ rpart) {
    static_assert(kDpdThreads == kRealThreads, "one block size for both roles");
    if ((int)blockIdx.x < nd)
        k_dpd_body<R>(d, B, sp, sv, cstart, atab, pos, bnd, stepp, F, dpart, Blk{(int)blockIdx.x, nd});
    else
        k_real_body<R>(g, tstart, sq, sw, F, rpart, Blk{(int)blockIdx.x - nd, (int)gridDim.x - nd});
}

// Table 2 steps 0-2 (m = 1): v0 = v + lambda F dt; v += F dt/2; r += v dt; step += 1.
template <typename R>
__global__ void k_vv_pre(int N, R lam, R dt, R* __restrict__ pos, R* __restrict__ vel, R* __restrict__ v0,
                         const R* __restrict__ F, uint64_t* __restrict__ stepp) {
    pdl_enter();
    if (blockIdx.x == 0 && threadIdx.x == 0) *stepp += 1;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 3 * N; k += gridDim.x * blockDim.x) {
        const R f = F[k];
        const R v = vel[k];
        v0[k] = v + lam * f * dt;
        const R vn = v + (R)0.5 * f * dt;
        vel[k] = vn;
        pos[k] = pos[k] + vn * dt;
    }
}

// Table 2 step 6: v += F dt/2; kinetic energy partials.
// The last block then reduces all energies of the step (totals).
template <typename R>
__global__ void __launch_bounds__(256) k_vv_post(Geo g, int N, R dt, R* __restrict__ vel, const R* __restrict__ F,
                                                double* __restrict__ kpart, TotalsArgs tot) {
    pdl_enter();
    double ke = 0.0, dummy = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 3 * N; k += gridDim.x * blockDim.x) {
        const R v = vel[k] + (R)0.5 * F[k] * dt;
        vel[k] = v;
        ke += 0.5 * (double)v * (double)v;
    }
    block_sum2(ke, dummy);
    if (threadIdx.x == 0) kpart[blockIdx.x] = ke;
    if (tot.Edev) totals_if_last(g, tot, (int)gridDim.x);
}

// Standalone totals (one CTA), for evaluations outside a step graph.
static __global__ void __launch_bounds__(1024) k_totals(Geo g, TotalsArgs t) {
    pdl_enter();
    totals_block(g, t);
}

}  // namespace enuf
