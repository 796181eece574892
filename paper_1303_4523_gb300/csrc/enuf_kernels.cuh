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

__device__ __forceinline__ float r_exp(float x) { return expf(x); }
__device__ __forceinline__ double r_exp(double x) { return exp(x); }
__device__ __forceinline__ float r_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double r_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }

// ---------------------------------------------------------------------------
// Coordinates. Wrapping and grid coordinates are computed in double with the
// exact operation sequence of the definition (no fused multiply-add), so the
// integer decisions (grid base, tile, cell) are reproducible.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double wrap_pos(double x, double L) {
    if (x >= 0.0 && x < L) return x;
    double w = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
    if (w >= L || w < 0.0) w = 0.0;
    return w;
}

template <typename R>
__device__ __forceinline__ double wrap_to_real(R x, double L) {
    double w = wrap_pos((double)x, L);
    if (sizeof(R) == 4) w = (double)__double2float_rn(w);
    return w;
}

__device__ __forceinline__ void grid_coord(double xw, double L, int n, int& base, double& frac) {
    double s = __ddiv_rn(xw, L);
    s = __dsub_rn(s, floor(s));
    double u = __dmul_rn(s, (double)n);
    if (u >= (double)n) u = __dsub_rn(u, (double)n);
    const double bb = floor(u);
    base = (int)bb;
    frac = __dsub_rn(u, bb);
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
    a = warp_sum(a);
    b = warp_sum(b);
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

// Kahan-compensated accumulator (FP64).
struct Kahan {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double x) {
        const double y = x - c;
        const double t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// ---------------------------------------------------------------------------
// a1: binning of the charged beads into tiles of the oversampled grid.
// Block-local histograms in shared memory, one scan, one scatter: the only
// atomics are shared-memory ones.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(512) k_bin_count(Geo g, int N, const R* __restrict__ pos,
                                                  const R* __restrict__ q, int* __restrict__ key,
                                                  int* __restrict__ bhist, R* __restrict__ Fzero,
                                                  double* __restrict__ qpart) {
    extern __shared__ int hist[];
    for (int t = threadIdx.x; t < g.ntiles; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    const int b = blockIdx.x;
    const int i0 = b * g.chunk;
    const int i1 = min(N, i0 + g.chunk);
    double s1 = 0.0, s2 = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const R qi = q[i];
        int kk = -1;
        if (qi != (R)0) {
            int bs[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                double fr;
                grid_coord(wrap_to_real<R>(pos[3 * i + t], g.L), g.L, g.n, bs[t], fr);
            }
            kk = ((bs[2] / g.T) * g.ntd + bs[1] / g.T) * g.ntd + bs[0] / g.T;
            atomicAdd(&hist[kk], 1);
            s1 += (double)qi;
            s2 += (double)qi * (double)qi;
        }
        key[i] = kk;
        if (Fzero) {
            Fzero[3 * i] = (R)0;
            Fzero[3 * i + 1] = (R)0;
            Fzero[3 * i + 2] = (R)0;
        }
    }
    block_sum2(s1, s2);
    if (threadIdx.x == 0) {
        qpart[2 * b] = s1;
        qpart[2 * b + 1] = s2;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < g.ntiles; t += blockDim.x) bhist[b * g.ntiles + t] = hist[t];
}

// Exclusive scan over (tile, block) in tile-major order; one CTA of 1024 threads.
static __global__ void __launch_bounds__(1024) k_bin_scan(Geo g, const int* __restrict__ bhist,
                                                   int* __restrict__ boff, int* __restrict__ tstart) {
    __shared__ int wsum[32];
    const int nt = g.ntiles, nb = g.nbin;
    const int per = (nt + blockDim.x - 1) / blockDim.x;
    const int t0 = min(nt, (int)threadIdx.x * per), t1 = min(nt, t0 + per);
    int local = 0;
    for (int t = t0; t < t1; ++t)
        for (int b = 0; b < nb; ++b) local += bhist[b * nt + t];
    // block exclusive scan of local
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    int v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (l >= o) v += u;
    }
    if (l == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        int x = wsum[l];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, x, o);
            if (l >= o) x += u;
        }
        wsum[l] = x;
    }
    __syncthreads();
    int run = v - local + (w > 0 ? wsum[w - 1] : 0);
    for (int t = t0; t < t1; ++t) {
        tstart[t] = run;
        for (int b = 0; b < nb; ++b) {
            boff[b * nt + t] = run;
            run += bhist[b * nt + t];
        }
    }
    if (threadIdx.x == blockDim.x - 1) tstart[nt] = wsum[31];
}

template <typename R>
__global__ void __launch_bounds__(512) k_bin_scatter(Geo g, int N, const R* __restrict__ pos,
                                                    const R* __restrict__ q, const int* __restrict__ key,
                                                    const int* __restrict__ boff,
                                                    typename V4<R>::T* __restrict__ sq,
                                                    typename V4<R>::T* __restrict__ sw,
                                                    int* __restrict__ sb) {
    extern __shared__ int cur[];
    const int b = blockIdx.x;
    for (int t = threadIdx.x; t < g.ntiles; t += blockDim.x) cur[t] = boff[b * g.ntiles + t];
    __syncthreads();
    const int i0 = b * g.chunk;
    const int i1 = min(N, i0 + g.chunk);
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int kk = key[i];
        if (kk < 0) continue;
        const int slot = atomicAdd(&cur[kk], 1);
        double xw[3], fr[3];
        int bs[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            xw[t] = wrap_to_real<R>(pos[3 * i + t], g.L);
            grid_coord(xw[t], g.L, g.n, bs[t], fr[t]);
        }
        typename V4<R>::T a, c;
        a.x = (R)xw[0]; a.y = (R)xw[1]; a.z = (R)xw[2]; a.w = q[i];
        c.x = (R)fr[0]; c.y = (R)fr[1]; c.z = (R)fr[2]; c.w = int_as_real(i, (R)0);
        sq[slot] = a;
        sw[slot] = c;
        sb[slot] = bs[0] | (bs[1] << 10) | (bs[2] << 20);
    }
}

// ---------------------------------------------------------------------------
// a2: spreading g(l) = sum_j q_j prod_t psi(u_jt - l_t)   (Eq. 14/19, first half)
// One CTA owns one T^3 tile of the grid: it visits the beads of the (up to)
// 27 neighbouring bins, deposits the taps that fall inside its tile into
// shared memory, and writes the finished tile once. No global atomics.
// ---------------------------------------------------------------------------
constexpr int kSpreadThreads = 256;
constexpr int kMaxTaps = 16;

template <typename R>
__global__ void __launch_bounds__(kSpreadThreads) k_spread(Geo g, const int* __restrict__ tstart,
                                                           const typename V4<R>::T* __restrict__ sq,
                                                           const typename V4<R>::T* __restrict__ sw,
                                                           const int* __restrict__ sb,
                                                           R* __restrict__ grid) {
    extern __shared__ unsigned char smraw[];
    const int T = g.T, T3 = T * T * T;
    R* acc = reinterpret_cast<R*>(smraw);
    constexpr int NW = kSpreadThreads / 32;
    R* wts = acc + T3;                                        // [NW][3][16]
    int* lix = reinterpret_cast<int*>(wts + NW * 3 * kMaxTaps); // [NW][3][16]
    __shared__ int nb_start[27], nb_pre[28];
    __shared__ int nnb;

    const int tile = blockIdx.x;
    const int tx = tile % g.ntd, ty = (tile / g.ntd) % g.ntd, tz = tile / (g.ntd * g.ntd);
    const int o[3] = {tx * T, ty * T, tz * T};
    for (int e = threadIdx.x; e < T3; e += blockDim.x) acc[e] = (R)0;
    if (threadIdx.x == 0) {
        const int no = g.ntd >= 3 ? 3 : g.ntd;
        int cnt = 0, pre = 0;
        for (int dz = 0; dz < no; ++dz)
            for (int dy = 0; dy < no; ++dy)
                for (int dx = 0; dx < no; ++dx) {
                    const int nz = g.ntd >= 3 ? (tz + dz - 1 + g.ntd) % g.ntd : dz;
                    const int ny = g.ntd >= 3 ? (ty + dy - 1 + g.ntd) % g.ntd : dy;
                    const int nx = g.ntd >= 3 ? (tx + dx - 1 + g.ntd) % g.ntd : dx;
                    const int nt = (nz * g.ntd + ny) * g.ntd + nx;
                    const int s = tstart[nt], c = tstart[nt + 1] - s;
                    nb_start[cnt] = s;
                    nb_pre[cnt] = pre;
                    pre += c;
                    ++cnt;
                }
        nb_pre[cnt] = pre;
        nnb = cnt;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    R* myw = wts + warp * 3 * kMaxTaps;
    int* myl = lix + warp * 3 * kMaxTaps;
    const int P2 = 2 * g.p;
    const int total = nb_pre[nnb];
    const R rb = (R)(1.0 / g.b), wn = (R)g.wnorm;
    for (int cand = warp; cand < total; cand += NW) {
        int k = 0;
        while (nb_pre[k + 1] <= cand) ++k;
        const int j = nb_start[k] + cand - nb_pre[k];
        const typename V4<R>::T wv = sw[j];
        const R qj = sq[j].w;
        const int pb = sb[j];
        const int base[3] = {pb & 1023, (pb >> 10) & 1023, (pb >> 20) & 1023};
        const R fr[3] = {wv.x, wv.y, wv.z};
        unsigned msk[3];
        int lw[3];
        bool inside[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            int l = base[t] - g.p + 1 + lane;
            l = l < 0 ? l + g.n : (l >= g.n ? l - g.n : l);
            lw[t] = l - o[t];
            inside[t] = lane < P2 && (unsigned)lw[t] < (unsigned)T;
            msk[t] = __ballot_sync(0xffffffffu, inside[t]);
        }
        if (!msk[0] || !msk[1] || !msk[2]) continue;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (inside[t]) {
                const int slot = __popc(msk[t] & ((1u << lane) - 1u));
                const R d = fr[t] + (R)(g.p - 1 - lane);
                myw[t * kMaxTaps + slot] = wn * r_exp(-d * d * rb);
                myl[t * kMaxTaps + slot] = lw[t];
            }
        }
        __syncwarp();
        const int cx = __popc(msk[0]), cy = __popc(msk[1]), cz = __popc(msk[2]);
        const int npt = cx * cy * cz;
        for (int s = lane; s < npt; s += 32) {
            const int ix = s % cx;
            const int r2 = s / cx;
            const int iy = r2 % cy, iz = r2 / cy;
            const R v = qj * myw[ix] * myw[kMaxTaps + iy] * myw[2 * kMaxTaps + iz];
            atomicAdd(&acc[(myl[2 * kMaxTaps + iz] * T + myl[kMaxTaps + iy]) * T + myl[ix]], v);
        }
        __syncwarp();
    }
    __syncthreads();
    const int n = g.n;
    for (int e = threadIdx.x; e < T3; e += blockDim.x) {
        const int lx = e % T, ly = (e / T) % T, lz = e / (T * T);
        grid[((size_t)(o[2] + lz) * n + (o[1] + ly)) * n + (o[0] + lx)] = acc[e];
    }
}

// ---------------------------------------------------------------------------
// a3: forward FFT pass along x (R2C, two real rows per complex line), keep
// k_x = 0..nc; output spec1[z][kx][y].
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_fft_x(Geo g, FftPlanDev fp, const R* __restrict__ grid,
                                              const typename Cx<R>::T* __restrict__ twg,
                                              typename Cx<R>::T* __restrict__ spec1, int LP) {
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc1 = g.nc + 1;
    C* tw = reinterpret_cast<C*>(smraw);
    C* b0 = tw + n;
    C* b1 = b0 + LP * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const int row0 = blockIdx.x * 2 * LP;     // first real row (z*n + y), y even
    const int nrows = n * n;
    const int nl = min(LP, (nrows - row0) / 2);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int c = idx / n, x = idx - c * n;
        C v;
        v.x = grid[(size_t)(row0 + 2 * c) * n + x];
        v.y = grid[(size_t)(row0 + 2 * c + 1) * n + x];
        b0[c * n + x] = v;
    }
    __syncthreads();
    C* res = fft_lines<R, false>(b0, b1, tw, fp, nl, n);
    // split the two real transforms: A = (Z_k + conj Z_{n-k})/2, B = -i (Z_k - conj Z_{n-k})/2
    for (int idx = threadIdx.x; idx < nl * nc1; idx += blockDim.x) {
        const int k = idx / nl, c = idx - k * nl;
        const C z = res[c * n + k];
        const C zm = res[c * n + (k == 0 ? 0 : n - k)];
        C A, B;
        A.x = (R)0.5 * (z.x + zm.x);
        A.y = (R)0.5 * (z.y - zm.y);
        B.x = (R)0.5 * (z.y + zm.y);
        B.y = (R)0.5 * (zm.x - z.x);
        const int row = row0 + 2 * c;
        const int zz = row / n, y = row - zz * n;
        C* dst = spec1 + ((size_t)zz * nc1 + k) * n + y;
        dst[0] = A;
        dst[1] = B;
    }
}

// forward pass along y for lines (z, kx), keep |ky| <= nc; output spec2[kx][ky][z]
template <typename R>
__global__ void __launch_bounds__(256) k_fft_y(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec1,
                                              const typename Cx<R>::T* __restrict__ twg,
                                              typename Cx<R>::T* __restrict__ spec2, int LB) {
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc1 = g.nc + 1, K = g.K;
    C* tw = reinterpret_cast<C*>(smraw);
    C* b0 = tw + n;
    C* b1 = b0 + LB * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const int kx = blockIdx.x;
    const int z0 = blockIdx.y * LB;
    const int nl = min(LB, n - z0);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int c = idx / n, y = idx - c * n;
        b0[c * n + y] = spec1[((size_t)(z0 + c) * nc1 + kx) * n + y];
    }
    __syncthreads();
    C* res = fft_lines<R, false>(b0, b1, tw, fp, nl, n);
    for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
        const int ki = idx / nl, c = idx - ki * nl;
        const int ky = ki - g.nc;
        spec2[((size_t)kx * K + ki) * n + z0 + c] = res[c * n + (ky < 0 ? ky + n : ky)];
    }
}

// z pass: forward z; E += w D |F|^2, W += w D v |F|^2 (FP64, Kahan);
// G_a = -i k_a D F (a = x, y, z); inverse z of each G_a; output spec3[a][z][kx][ky].
template <typename R>
__global__ void __launch_bounds__(256) k_fft_z(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec2,
                                              const typename Cx<R>::T* __restrict__ twg,
                                              const double* __restrict__ tab, const double* __restrict__ tabv,
                                              const R* __restrict__ tabr, typename Cx<R>::T* __restrict__ spec3,
                                              double* __restrict__ epart, int LB) {
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, K = g.K;
    const int NL = (nc + 1) * K;
    C* tw = reinterpret_cast<C*>(smraw);
    C* b0 = tw + n;
    C* b1 = b0 + LB * n;
    C* b2 = b1 + LB * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const int l0 = blockIdx.x * LB;
    const int nl = min(LB, NL - l0);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) b0[idx] = spec2[(size_t)l0 * n + idx];
    __syncthreads();
    C* Fh = fft_lines<R, false>(b0, b1, tw, fp, nl, n);
    C* wa = (Fh == b0) ? b1 : b0;
    C* wb = b2;
    // energy and virial of the kept modes (half space kx >= 0, kx > 0 counted twice)
    Kahan ke, kw;
    for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
        const int c = idx / K, kzi = idx - c * K;
        const int l = l0 + c;
        const int kx = l / K;
        const int kz = kzi - nc;
        const C f = Fh[c * n + (kz < 0 ? kz + n : kz)];
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
    for (int a = 0; a < 3; ++a) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
            const int c = idx / n, m = idx - c * n;
            const int kz = m <= n / 2 ? m : m - n;
            C v;
            v.x = (R)0;
            v.y = (R)0;
            if (kz >= -nc && kz <= nc) {
                const int l = l0 + c;
                const int kx = l / K, ky = (l - kx * K) - nc;
                const int ka = a == 0 ? kx : (a == 1 ? ky : kz);
                const R s = (R)ka * tabr[(size_t)l * K + (kz + nc)];
                const C f = Fh[c * n + m];
                v.x = s * f.y;     // -i s F
                v.y = -s * f.x;
            }
            wa[idx] = v;
        }
        __syncthreads();
        C* res = fft_lines<R, true>(wa, wb, tw, fp, nl, n);
        for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
            const int z = idx / nl, c = idx - z * nl;
            spec3[((size_t)a * n + z) * NL + l0 + c] = res[c * n + z];
        }
        // res is wa or wb; the next field rebuilds into wa, so keep both free
        __syncthreads();
    }
}

// inverse pass along y for lines (a, z, kx): K inputs zero-padded to n; output spec4[a][z][y][kx]
template <typename R>
__global__ void __launch_bounds__(256) k_fft_iy(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec3,
                                               const typename Cx<R>::T* __restrict__ twg,
                                               typename Cx<R>::T* __restrict__ spec4, int LB) {
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1, K = g.K;
    const int NLT = 3 * n * nc1;
    C* tw = reinterpret_cast<C*>(smraw);
    C* b0 = tw + n;
    C* b1 = b0 + LB * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const int l0 = blockIdx.x * LB;
    const int nl = min(LB, NLT - l0);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int c = idx / n, m = idx - c * n;
        const int ky = m <= n / 2 ? m : m - n;
        C v;
        v.x = (R)0;
        v.y = (R)0;
        if (ky >= -nc && ky <= nc) v = spec3[(size_t)(l0 + c) * K + (ky + nc)];
        b0[idx] = v;
    }
    __syncthreads();
    C* res = fft_lines<R, true>(b0, b1, tw, fp, nl, n);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int y = idx / nl, c = idx - y * nl;
        const int l = l0 + c;
        const int az = l / nc1, kx = l - az * nc1;
        spec4[((size_t)az * n + y) * nc1 + kx] = res[c * n + y];
    }
}

// inverse pass along x (C2R, two Hermitian rows per complex line); output h[a][z][y][x]
template <typename R>
__global__ void __launch_bounds__(256) k_fft_ix(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec4,
                                               const typename Cx<R>::T* __restrict__ twg,
                                               R* __restrict__ h, int LP) {
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1;
    const int nrows = 3 * n * n;
    C* tw = reinterpret_cast<C*>(smraw);
    C* b0 = tw + n;
    C* b1 = b0 + LP * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = twg[t];
    const int row0 = blockIdx.x * 2 * LP;
    const int nl = min(LP, (nrows - row0) / 2);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int c = idx / n, m = idx - c * n;
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
        b0[idx] = z;
    }
    __syncthreads();
    C* res = fft_lines<R, true>(b0, b1, tw, fp, nl, n);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int c = idx / n, x = idx - c * n;
        const C v = res[idx];
        h[(size_t)(row0 + 2 * c) * n + x] = v.x;
        h[(size_t)(row0 + 2 * c + 1) * n + x] = v.y;
    }
}

// ---------------------------------------------------------------------------
// a6: gather (conjugated NFFT part 2, Eq. 25). Warp per charged bead.
// ---------------------------------------------------------------------------
constexpr int kGatherThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kGatherThreads) k_gather(Geo g, const int* __restrict__ tstart,
                                                           const typename V4<R>::T* __restrict__ sq,
                                                           const typename V4<R>::T* __restrict__ sw,
                                                           const int* __restrict__ sb,
                                                           const R* __restrict__ h, R* __restrict__ F) {
    constexpr int NW = kGatherThreads / 32;
    __shared__ R wts[NW][3][kMaxTaps];
    __shared__ int lix[NW][3][kMaxTaps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Nq = tstart[g.ntiles];
    const int n = g.n;
    const size_t n3 = (size_t)n * n * n;
    const int P2 = 2 * g.p, ntap = P2 * P2 * P2;
    const R rb = (R)(1.0 / g.b), wn = (R)g.wnorm;
    const R pref = (R)(g.kappa * 2.0 / (g.L * g.L));
    for (int s = blockIdx.x * NW + warp; s < Nq; s += gridDim.x * NW) {
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
                lix[warp][t][lane] = l;
                const R d = fr[t] + (R)(g.p - 1 - lane);
                wts[warp][t][lane] = wn * r_exp(-d * d * rb);
            }
        }
        __syncwarp();
        R ax = 0, ay = 0, az = 0;
        for (int tap = lane; tap < ntap; tap += 32) {
            const int a = tap % P2;
            const int r2 = tap / P2;
            const int b = r2 % P2, c = r2 / P2;
            const R w = wts[warp][0][a] * wts[warp][1][b] * wts[warp][2][c];
            const size_t off = ((size_t)lix[warp][2][c] * n + lix[warp][1][b]) * n + lix[warp][0][a];
            ax += w * h[off];
            ay += w * h[n3 + off];
            az += w * h[2 * n3 + off];
        }
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
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// a7 (electrostatic part): real-space erfc + Slater-correction pairs on the
// tile bins (Eq. 31, corrected Eq. 32, Eq. 27-28). Warp per charged bead; lanes
// stride over the candidates of each contiguous run of tiles.
// ---------------------------------------------------------------------------
constexpr int kRealThreads = 256;

__device__ __forceinline__ void stencil_dim(int t, int rs, int ntd, int& lo, int& cnt, bool& whole) {
    whole = 2 * rs + 1 >= ntd;
    if (whole) { lo = 0; cnt = ntd; }
    else { lo = t - rs; cnt = 2 * rs + 1; }
}

template <typename R>
__global__ void __launch_bounds__(kRealThreads) k_real(Geo g, const int* __restrict__ tstart,
                                                       const typename V4<R>::T* __restrict__ sq,
                                                       const typename V4<R>::T* __restrict__ sw,
                                                       const int* __restrict__ sb,
                                                       R* __restrict__ F, double* __restrict__ rpart) {
    constexpr int NW = kRealThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Nq = tstart[g.ntiles];
    const R L = (R)g.L, hL = (R)(0.5 * g.L);
    const R rc2 = (R)(g.rc * g.rc);
    const R al = (R)g.alpha, c2a = (R)(2.0 * g.alpha / 1.7724538509055160273);
    const R be = (R)g.beta;
    const bool slater = g.beta > 0.0;
    double eacc = 0.0, wacc = 0.0;
    for (int s = blockIdx.x * NW + warp; s < Nq; s += gridDim.x * NW) {
        const typename V4<R>::T pi = sq[s];
        const int pb = sb[s];
        const int tx = (pb & 1023) / g.T, ty = ((pb >> 10) & 1023) / g.T, tz = ((pb >> 20) & 1023) / g.T;
        R fx = 0, fy = 0, fz = 0;
        int zlo, zc, ylo, yc, xlo, xc;
        bool zw, yw, xw;
        stencil_dim(tz, g.rs, g.ntd, zlo, zc, zw);
        stencil_dim(ty, g.rs, g.ntd, ylo, yc, yw);
        stencil_dim(tx, g.rs, g.ntd, xlo, xc, xw);
        for (int iz = 0; iz < zc; ++iz) {
            const int nz = (zlo + iz + g.ntd) % g.ntd;
            for (int iy = 0; iy < yc; ++iy) {
                const int ny = (ylo + iy + g.ntd) % g.ntd;
                const int rowbase = (nz * g.ntd + ny) * g.ntd;
                // the x run is contiguous unless it wraps: at most two ranges
                int r0s[2], r0e[2], nr;
                if (xw) {
                    r0s[0] = tstart[rowbase]; r0e[0] = tstart[rowbase + g.ntd]; nr = 1;
                } else if (xlo >= 0 && xlo + xc <= g.ntd) {
                    r0s[0] = tstart[rowbase + xlo]; r0e[0] = tstart[rowbase + xlo + xc]; nr = 1;
                } else if (xlo < 0) {
                    r0s[0] = tstart[rowbase + xlo + g.ntd]; r0e[0] = tstart[rowbase + g.ntd];
                    r0s[1] = tstart[rowbase]; r0e[1] = tstart[rowbase + xlo + xc]; nr = 2;
                } else {
                    r0s[0] = tstart[rowbase + xlo]; r0e[0] = tstart[rowbase + g.ntd];
                    r0s[1] = tstart[rowbase]; r0e[1] = tstart[rowbase + xlo + xc - g.ntd]; nr = 2;
                }
                for (int rr = 0; rr < nr; ++rr) {
                    for (int j = r0s[rr] + lane; j < r0e[rr]; j += 32) {
                        if (j == s) continue;
                        const typename V4<R>::T pj = sq[j];
                        const R dx = min_image(pi.x, pj.x, L, hL);
                        const R dy = min_image(pi.y, pj.y, L, hL);
                        const R dz = min_image(pi.z, pj.z, L, hL);
                        const R r2 = dist2(dx, dy, dz);
                        if (!(r2 < rc2) || r2 <= (R)0) continue;
                        const R r = r_sqrt(r2);
                        const R ir = (R)1 / r;
                        const R ar = al * r;
                        const R ec = r_erfc(ar);
                        R u = ec * ir;
                        R f = ec * ir * ir + c2a * r_exp(-ar * ar) * ir;
                        if (slater) {
                            const R br = be * r;
                            const R e2 = r_exp((R)-2 * br);
                            u -= ((R)1 + br) * e2 * ir;
                            f -= ((R)1 + (R)2 * br + (R)2 * br * br) * e2 * ir * ir;
                        }
                        const R qq = (R)g.kappa * pi.w * pj.w;
                        const R fm = qq * f * ir;
                        fx += fm * dx;
                        fy += fm * dy;
                        fz += fm * dz;
                        eacc += 0.5 * (double)(qq * u);
                        wacc += 0.5 * (double)(qq * f * r);
                    }
                }
            }
        }
        fx = warp_sum_r(fx);
        fy = warp_sum_r(fy);
        fz = warp_sum_r(fz);
        if (lane == 0) {
            const int i = real_as_int(sw[s].w);
            F[3 * i] += fx;
            F[3 * i + 1] += fy;
            F[3 * i + 2] += fz;
        }
    }
    block_sum2(eacc, wacc);
    if (threadIdx.x == 0) {
        rpart[2 * blockIdx.x] = eacc;
        rpart[2 * blockIdx.x + 1] = wacc;
    }
}

// ---------------------------------------------------------------------------
// DPD: cell list of all beads (edge >= 1) by a counting sort.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_cell_count(int N, int ncd, double L, const R* __restrict__ pos, int* __restrict__ ckey,
                             int* __restrict__ ccount) {
    const double inv = (double)ncd / L;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        int c[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            int v = (int)floor(wrap_to_real<R>(pos[3 * i + t], L) * inv);
            c[t] = v < 0 ? 0 : (v >= ncd ? ncd - 1 : v);
        }
        const int cell = (c[2] * ncd + c[1]) * ncd + c[0];
        ckey[i] = cell;
        atomicAdd(&ccount[cell], 1);
    }
}

static __global__ void __launch_bounds__(1024) k_cell_scan(int ncells, int* __restrict__ ccount,
                                                    int* __restrict__ cstart, int* __restrict__ ccur) {
    __shared__ int wsum[32];
    const int per = (ncells + blockDim.x - 1) / blockDim.x;
    const int t0 = min(ncells, (int)threadIdx.x * per), t1 = min(ncells, t0 + per);
    int local = 0;
    for (int t = t0; t < t1; ++t) local += ccount[t];
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    int v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (l >= o) v += u;
    }
    if (l == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        int x = wsum[l];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, x, o);
            if (l >= o) x += u;
        }
        wsum[l] = x;
    }
    __syncthreads();
    int run = v - local + (w > 0 ? wsum[w - 1] : 0);
    for (int t = t0; t < t1; ++t) {
        cstart[t] = run;
        ccur[t] = run;
        run += ccount[t];
        ccount[t] = 0;   // ready for the next step
    }
    if (threadIdx.x == blockDim.x - 1) cstart[ncells] = wsum[31];
}

template <typename R>
__global__ void k_cell_scatter(int N, double L, const R* __restrict__ pos, const R* __restrict__ v0,
                               const int* __restrict__ type, const int* __restrict__ ckey,
                               int* __restrict__ ccur, typename V4<R>::T* __restrict__ sp,
                               typename V4<R>::T* __restrict__ sv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int slot = atomicAdd(&ccur[ckey[i]], 1);
        typename V4<R>::T a, b;
        a.x = (R)wrap_to_real<R>(pos[3 * i], L);
        a.y = (R)wrap_to_real<R>(pos[3 * i + 1], L);
        a.z = (R)wrap_to_real<R>(pos[3 * i + 2], L);
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
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return c0;
}

// theta_ij of Eq. 5: uniform on [-sqrt3, sqrt3], counter (min, max, step), key = seed.
template <typename R>
__device__ __forceinline__ R dpd_theta(uint64_t seed, uint64_t step, int i, int j) {
    const uint32_t lo = (uint32_t)min(i, j), hi = (uint32_t)max(i, j);
    const uint32_t w = philox_word0(lo, hi, (uint32_t)step, (uint32_t)(step >> 32), (uint32_t)seed,
                                    (uint32_t)(seed >> 32));
    const R u = ((R)w + (R)0.5) * (R)2.3283064365386962890625e-10;  // 2^-32
    return (R)1.7320508075688772935 * ((R)2 * u - (R)1);
}

// DPD pair forces (Eq. 2-7, R_c = 1) + bonds (Sec. 2); thread per bead in
// cell order; F[i] = F^C + F^D + F^R/sqrt(dt) + F^S (overwrites F).
template <typename R>
__global__ void __launch_bounds__(256) k_dpd(DpdDev d, const typename V4<R>::T* __restrict__ sp,
                                            const typename V4<R>::T* __restrict__ sv,
                                            const int* __restrict__ ckey, const int* __restrict__ cstart,
                                            const R* __restrict__ atab, const R* __restrict__ pos,
                                            const int* __restrict__ bptr, const int* __restrict__ blist,
                                            const uint64_t* __restrict__ stepp, R* __restrict__ F,
                                            double* __restrict__ dpart) {
    const R L = (R)d.L, hL = (R)(0.5 * d.L);
    const R gam = (R)d.gamma, sig = (R)d.sigma, rdt = (R)(1.0 / sqrt(d.dt));
    const R Kb = (R)d.K_bond, r0b = (R)d.r0_bond;
    const uint64_t step = *stepp;
    const int ncd = d.ncd;
    double ec = 0.0, eb = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.N; s += gridDim.x * blockDim.x) {
        const typename V4<R>::T pi = sp[s];
        const typename V4<R>::T vi = sv[s];
        const int i = real_as_int(pi.w), ti = real_as_int(vi.w);
        const int cell = ckey[i];
        const int cx = cell % ncd, cy = (cell / ncd) % ncd, cz = cell / (ncd * ncd);
        R fx = 0, fy = 0, fz = 0;
        const int no = ncd >= 3 ? 3 : ncd;
        for (int dz = 0; dz < no; ++dz) {
            const int nz = ncd >= 3 ? (cz + dz - 1 + ncd) % ncd : dz;
            for (int dy = 0; dy < no; ++dy) {
                const int ny = ncd >= 3 ? (cy + dy - 1 + ncd) % ncd : dy;
                for (int dx = 0; dx < no; ++dx) {
                    const int nx = ncd >= 3 ? (cx + dx - 1 + ncd) % ncd : dx;
                    const int nb = (nz * ncd + ny) * ncd + nx;
                    const int e = cstart[nb + 1];
                    for (int j = cstart[nb]; j < e; ++j) {
                        if (j == s) continue;
                        const typename V4<R>::T pj = sp[j];
                        const R rx = min_image(pi.x, pj.x, L, hL);
                        const R ry = min_image(pi.y, pj.y, L, hL);
                        const R rz = min_image(pi.z, pj.z, L, hL);
                        const R r2 = dist2(rx, ry, rz);
                        if (!(r2 < (R)1) || r2 <= (R)0) continue;
                        const typename V4<R>::T vj = sv[j];
                        const int jj = real_as_int(pj.w), tj = real_as_int(vj.w);
                        const R r = r_sqrt(r2);
                        const R ir = (R)1 / r;
                        const R ex = rx * ir, ey = ry * ir, ez = rz * ir;
                        const R w = (R)1 - r;
                        const R a = atab[ti * d.ntypes + tj];
                        const R vr = (vi.x - vj.x) * ex + (vi.y - vj.y) * ey + (vi.z - vj.z) * ez;
                        const R th = dpd_theta<R>(d.seed, step, i, jj);
                        const R fm = a * w - gam * w * w * vr + sig * w * th * rdt;
                        fx += fm * ex;
                        fy += fm * ey;
                        fz += fm * ez;
                        ec += 0.25 * (double)(a * w * w);
                    }
                }
            }
        }
        // harmonic bonds
        for (int k = bptr[i]; k < bptr[i + 1]; ++k) {
            const int j = blist[k];
            R dd[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const R xi = (R)wrap_to_real<R>(pos[3 * i + t], d.L);
                const R xj = (R)wrap_to_real<R>(pos[3 * j + t], d.L);
                dd[t] = min_image(xi, xj, L, hL);
            }
            const R r = r_sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
            eb += 0.25 * (double)(Kb * (r - r0b) * (r - r0b));
            if (r > (R)0) {
                const R fm = -Kb * (r - r0b) / r;
                fx += fm * dd[0];
                fy += fm * dd[1];
                fz += fm * dd[2];
            }
        }
        F[3 * i] = fx;
        F[3 * i + 1] = fy;
        F[3 * i + 2] = fz;
    }
    block_sum2(ec, eb);
    if (threadIdx.x == 0) {
        dpart[2 * blockIdx.x] = ec;
        dpart[2 * blockIdx.x + 1] = eb;
    }
}

// Table 2 steps 0-2 (m = 1): v0 = v + lambda F dt; v += F dt/2; r += v dt; step += 1.
template <typename R>
__global__ void k_vv_pre(int N, R lam, R dt, R* __restrict__ pos, R* __restrict__ vel, R* __restrict__ v0,
                         const R* __restrict__ F, uint64_t* __restrict__ stepp) {
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
template <typename R>
__global__ void __launch_bounds__(256) k_vv_post(int N, R dt, R* __restrict__ vel, const R* __restrict__ F,
                                                double* __restrict__ kpart) {
    double ke = 0.0, dummy = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 3 * N; k += gridDim.x * blockDim.x) {
        const R v = vel[k] + (R)0.5 * F[k] * dt;
        vel[k] = v;
        ke += 0.5 * (double)v * (double)v;
    }
    block_sum2(ke, dummy);
    if (threadIdx.x == 0) kpart[blockIdx.x] = ke;
}

// Final FP64 totals (Kahan over the per-block partials), one CTA of 256 threads.
// Edev: [0] E_real [1] E_recip [2] E_self+E_neutral [3] E_elec [4] E_conservative
//       [5] E_bond [6] E_kinetic [7] virial_elec
static __global__ void __launch_bounds__(256) k_totals(Geo g, const double* __restrict__ part, int off_q, int nq,
                                               int off_real, int nreal, int off_recip, int nrecip,
                                               int off_dpd, int ndpd, int off_kin, int nkin,
                                               double* __restrict__ Edev) {
    __shared__ double vals[16];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    // warp w reduces quantity w: 0 sum q, 1 sum q^2, 2 E_real, 3 W_real, 4 E_k, 5 W_k, 6 E_c, 7 E_b
    if (w < 8) {
        int off, cnt, stride = 2, sub = w & 1;
        if (w < 2) { off = off_q; cnt = nq; }
        else if (w < 4) { off = off_real; cnt = nreal; }
        else if (w < 6) { off = off_recip; cnt = nrecip; }
        else { off = off_dpd; cnt = ndpd; }
        Kahan k;
        for (int i = l; i < cnt; i += 32) k.add(part[off + stride * i + sub]);
        double v = warp_sum(k.s);
        if (l == 0) vals[w] = v;
    }
    if (w == 0) {
        Kahan k;
        for (int i = l; i < nkin; i += 32) k.add(part[off_kin + i]);
        const double v = warp_sum(k.s);
        if (l == 0) vals[8] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double pi = 3.14159265358979323846;
        const double V = g.L * g.L * g.L;
        const double Q = vals[0], Q2 = vals[1];
        const double e_self = -g.kappa * g.alpha / sqrt(pi) * Q2;
        const double e_neut = -g.kappa * pi * Q * Q / (2.0 * V * g.alpha * g.alpha);
        const double pk = g.kappa / (2.0 * pi * g.L);
        const double e_real = vals[2], e_recip = pk * vals[4];
        Edev[0] = e_real;
        Edev[1] = e_recip;
        Edev[2] = e_self + e_neut;
        Edev[3] = e_real + e_recip + e_self + e_neut;
        Edev[4] = vals[6];
        Edev[5] = vals[7];
        Edev[6] = vals[8];
        Edev[7] = vals[3] + pk * vals[5] + 3.0 * e_neut;
        for (int i = 8; i < 16; ++i) Edev[i] = 0.0;
    }
}

}  // namespace enuf
