// enuf_fft2.cuh -- the FFT passes of the NFFT (Sec. 3.3; the plain FFT inside
// the transposed and conjugated NFFT of Eq. 13-14) on the two-factor line
// transform of enuf_fft.cuh, for FP32 grids whose n = f1 f2 splits into two
// of its radices. Same passes, layouts and results as the Stockham kernels of
// enuf_kernels.cuh (which serve every other n and FP64):
//   k2_fft_x  : forward R2C along x (two real rows per complex line), keep kx <= nc
//   k2_fft_y  : forward along y, keep |ky| <= nc
//   k2_fft_z  : forward along z, influence x deconvolution, FP64 energy and
//               virial, the nf force fields, their inverse along z
//   k2_fft_iy : inverse along y (zero-padded)
//   k2_fft_ix : inverse C2R along x (two Hermitian rows per complex line)
//   k2_fft_xy / k2_fft_yx : the x+y and y+x passes of one z-plane in shared
//               memory (small grids)
// The x, z (five-pass layout) and inverse x passes run persistent CTAs over
// groups of lines whose input is one contiguous run of memory: the next
// group's input is copied into shared memory asynchronously (cp.async, double
// buffered) while the current group is transformed, and phase A reads it from
// there. The y and inverse y passes and the fused plane kernels load phase A's
// elements straight from global memory. Phase B writes the natural-order
// results to a shared buffer, from which the pass writes its output in the
// layout the next pass reads contiguously.
#pragma once
#include "enuf_kernels.cuh"

namespace enuf {

// Persistent CTAs over groups of LP line pairs (2 LP consecutive real rows,
// one contiguous run of the grid), the next group's rows copied into shared
// memory asynchronously while the current group is transformed.
template <typename R>
__global__ void __launch_bounds__(512) k2_fft_x(Geo g, FftPlanDev fp, const R* __restrict__ grid,
                                               const typename Cx<R>::T* __restrict__ twg,
                                               typename Cx<R>::T* __restrict__ spec1, int LP) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1, lsb = fft2_lsb(n);
    const int npairs = n * n / 2, ngroups = (npairs + LP - 1) / LP, per = 2 * LP * n;
    C* tw = reinterpret_cast<C*>(smraw);
    C* A = tw + n;
    C* B = A + LP * fft2_lsa(fp.f1, fp.f2);
    R* In = reinterpret_cast<R*>((reinterpret_cast<size_t>(B + LP * lsb) + 15) & ~(size_t)15);   // [2][per]
    fft2_twiddles(tw, twg, fp);
    auto prefetch = [&](int grp, int buf) {
        const int nl = min(LP, npairs - grp * LP);
        cp_async_block(In + buf * per, grid + (size_t)grp * per, 2 * nl * n * (int)sizeof(R));
        cp_async_commit();
    };
    int buf = 0;
    if (blockIdx.x < ngroups) prefetch(blockIdx.x, 0);
    const float rn = 1.0f / (float)n;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x, buf ^= 1) {
        const int nxt = grp + gridDim.x;
        if (nxt < ngroups) prefetch(nxt, buf ^ 1);
        else cp_async_commit();
        cp_async_wait_prior();
        __syncthreads();
        const R* src = In + buf * per;
        const int row0 = grp * 2 * LP;   // first real row (z n + y), y even
        const int nl = min(LP, npairs - grp * LP);
        fft2_lines<R, false>(
            A, tw, fp, nl,
            [&](int c, int x) {
                C v;
                v.x = src[(2 * c) * n + x];
                v.y = src[(2 * c + 1) * n + x];
                return v;
            },
            [&](int c, int k, C v) {
                if (k <= nc || k >= n - nc) B[c * lsb + k] = v;
            });
        __syncthreads();
        // split the two real transforms: A = (Z_k + conj Z_{n-k})/2, B = -i (Z_k - conj Z_{n-k})/2
        const float rnl = 1.0f / (float)max(nl, 1);
        for (int idx = threadIdx.x; idx < nl * nc1; idx += blockDim.x) {
            const int k = qdiv(idx, nl, rnl), c = idx - k * nl;
            const C z = B[c * lsb + k];
            const C zm = B[c * lsb + (k == 0 ? 0 : n - k)];
            C a, b;
            a.x = (R)0.5 * (z.x + zm.x);
            a.y = (R)0.5 * (z.y - zm.y);
            b.x = (R)0.5 * (z.y + zm.y);
            b.y = (R)0.5 * (zm.x - z.x);
            const int row = row0 + 2 * c;
            const int zz = qdiv(row, n, rn), y = row - zz * n;
            C* dst = spec1 + ((size_t)zz * nc1 + k) * n + y;
            dst[0] = a;
            dst[1] = b;
        }
        __syncthreads();
    }
    cp_async_wait_all();
}

// forward y for lines (z, kx): spec1[z][kx][y] -> spec2[kx][ky][z], |ky| <= nc
template <typename R>
__global__ void __launch_bounds__(512) k2_fft_y(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec1,
                                               const typename Cx<R>::T* __restrict__ twg,
                                               typename Cx<R>::T* __restrict__ spec2, int LB) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1, K = g.K, lsb = fft2_lsb(n);
    C* tw = reinterpret_cast<C*>(smraw);
    C* A = tw + n;
    C* B = A + LB * fft2_lsa(fp.f1, fp.f2);
    fft2_twiddles(tw, twg, fp);
    const int kx = blockIdx.x;
    const int z0 = blockIdx.y * LB;
    const int nl = min(LB, n - z0);
    __syncthreads();
    fft2_lines<R, false>(
        A, tw, fp, nl, [&](int c, int y) { return spec1[((size_t)(z0 + c) * nc1 + kx) * n + y]; },
        [&](int c, int k, C v) {
            if (k <= nc || k >= n - nc) B[c * lsb + k] = v;
        });
    __syncthreads();
    const float rnl = 1.0f / (float)max(nl, 1);
    for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
        const int ki = qdiv(idx, nl, rnl), c = idx - ki * nl;
        const int ky = ki - nc;
        spec2[((size_t)kx * K + ki) * n + z0 + c] = B[c * lsb + (ky < 0 ? ky + n : ky)];
    }
}

// z pass: forward z of lines l = (kx, ky); E += w D |F|^2 and W += w D v |F|^2
// (FP64, Kahan); the nf fields -i k_a D F (gradient mode: D F), inverse z;
// output spec3[a][z][kx][ky]. kx and ky are constant along a z line, so the
// x and y fields are kx G and ky G of one transform G = IFFT_z(-i D F): with
// nf = 3 a line takes two inverse transforms (G and IFFT_z(-i kz D F)), built
// in the inverse transform's loader.
// The z pass of lines l0 .. l0 + nl - 1 (tw filled, A and B as below): forward
// transform of the lines (elements from load(c, z)), the energy and virial
// sums of their kept modes added to se, sv, the inverse transforms, and the
// fields written to spec3. Contains __syncthreads (call from all threads).
template <typename R, typename Load>
__device__ __forceinline__ void k2_z_lines(const Geo& g, const FftPlanDev& fp, const typename Cx<R>::T* tw,
                                           typename Cx<R>::T* A, typename Cx<R>::T* B, int l0, int nl, Load&& load,
                                           const double* __restrict__ tab, const double* __restrict__ tabv,
                                           const R* __restrict__ tabr, typename Cx<R>::T* __restrict__ spec3,
                                           double& se, double& sv) {
    using C = typename Cx<R>::T;
    const int n = g.n, nc = g.nc, K = g.K, nf = g.nf, lsb = fft2_lsb(n);
    const int NL = (nc + 1) * K;
    const int ni = nf == 3 ? 2 : 1;   // inverse transforms per line
    fft2_lines<R, false>(A, tw, fp, nl, load, [&](int c, int k, C v) {
        if (k <= nc || k >= n - nc) B[c * lsb + k] = v;
    });
    __syncthreads();
    // energy and virial of the kept modes (half space kx >= 0, kx > 0 counted twice);
    // each thread adds a few modes in plain FP64 (the FP64 units are few), the
    // compensated summation runs over the blocks' partials in the totals
    const float rK = 1.0f / (float)K;
    for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
        const int c = qdiv(idx, K, rK), kzi = idx - c * K;
        const int l = l0 + c;
        const int kx = qdiv(l, K, rK);
        const int kz = kzi - nc;
        const C f = B[c * lsb + (kz < 0 ? kz + n : kz)];
        double a2 = fma((double)f.x, (double)f.x, (double)f.y * (double)f.y);
        if (kx != 0) a2 += a2;   // the -kx half space
        se = fma(tab[(size_t)l * K + kzi], a2, se);
        sv = fma(tabv[(size_t)l * K + kzi], a2, sv);
    }
    // inverse transforms of every line: line b nl + c of the batch (b = 0: G,
    // or D F in gradient mode; b = 1: Gz)
    fft2_lines<R, true>(
        A, tw, fp, ni * nl,
        [&](int line, int m) {
            const int b = line >= nl ? 1 : 0;
            const int c = line - b * nl;
            const int kz = m <= n / 2 ? m : m - n;
            C v;
            v.x = (R)0;
            v.y = (R)0;
            if (kz >= -nc && kz <= nc) {
                const R d = tabr[(size_t)(l0 + c) * K + (kz + nc)];
                const C f = B[c * lsb + m];
                if (nf == 1) {
                    v.x = d * f.x;   // D F
                    v.y = d * f.y;
                } else {
                    const R s = b == 0 ? d : (R)kz * d;
                    v.x = s * f.y;   // -i D F, -i kz D F
                    v.y = -s * f.x;
                }
            }
            return v;
        },
        [&](int line, int z, C v) { B[line * lsb + z] = v; });
    __syncthreads();
    // B no longer holds the forward result: phase B of the inverse read A only
    const int per = nl * n;
    const float rper = 1.0f / (float)per, rnl = 1.0f / (float)max(nl, 1);
    for (int idx = threadIdx.x; idx < nf * per; idx += blockDim.x) {
        const int a = qdiv(idx, per, rper), e = idx - a * per;
        const int z = qdiv(e, nl, rnl), c = e - z * nl;
        C v = B[((a == 2 ? nl : 0) + c) * lsb + z];
        if (nf == 3 && a < 2) {   // kx G, ky G
            const int l = l0 + c;
            const int kx = qdiv(l, K, rK);
            const R ka = (R)(a == 0 ? kx : (l - kx * K) - nc);
            v.x *= ka;
            v.y *= ka;
        }
        spec3[((size_t)a * n + z) * NL + l0 + c] = v;
    }
}

template <typename R>
__device__ __forceinline__ void k2_fft_z_body(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec2,
                                               const typename Cx<R>::T* __restrict__ twg,
                                               const double* __restrict__ tab, const double* __restrict__ tabv,
                                               const R* __restrict__ tabr, typename Cx<R>::T* __restrict__ spec3,
                                               double* __restrict__ epart, int LB, int plane_major, Blk blk) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, NL = (g.nc + 1) * g.K;
    const int ni = g.nf == 3 ? 2 : 1;
    C* tw = reinterpret_cast<C*>(smraw);
    C* A = tw + n;                                    // [ni LB] phase-A rows
    C* B = A + ni * LB * fft2_lsa(fp.f1, fp.f2);     // [ni LB][lsb]: forward result, then G (and Gz)
    fft2_twiddles(tw, twg, fp);
    const int l0 = blk.id * LB;
    const int nl = min(LB, NL - l0);
    __syncthreads();
    double se = 0.0, sv = 0.0;
    if (plane_major)   // spec2[z][l]: lines gathered across planes
        k2_z_lines<R>(g, fp, tw, A, B, l0, nl, [&](int c, int z) { return spec2[(size_t)z * NL + l0 + c]; }, tab,
                      tabv, tabr, spec3, se, sv);
    else               // spec2[l][z]: lines contiguous
        k2_z_lines<R>(g, fp, tw, A, B, l0, nl, [&](int c, int z) { return spec2[(size_t)(l0 + c) * n + z]; }, tab,
                      tabv, tabr, spec3, se, sv);
    block_sum2(se, sv);
    if (threadIdx.x == 0) {
        epart[2 * blk.id] = se;
        epart[2 * blk.id + 1] = sv;
    }
}

template <typename R>
__global__ void __launch_bounds__(512) k2_fft_z(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec2,
                                               const typename Cx<R>::T* __restrict__ twg,
                                               const double* __restrict__ tab, const double* __restrict__ tabv,
                                               const R* __restrict__ tabr, typename Cx<R>::T* __restrict__ spec3,
                                               double* __restrict__ epart, int LB, int plane_major) {
    k2_fft_z_body<R>(g, fp, spec2, twg, tab, tabv, tabr, spec3, epart, LB, plane_major, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// The z pass over lines contiguous in spec2 ([l][z], the five-pass layout) with
// persistent CTAs: groups of LB lines, the next group's lines copied into
// shared memory asynchronously while this one is transformed; one energy
// partial per CTA.
template <typename R>
__global__ void __launch_bounds__(512) k2_fft_zp(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec2,
                                                const typename Cx<R>::T* __restrict__ twg,
                                                const double* __restrict__ tab, const double* __restrict__ tabv,
                                                const R* __restrict__ tabr, typename Cx<R>::T* __restrict__ spec3,
                                                double* __restrict__ epart, int LB) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = g.n, NL = (g.nc + 1) * g.K, lsb = fft2_lsb(n);
    const int ni = g.nf == 3 ? 2 : 1;
    const int ngroups = (NL + LB - 1) / LB, per = LB * n;
    C* tw = reinterpret_cast<C*>(smraw);
    C* A = tw + n;
    C* B = A + ni * LB * fft2_lsa(fp.f1, fp.f2);
    C* In = reinterpret_cast<C*>((reinterpret_cast<size_t>(B + ni * LB * lsb) + 15) & ~(size_t)15);   // [2][per]
    fft2_twiddles(tw, twg, fp);
    auto prefetch = [&](int grp, int buf) {
        const int nl = min(LB, NL - grp * LB);
        cp_async_block(In + buf * per, spec2 + (size_t)grp * per, nl * n * (int)sizeof(C));
        cp_async_commit();
    };
    int buf = 0;
    if (blockIdx.x < ngroups) prefetch(blockIdx.x, 0);
    double se = 0.0, sv = 0.0;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x, buf ^= 1) {
        const int nxt = grp + gridDim.x;
        if (nxt < ngroups) prefetch(nxt, buf ^ 1);
        else cp_async_commit();
        cp_async_wait_prior();
        __syncthreads();
        const C* Ig = In + buf * per;
        const int l0 = grp * LB, nl = min(LB, NL - l0);
        k2_z_lines<R>(g, fp, tw, A, B, l0, nl, [&](int c, int z) { return Ig[c * n + z]; }, tab, tabv, tabr, spec3,
                      se, sv);
        __syncthreads();
    }
    cp_async_wait_all();
    block_sum2(se, sv);
    if (threadIdx.x == 0) {
        epart[2 * blockIdx.x] = se;
        epart[2 * blockIdx.x + 1] = sv;
    }
}

// inverse y for lines (a, z, kx): K inputs zero-padded to n; output spec4[a][z][y][kx]
template <typename R>
__global__ void __launch_bounds__(512) k2_fft_iy(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec3,
                                                const typename Cx<R>::T* __restrict__ twg,
                                                typename Cx<R>::T* __restrict__ spec4, int LB) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1, K = g.K, lsb = fft2_lsb(n);
    const int NLT = g.nf * n * nc1;
    C* tw = reinterpret_cast<C*>(smraw);
    C* A = tw + n;
    C* B = A + LB * fft2_lsa(fp.f1, fp.f2);
    fft2_twiddles(tw, twg, fp);
    const int l0 = blockIdx.x * LB;
    const int nl = min(LB, NLT - l0);
    __syncthreads();
    fft2_lines<R, true>(
        A, tw, fp, nl,
        [&](int c, int m) {
            const int ky = m <= n / 2 ? m : m - n;
            C v;
            v.x = (R)0;
            v.y = (R)0;
            if (ky >= -nc && ky <= nc) v = spec3[(size_t)(l0 + c) * K + (ky + nc)];
            return v;
        },
        [&](int c, int y, C v) { B[c * lsb + y] = v; });
    __syncthreads();
    const float rnl = 1.0f / (float)max(nl, 1), rnc1 = 1.0f / (float)nc1;
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int y = qdiv(idx, nl, rnl), c = idx - y * nl;
        const int l = l0 + c;
        const int az = qdiv(l, nc1, rnc1), kx = l - az * nc1;
        spec4[((size_t)az * n + y) * nc1 + kx] = B[c * lsb + y];
    }
}

// inverse x (C2R, two Hermitian rows per complex line); output h[a][z][y][x].
// Persistent CTAs over groups of LP line pairs: the 2 LP input rows of a group
// are one contiguous run of spec4 (2 LP nc1 values, a multiple of 16 bytes at a
// 16-byte offset), copied into shared memory with asynchronous 16-byte copies
// one group ahead, so a group's transform runs while the next group's rows are
// in flight (the pass was bound by the latency of its loads).
template <typename R>
__global__ void __launch_bounds__(512) k2_fft_ix(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec4,
                                                const typename Cx<R>::T* __restrict__ twg, R* __restrict__ h,
                                                int LP) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1, lsb = fft2_lsb(n);
    const int npairs = g.nf * n * n / 2;
    const int ngroups = (npairs + LP - 1) / LP;
    const int per = 2 * LP * nc1;   // input values of a group
    C* tw = reinterpret_cast<C*>(smraw);
    C* A = tw + n;
    C* B = A + LP * fft2_lsa(fp.f1, fp.f2);
    C* In = reinterpret_cast<C*>((reinterpret_cast<size_t>(B + LP * lsb) + 15) & ~(size_t)15);   // [2][per]
    fft2_twiddles(tw, twg, fp);
    auto prefetch = [&](int grp, int buf) {
        const int nl = min(LP, npairs - grp * LP);
        cp_async_block(In + buf * per, spec4 + (size_t)grp * per, 2 * nl * nc1 * (int)sizeof(C));
        cp_async_commit();
    };
    int buf = 0;
    if (blockIdx.x < ngroups) prefetch(blockIdx.x, 0);
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x, buf ^= 1) {
        const int nxt = grp + gridDim.x;
        if (nxt < ngroups) prefetch(nxt, buf ^ 1);
        else cp_async_commit();   // an empty group keeps the count of groups in flight
        cp_async_wait_prior();    // this group's rows have arrived (the next may be in flight)
        __syncthreads();
        const C* Ig = In + buf * per;
        const int row0 = grp * 2 * LP;
        const int nl = min(LP, npairs - grp * LP);
        fft2_lines<R, true>(
            A, tw, fp, nl,
            [&](int c, int m) {
                const C* ra = Ig + 2 * c * nc1;
                const C* rb = ra + nc1;
                C a, b;
                a.x = a.y = b.x = b.y = (R)0;
                if (m == 0) {
                    a.x = ra[0].x;
                    b.x = rb[0].x;
                } else if (m <= nc) {
                    a = ra[m];
                    b = rb[m];
                } else if (m >= n - nc) {
                    a = ra[n - m];
                    a.y = -a.y;
                    b = rb[n - m];
                    b.y = -b.y;
                }
                C z;
                z.x = a.x - b.y;   // A + i B
                z.y = a.y + b.x;
                return z;
            },
            [&](int c, int x, C v) { B[c * lsb + x] = v; });
        __syncthreads();
        // two consecutive x per thread (n is even): one 8-byte store on each row
        const int hn = n / 2;
        const float rhn = 1.0f / (float)hn;
        for (int idx = threadIdx.x; idx < nl * hn; idx += blockDim.x) {
            const int c = qdiv(idx, hn, rhn), x = 2 * (idx - c * hn);
            const C v0 = B[c * lsb + x], v1 = B[c * lsb + x + 1];
            typename Cx<R>::T ra, rb;   // (row 2c, row 2c + 1) at x, x + 1
            ra.x = v0.x;
            ra.y = v1.x;
            rb.x = v0.y;
            rb.y = v1.y;
            *reinterpret_cast<typename Cx<R>::T*>(h + (size_t)(row0 + 2 * c) * n + x) = ra;
            *reinterpret_cast<typename Cx<R>::T*>(h + (size_t)(row0 + 2 * c + 1) * n + x) = rb;
        }
        __syncthreads();   // A, B and this buffer are free for the next group
    }
    cp_async_wait_all();
}

// Forward x and y of one z-plane in shared memory (small grids): the n real
// rows as n/2 complex lines, x transforms split into the half spectra
// kx = 0..nc (the y columns), y transforms of the nc + 1 columns, keep
// |ky| <= nc; output spec2[z][kx][ky] (plane-major).
template <typename R>
__device__ __forceinline__ void k2_fft_xy_body(Geo g, FftPlanDev fp, const R* __restrict__ grid,
                                                const typename Cx<R>::T* __restrict__ twg,
                                                typename Cx<R>::T* __restrict__ spec2, Blk blk) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1, K = g.K, h = n / 2, lsb = fft2_lsb(n);
    C* tw = reinterpret_cast<C*>(smraw);
    C* A = tw + n;                            // [n/2] phase-A rows; then the y columns P[kx][y]
    C* B = A + h * fft2_lsa(fp.f1, fp.f2);    // [n/2][lsb] x results; then the y phase-A rows
    fft2_twiddles(tw, twg, fp);
    const int z = blk.id;
    const R* gz = grid + (size_t)z * n * n;
    __syncthreads();
    fft2_lines<R, false>(
        A, tw, fp, h,
        [&](int c, int x) {
            C v;
            v.x = gz[(size_t)(2 * c) * n + x];
            v.y = gz[(size_t)(2 * c + 1) * n + x];
            return v;
        },
        [&](int c, int k, C v) {
            if (k <= nc || k >= n - nc) B[c * lsb + k] = v;
        });
    __syncthreads();
    C* P = A;   // [nc + 1][n]: column kx over y
    const float rh = 1.0f / (float)h;
    for (int idx = threadIdx.x; idx < nc1 * h; idx += blockDim.x) {
        const int k = qdiv(idx, h, rh), c = idx - k * h;
        const C zk = B[c * lsb + k];
        const C zm = B[c * lsb + (k == 0 ? 0 : n - k)];
        C a, b;
        a.x = (R)0.5 * (zk.x + zm.x);
        a.y = (R)0.5 * (zk.y - zm.y);
        b.x = (R)0.5 * (zk.y + zm.y);
        b.y = (R)0.5 * (zm.x - zk.x);
        P[k * n + 2 * c] = a;
        P[k * n + 2 * c + 1] = b;
    }
    __syncthreads();
    C* out = spec2 + (size_t)z * nc1 * K;
    fft2_lines<R, false>(
        B, tw, fp, nc1, [&](int kx, int y) { return P[kx * n + y]; },
        [&](int kx, int k, C v) {
            if (k <= nc) out[kx * K + k + nc] = v;
            else if (k >= n - nc) out[kx * K + k - n + nc] = v;
        });
}

template <typename R>
__global__ void __launch_bounds__(512) k2_fft_xy(Geo g, FftPlanDev fp, const R* __restrict__ grid,
                                                const typename Cx<R>::T* __restrict__ twg,
                                                typename Cx<R>::T* __restrict__ spec2) {
    k2_fft_xy_body<R>(g, fp, grid, twg, spec2, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// Inverse y and x of one (field, z-plane) in shared memory (small grids):
// the plane spec3[a][z][kx][ky] zero-padded to n along y, inverse y of the
// nc + 1 columns, then two Hermitian rows per complex line (C2R) inverse
// along x; output h[a][z][y][x].
template <typename R>
__device__ __forceinline__ void k2_fft_yx_body(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec3,
                                                const typename Cx<R>::T* __restrict__ twg, R* __restrict__ h, Blk blk) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ unsigned char smraw[];
    const int n = g.n, nc = g.nc, nc1 = nc + 1, K = g.K, hn = n / 2, lsb = fft2_lsb(n);
    C* tw = reinterpret_cast<C*>(smraw);
    C* A = tw + n;                             // [n/2] phase-A rows
    C* Yc = A + hn * fft2_lsa(fp.f1, fp.f2);   // [nc + 1][lsb]: inverse y results [kx][y]
    fft2_twiddles(tw, twg, fp);
    const int az = blk.id;   // a * n + z
    const C* in = spec3 + (size_t)az * nc1 * K;
    __syncthreads();
    fft2_lines<R, true>(
        A, tw, fp, nc1,
        [&](int kx, int m) {
            const int ky = m <= n / 2 ? m : m - n;
            C v;
            v.x = (R)0;
            v.y = (R)0;
            if (ky >= -nc && ky <= nc) v = in[kx * K + (ky + nc)];
            return v;
        },
        [&](int kx, int y, C v) { Yc[kx * lsb + y] = v; });
    __syncthreads();
    R* out = h + (size_t)az * n * n;
    fft2_lines<R, true>(
        A, tw, fp, hn,
        [&](int c, int m) {
            C a, b;
            a.x = a.y = b.x = b.y = (R)0;
            if (m == 0) {
                a.x = Yc[2 * c].x;
                b.x = Yc[2 * c + 1].x;
            } else if (m <= nc) {
                a = Yc[m * lsb + 2 * c];
                b = Yc[m * lsb + 2 * c + 1];
            } else if (m >= n - nc) {
                a = Yc[(n - m) * lsb + 2 * c];
                a.y = -a.y;
                b = Yc[(n - m) * lsb + 2 * c + 1];
                b.y = -b.y;
            }
            C zz;
            zz.x = a.x - b.y;   // A + i B
            zz.y = a.y + b.x;
            return zz;
        },
        [&](int c, int x, C v) {
            out[(size_t)(2 * c) * n + x] = v.x;
            out[(size_t)(2 * c + 1) * n + x] = v.y;
        });
}

template <typename R>
__global__ void __launch_bounds__(512) k2_fft_yx(Geo g, FftPlanDev fp, const typename Cx<R>::T* __restrict__ spec3,
                                                const typename Cx<R>::T* __restrict__ twg, R* __restrict__ h) {
    k2_fft_yx_body<R>(g, fp, spec3, twg, h, Blk{(int)blockIdx.x, (int)gridDim.x});
}

}  // namespace enuf

namespace enuf {

// ---------------------------------------------------------------------------
// a2 (FP32): footprint spreading on bricks, optionally fused with the forward
// x pass (the NFFT's window convolution followed by its FFT, Sec. 3.3 and
// Eq. 14, without the grid's round trip through memory).
// One CTA per brick [x0, x0 + BX) x [y0, y0 + T) x [z0, z0 + T) of the grid
// (BX a multiple of the tile edge T dividing n), one warp per z-plane of the
// brick (T warps). Candidates are the charged beads of the tiles around the
// brick (x tiles x0/T - 1 .. (x0 + BX)/T, y and z tiles +-1, periodic), the
// items those whose window meets the brick. Per item, the warp that owns
// plane z adds q w_z w_y w_x into the item's (x, y) taps inside the brick,
// lanes over the taps: every lane of a warp writes a distinct address and no
// other warp writes that plane, so there are no atomics, and no multiply-add
// is spent on a weight outside the item's window (the column form multiplies
// every column of its tile by every z-slot).
// FX (BX = n, T even): the brick's T^2 rows of length n are then transformed
// along x (R2C, two rows per complex line, the two-factor kernels' line
// transform) and written as spec1[z][kx][y] for kx <= nc; otherwise the brick
// is written to the grid.
// ---------------------------------------------------------------------------
static_assert(kBrickTaps == kMaxTaps, "brick weight rows hold the widest window");

template <typename R, bool FX>
__global__ void __launch_bounds__(768) k_spread_brick(Geo g, FftPlanDev fp, int BX, const int* __restrict__ tstart,
                                                      const typename V4<R>::T* __restrict__ sq,
                                                      const int* __restrict__ sb, const R* __restrict__ wb,
                                                      R* __restrict__ grid, const typename Cx<R>::T* __restrict__ twg,
                                                      typename Cx<R>::T* __restrict__ spec1, int LP) {
    pdl_enter();
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int T = g.T, n = g.n, p = g.p, P2 = 2 * p, ntd = g.ntd;
    R* acc = reinterpret_cast<R*>(smraw);                          // [T][T][BX]
    unsigned char* stage = smraw + (size_t)T * T * BX * sizeof(R);
    int* cslot = reinterpret_cast<int*>(stage);                    // [kBrickCand]
    int* cbase = cslot + kBrickCand;                               // [kBrickCand]
    R* cq = reinterpret_cast<R*>(cbase + kBrickCand);              // [kBrickCand]
    int* items = reinterpret_cast<int*>(cq + kBrickCand);          // [kBrickCand] candidate indices
    R* wt = reinterpret_cast<R*>(items + kBrickCand);              // [kBrickItems][3][kMaxTaps]
    int* ibase = reinterpret_cast<int*>(wt + kBrickItems * 3 * kMaxTaps);   // [kBrickItems]
    R* iq = reinterpret_cast<R*>(ibase + kBrickItems);             // [kBrickItems]
    __shared__ int rstart[kBrickRanges], rpre[kBrickRanges + 1];
    __shared__ int nranges, nitems;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nbx = n / BX;
    const int bxi = blockIdx.x % nbx, byz = blockIdx.x / nbx;
    const int ty = byz % ntd, tz = byz / ntd;
    const int x0 = bxi * BX, y0 = ty * T, z0 = tz * T;
    for (int e = tid; e < T * T * BX; e += blockDim.x) acc[e] = (R)0;
    if (warp == 0) {   // runs of sorted beads: the x tiles around the brick in each of the <= 9 (y, z) tile rows
        const int noy = ntd >= 3 ? 3 : ntd;
        const int nrow = noy * noy;
        const int ntx = BX / T;
        const bool full = ntx + 2 >= ntd;   // the whole row of x tiles
        int st = 0, c = 0;
        if (lane < 2 * nrow) {
            const int r = lane >> 1, half = lane & 1;
            const int dy = r % noy, dz = r / noy;
            const int yy = ntd >= 3 ? (ty + dy - 1 + ntd) % ntd : dy;
            const int zz = ntd >= 3 ? (tz + dz - 1 + ntd) % ntd : dz;
            const int row = (zz * ntd + yy) * ntd;
            int a = 0, b = -1;   // x tiles [a, b] of this half
            if (full) {
                if (!half) { a = 0; b = ntd - 1; }
            } else {
                int ta = bxi * ntx - 1, tb = bxi * ntx + ntx;   // inclusive, may leave [0, ntd)
                if (ta < 0) {        // [ntd - 1] and [0, tb]
                    if (half) { a = ntd - 1; b = ntd - 1; } else { a = 0; b = tb; }
                } else if (tb >= ntd) {   // [ta, ntd - 1] and [0, tb - ntd]
                    if (half) { a = 0; b = tb - ntd; } else { a = ta; b = ntd - 1; }
                } else if (!half) {
                    a = ta;
                    b = tb;
                }
            }
            if (b >= a) {
                st = tstart[row + a];
                c = tstart[row + b + 1] - st;
            }
        }
        int x = c;
#pragma unroll
        for (int of = 1; of < 32; of <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, of);
            if (lane >= of) x += y;
        }
        if (lane < 2 * nrow) {
            rstart[lane] = st;
            rpre[lane] = x - c;
        }
        if (lane == 2 * nrow - 1) {
            rpre[2 * nrow] = x;
            nranges = 2 * nrow;
        }
    }
    __syncthreads();
    const int nr = nranges, total = rpre[nr];
    // this lane's tap pair (a, b): a = lane % P2, b = lane / P2 + k rpi
    const int rpi = 32 / P2, la = lane % P2, lb = lane / P2;
    const int z = z0 + warp;   // this warp's plane (warp < T)
    for (int cb = 0; cb < total; cb += kBrickCand) {
        const int cn = min(kBrickCand, total - cb);
        if (tid == 0) nitems = 0;
        for (int idx = tid; idx < cn; idx += blockDim.x) {   // stage: one thread per candidate
            const int f = cb + idx;
            int lo = 0, hi = nr;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (rpre[mid] <= f) lo = mid; else hi = mid;
            }
            const int j = rstart[lo] + f - rpre[lo];
            cslot[idx] = j;
            cbase[idx] = sb[j];
            cq[idx] = sq[j].w;
        }
        __syncthreads();
        for (int c0 = 0; c0 < cn; c0 += blockDim.x) {   // items: the window meets the brick
            const int c = c0 + tid;
            bool keep = false;
            if (c < cn) {
                const int pb = cbase[c];
                keep = tap_mask((pb >> 20) & 1023, z0, T, n, ntd, p) != 0u &&
                       tap_mask((pb >> 10) & 1023, y0, T, n, ntd, p) != 0u;
                if (keep && BX < n) {   // x: some tap in [x0, x0 + BX)
                    int l = (pb & 1023) - p + 1 - x0;
                    l = l < 0 ? l + n : (l >= n ? l - n : l);
                    keep = l < BX || l + P2 > n;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            int basei = 0;
            if (lane == 0 && bal) basei = atomicAdd(&nitems, __popc(bal));
            basei = __shfl_sync(0xffffffffu, basei, 0);
            const int at = basei + __popc(bal & ((1u << lane) - 1u));
            if (keep && ENUF_GUARD(g.check, at < kBrickCand, 3)) items[at] = c;
        }
        __syncthreads();
        const int ni = nitems;
        for (int ib = 0; ib < ni; ib += kBrickItems) {
            const int nb = min(kBrickItems, ni - ib);
            for (int e = tid; e < nb * 3 * P2; e += blockDim.x) {   // the batch's window weights
                const int i = e / (3 * P2), r = e - i * (3 * P2);
                const int c = items[ib + i];
                wt[i * 3 * kMaxTaps + (r / P2) * kMaxTaps + r % P2] = wb[(size_t)cslot[c] * 3 * P2 + r];
                if (r == 0) {
                    ibase[i] = cbase[c];
                    iq[i] = cq[c];
                }
            }
            __syncthreads();
            if (warp < T) {
                R* plane = acc + warp * T * BX;
                for (int i = 0; i < nb; ++i) {
                    const int pb = ibase[i];
                    int az = z - ((pb >> 20) & 1023) + p - 1;   // tap of plane z
                    az = az < 0 ? az + n : (az >= n ? az - n : az);
                    if (az >= P2) continue;                      // warp-uniform
                    const R* w = wt + i * 3 * kMaxTaps;
                    int x = (pb & 1023) - p + 1 + la;
                    x = x < 0 ? x + n : (x >= n ? x - n : x);
                    x -= x0;
                    if (lb < rpi && x >= 0 && x < BX) {
                        const R wxz = iq[i] * w[2 * kMaxTaps + az] * w[la];
                        const int yb = ((pb >> 10) & 1023) - p + 1 - y0;
                        for (int b = lb; b < P2; b += rpi) {
                            int y = yb + b;
                            y = y < 0 ? y + n : (y >= n ? y - n : y);
                            if (y < T) plane[y * BX + x] += wxz * w[kMaxTaps + b];
                        }
                    }
                    // the next item may add into addresses this item's lanes wrote
                    __syncwarp();
                }
            }
            __syncthreads();
        }
    }
    if constexpr (!FX) {   // write the brick: rows of BX points
        for (int e = tid; e < T * T * BX; e += blockDim.x) {
            const int r = e / BX, x = e - r * BX;
            const int zz = r / T, yy = r - zz * T;
            grid[((size_t)(z0 + zz) * n + (y0 + yy)) * n + x0 + x] = acc[e];
        }
    } else {   // forward x of the brick's rows (BX = n), kx <= nc, into spec1[z][kx][y]
        const int nc = g.nc, nc1 = nc + 1, lsb = fft2_lsb(n);
        C* tw = reinterpret_cast<C*>(stage);
        C* A = tw + n;
        C* B = A + LP * fft2_lsa(fp.f1, fp.f2);
        fft2_twiddles(tw, twg, fp);
        const int npair = T * T / 2;
        for (int c0 = 0; c0 < npair; c0 += LP) {
            const int nl = min(LP, npair - c0);
            __syncthreads();
            fft2_lines<R, false>(
                A, tw, fp, nl,
                [&](int c, int x) {
                    C v;
                    v.x = acc[(size_t)(2 * (c0 + c)) * n + x];
                    v.y = acc[(size_t)(2 * (c0 + c) + 1) * n + x];
                    return v;
                },
                [&](int c, int k, C v) {
                    if (k <= nc || k >= n - nc) B[c * lsb + k] = v;
                });
            __syncthreads();
            for (int idx = tid; idx < nl * nc1; idx += blockDim.x) {
                const int k = idx / nl, c = idx - k * nl;
                const C zk = B[c * lsb + k];
                const C zm = B[c * lsb + (k == 0 ? 0 : n - k)];
                C a, b;
                a.x = (R)0.5 * (zk.x + zm.x);
                a.y = (R)0.5 * (zk.y - zm.y);
                b.x = (R)0.5 * (zk.y + zm.y);
                b.y = (R)0.5 * (zm.x - zk.x);
                const int r = 2 * (c0 + c), zz = r / T, yy = r - zz * T;   // rows r, r + 1: y and y + 1
                C* dst = spec1 + ((size_t)(z0 + zz) * nc1 + k) * n + y0 + yy;
                dst[0] = a;
                dst[1] = b;
            }
        }
    }
}

}  // namespace enuf
