// enuf_fft.cuh -- batched shared-memory FFT of length n = 2^a 3^b 5^c (n <= 1024).
//
// The 3-D transforms of the NFFT (the plain FFT step of Sec. 3.3 inside the
// transposed and conjugated NFFT, Eq. 13-14) are done one dimension at a time;
// each CTA loads a batch of lines into shared memory and runs this Stockham
// auto-sort FFT on all of them. Stage s with radix R combines R sub-transforms
// of length Ns (product of the earlier radices): butterfly j of a line reads
// x[j + r n/R], twiddles element r by w^{r k n/(Ns R)} (k = j mod Ns,
// w = e^{-+2 pi i/n}), does an R-point DFT and writes the results to
// (j - k) R + k + m Ns. After the last stage the line is in natural order.
// Radices 2, 3, 4, 5, 8 and the composites 6, 10, 12, 16, 20 (two small DFTs
// in registers with compile-time twiddles), so most lengths take two stages.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

namespace enuf {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

struct FftPlanDev {
    int n;
    int nst;
    int rad[8];
    int f1, f2;   // two-factor split n = f1 f2 of the FP32 two-factor kernels (0: none)
};

// a / b for 0 <= a < 2^23, b >= 1, given rb = 1/b in float: the float quotient
// of a + 1/2 is within one of the true one, and one integer step corrects it.
__device__ __forceinline__ int qdiv(int a, int b, float rb) {
    int q = (int)(((float)a + 0.5f) * rb);
    const int r = a - q * b;
    q += (r >= b ? 1 : 0) - (r < 0 ? 1 : 0);
    return q;
}

// Shared-memory layout of the line buffers. A bank row holds 128 B, i.e. B
// complex values (16 float2 or 8 double2). The index inside a line is
// swizzled, i -> i XOR (row of i mod B), so that both unit-stride accesses
// and the strided writes of the early Stockham stages spread over all banks;
// lines are padded to whole bank rows plus one value, which skews consecutive
// lines for the accesses that run across lines.
template <typename C> struct SwzBits;
template <> struct SwzBits<float2> { static constexpr int v = 4; };
template <> struct SwzBits<double2> { static constexpr int v = 3; };
template <typename C>
__device__ __forceinline__ int swz(int i) {
    constexpr int b = SwzBits<C>::v;
    return i ^ ((i >> b) & ((1 << b) - 1));
}
template <typename C>
__host__ __device__ constexpr int line_stride(int n) {
    return ((n + (1 << SwzBits<C>::v) - 1) >> SwzBits<C>::v << SwzBits<C>::v) + 1;
}

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// multiply by -i (forward) or +i (inverse): the rotation of the 4-point DFT
template <typename C, bool INV>
__device__ __forceinline__ C rot_i(C a) {
    C r;
    if (INV) { r.x = -a.y; r.y = a.x; }   // +i a
    else     { r.x = a.y;  r.y = -a.x; }  // -i a
    return r;
}

template <typename R, int RAD, bool INV> struct SmallDft;

template <typename R, bool INV> struct SmallDft<R, 2, INV> {
    template <typename C> __device__ __forceinline__ static void run(C* v) {
        C a = cadd(v[0], v[1]), b = csub(v[0], v[1]);
        v[0] = a; v[1] = b;
    }
};

template <typename R, bool INV> struct SmallDft<R, 4, INV> {
    template <typename C> __device__ __forceinline__ static void run(C* v) {
        C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        C s13 = cadd(v[1], v[3]), d13 = rot_i<C, INV>(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <typename R, bool INV> struct SmallDft<R, 8, INV> {
    template <typename C> __device__ __forceinline__ static void run(C* v) {
        // even / odd 4-point DFTs, then combine with w8^m
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        SmallDft<R, 4, INV>::run(e);
        SmallDft<R, 4, INV>::run(o);
        const R h = (R)0.70710678118654752440;
        C t1, t3;
        // w8 = (1 -+ i)/sqrt2 ; w8^2 = -+ i ; w8^3 = (-1 -+ i)/sqrt2
        if (INV) {
            t1.x = h * (o[1].x - o[1].y); t1.y = h * (o[1].x + o[1].y);
            t3.x = -h * (o[3].x + o[3].y); t3.y = h * (o[3].x - o[3].y);
        } else {
            t1.x = h * (o[1].x + o[1].y); t1.y = h * (o[1].y - o[1].x);
            t3.x = h * (o[3].y - o[3].x); t3.y = -h * (o[3].x + o[3].y);
        }
        C t2 = rot_i<C, INV>(o[2]);
        v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], t1);   v[5] = csub(e[1], t1);
        v[2] = cadd(e[2], t2);   v[6] = csub(e[2], t2);
        v[3] = cadd(e[3], t3);   v[7] = csub(e[3], t3);
    }
};

template <typename R, bool INV> struct SmallDft<R, 3, INV> {
    template <typename C> __device__ __forceinline__ static void run(C* v) {
        const R s3 = (R)0.86602540378443864676;  // sqrt(3)/2
        C t = cadd(v[1], v[2]);
        C d = csub(v[1], v[2]);
        C m;
        m.x = v[0].x - (R)0.5 * t.x;
        m.y = v[0].y - (R)0.5 * t.y;
        // forward: y1 = m - i s3 d, y2 = m + i s3 d ; inverse swaps the sign of i
        C id = rot_i<C, INV>(d);   // -i d (fwd) or +i d (inv)
        v[0] = cadd(v[0], t);
        v[1].x = m.x + s3 * id.x; v[1].y = m.y + s3 * id.y;
        v[2].x = m.x - s3 * id.x; v[2].y = m.y - s3 * id.y;
    }
};

template <typename R, bool INV> struct SmallDft<R, 5, INV> {
    template <typename C> __device__ __forceinline__ static void run(C* v) {
        const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;
        const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;
        C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        C m1, m2, u1, u2;
        m1.x = v[0].x + c1 * a1.x + c2 * a2.x; m1.y = v[0].y + c1 * a1.y + c2 * a2.y;
        m2.x = v[0].x + c2 * a1.x + c1 * a2.x; m2.y = v[0].y + c2 * a1.y + c1 * a2.y;
        u1.x = s1 * b1.x + s2 * b2.x; u1.y = s1 * b1.y + s2 * b2.y;
        u2.x = s2 * b1.x - s1 * b2.x; u2.y = s2 * b1.y - s1 * b2.y;
        C iu1 = rot_i<C, INV>(u1), iu2 = rot_i<C, INV>(u2);  // -i u (fwd)
        v[0].x = v[0].x + a1.x + a2.x; v[0].y = v[0].y + a1.y + a2.y;
        v[1] = cadd(m1, iu1); v[4] = csub(m1, iu1);
        v[2] = cadd(m2, iu2); v[3] = csub(m2, iu2);
    }
};

// Compile-time loop: f(std::integral_constant<int, i>) for i = 0 .. N-1.
template <typename F, int... I>
__device__ __forceinline__ void sfor_(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
    sfor_(f, std::make_integer_sequence<int, N>{});
}

// cos and sin of 2 pi m / N, evaluated by the compiler: the angle is reduced
// to [0, pi/2) by its quadrant (exact integer arithmetic), then Taylor series
// to 30 terms (the last term is below 1e-60 there).
struct Root {
    double c, s;
};
__host__ __device__ constexpr double taylor_cos(double x) {
    double sum = 1.0, t = 1.0;
    for (int k = 1; k < 30; ++k) {
        t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += t;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_sin(double x) {
    double sum = x, t = x;
    for (int k = 1; k < 30; ++k) {
        t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += t;
    }
    return sum;
}
__host__ __device__ constexpr Root unit_root(int m, int N) {
    m = ((m % N) + N) % N;
    const int q = 4 * m / N;            // quadrant
    const int rn = 4 * m - q * N;       // remaining angle (pi/2) rn / N in [0, pi/2)
    const double r = 1.57079632679489661923 * rn / N;
    const double c = taylor_cos(r), sn = taylor_sin(r);
    return q == 0 ? Root{c, sn} : q == 1 ? Root{-sn, c} : q == 2 ? Root{-c, -sn} : Root{sn, -c};
}

// a omega^M with omega = e^{-2 pi i/N} (forward) or e^{+2 pi i/N} (inverse);
// the quarter turns are exact rotations.
template <int M, int N, bool INV, typename R, typename C>
__device__ __forceinline__ C twiddle_const(C a) {
    constexpr int m = M % N;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (4 * m == N) {
        return rot_i<C, INV>(a);
    } else if constexpr (2 * m == N) {
        a.x = -a.x;
        a.y = -a.y;
        return a;
    } else if constexpr (4 * m == 3 * N) {
        return rot_i<C, !INV>(a);
    } else {
        constexpr Root w = unit_root(m, N);
        const R c = (R)w.c, sn = INV ? (R)w.s : (R)-w.s;
        C r;
        r.x = a.x * c - a.y * sn;
        r.y = a.x * sn + a.y * c;
        return r;
    }
}

// Composite radix N1 N2 in registers (Cooley-Tukey): input index N2 n1 + n2,
// N2 DFTs of length N1 over n1, twiddle omega_{N1 N2}^{n2 k1}, N1 DFTs of
// length N2 over n2; output index k1 + N1 k2 (natural order).
template <typename R, int N1, int N2, bool INV>
struct CompositeDft {
    template <typename C>
    __device__ __forceinline__ static void run(C* v) {
        constexpr int RR = N1 * N2;
        C y[RR];   // y[n2 N1 + k1]
        sfor<N2>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            C a[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) a[n1] = v[N2 * n1 + n2];
            SmallDft<R, N1, INV>::run(a);
            sfor<N1>([&](auto k1c) {
                constexpr int k1 = decltype(k1c)::value;
                y[n2 * N1 + k1] = twiddle_const<n2 * k1, RR, INV, R>(a[k1]);
            });
        });
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            C b[N2];
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) b[n2] = y[n2 * N1 + k1];
            SmallDft<R, N2, INV>::run(b);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) v[k1 + N1 * k2] = b[k2];
        }
    }
};
template <typename R, bool INV> struct SmallDft<R, 6, INV> : CompositeDft<R, 2, 3, INV> {};
template <typename R, bool INV> struct SmallDft<R, 10, INV> : CompositeDft<R, 2, 5, INV> {};
template <typename R, bool INV> struct SmallDft<R, 12, INV> : CompositeDft<R, 4, 3, INV> {};
template <typename R, bool INV> struct SmallDft<R, 16, INV> : CompositeDft<R, 4, 4, INV> {};
template <typename R, bool INV> struct SmallDft<R, 20, INV> : CompositeDft<R, 4, 5, INV> {};

// One Stockham stage over nlines lines (line l at offset l*ls, swizzled inside).
template <typename R, int RAD, bool INV>
__device__ __forceinline__ void fft_stage(const typename Cx<R>::T* __restrict__ src,
                                          typename Cx<R>::T* __restrict__ dst,
                                          const typename Cx<R>::T* __restrict__ tw,
                                          int n, int Ns, int nlines, int ls) {
    using C = typename Cx<R>::T;
    const int m = n / RAD;
    const int tstep = n / (Ns * RAD);
    const int total = nlines * m;
    const float rm = 1.0f / (float)m, rNs = 1.0f / (float)Ns;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int line = qdiv(idx, m, rm);
        const int j = idx - line * m;
        const int k = j - qdiv(j, Ns, rNs) * Ns;
        const C* s = src + line * ls;
        C* d = dst + line * ls;
        C v[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[r] = s[swz<C>(j + r * m)];
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                C w = tw[r * k * tstep];
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        SmallDft<R, RAD, INV>::run(v);
        const int base = (j - k) * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) d[swz<C>(base + r * Ns)] = v[r];
    }
}

// Transform nlines lines held in b0; b1 is scratch of the same size. Returns
// the buffer holding the result. Contains __syncthreads (call from all threads).
// CR: the composite radices 6, 10, 12, 16, 20 are compiled in (the plan's
// radix list decides which instance runs; they raise the kernels' register
// count, so plans without them run the CR = false instance).
template <typename R, bool INV, bool CR = false>
__device__ typename Cx<R>::T* fft_lines(typename Cx<R>::T* b0, typename Cx<R>::T* b1,
                                        const typename Cx<R>::T* tw, const FftPlanDev& fp,
                                        int nlines, int ls) {
    using C = typename Cx<R>::T;
    C* src = b0;
    C* dst = b1;
    int Ns = 1;
    for (int st = 0; st < fp.nst; ++st) {
        const int rad = fp.rad[st];
        if constexpr (CR) {
            switch (rad) {
                case 16: fft_stage<R, 16, INV>(src, dst, tw, fp.n, Ns, nlines, ls); break;
                case 20: fft_stage<R, 20, INV>(src, dst, tw, fp.n, Ns, nlines, ls); break;
                case 12: fft_stage<R, 12, INV>(src, dst, tw, fp.n, Ns, nlines, ls); break;
                case 10: fft_stage<R, 10, INV>(src, dst, tw, fp.n, Ns, nlines, ls); break;
                case 6: fft_stage<R, 6, INV>(src, dst, tw, fp.n, Ns, nlines, ls); break;
                default: break;
            }
        }
        switch (rad) {
            case 8: fft_stage<R, 8, INV>(src, dst, tw, fp.n, Ns, nlines, ls); break;
            case 4: fft_stage<R, 4, INV>(src, dst, tw, fp.n, Ns, nlines, ls); break;
            case 2: fft_stage<R, 2, INV>(src, dst, tw, fp.n, Ns, nlines, ls); break;
            case 3: fft_stage<R, 3, INV>(src, dst, tw, fp.n, Ns, nlines, ls); break;
            case 5: fft_stage<R, 5, INV>(src, dst, tw, fp.n, Ns, nlines, ls); break;
            default: break;
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
        Ns *= rad;
    }
    return src;
}

}  // namespace enuf

namespace enuf {

// ---------------------------------------------------------------------------
// Two-factor line FFT for lengths n = f1 f2 with both factors among the
// radices above: the Cooley-Tukey split of the n-point DFT into f2 DFTs of
// length f1, one twiddle per element, and f1 DFTs of length f2. With
// element m = t + f2 j of a line (t < f2, j < f1) and output k = k1 + f1 k2,
//   X[k1 + f1 k2] = sum_t w_n^{t k1} w_f2^{t k2} sum_j x[t + f2 j] w_f1^{j k1}.
// Phase A (one task per line and t): loads its f1 elements (through the
//   caller's loader, usually straight from global memory), the f1-point DFT
//   in registers, the twiddles w_n^{t k1} from the shared table, and stores
//   row k1 of the line's buffer at k1 (f2 + 1) + t (rows padded by one value:
//   phase B reads a row per lane, and the odd stride spreads those reads
//   over the banks).
// Phase B (one task per line and k1): the f2-point DFT of row k1 in
//   registers; the caller's storer receives X[k1 + f1 k2].
// The factors are compile-time (the DFTs and every offset inside a task are
// constants); n, f1, f2 and the line count are runtime values, so one kernel
// serves every length with such a factorization. Per element this is one
// load, the DFT arithmetic of two radices, one twiddle multiply and two
// shared-memory accesses, against the runtime-radix Stockham stages'
// per-stage quotients, swizzles and twiddle indices.
// ---------------------------------------------------------------------------
template <typename R, int F1, bool INV, typename Load>
__device__ __forceinline__ void fft2_phase_a(typename Cx<R>::T* __restrict__ buf, int lsa, int nlines, int f2,
                                             const typename Cx<R>::T* __restrict__ tw, Load& load) {
    using C = typename Cx<R>::T;
    const int total = nlines * f2;
    const float rf2 = 1.0f / (float)f2;
    for (int task = threadIdx.x; task < total; task += blockDim.x) {
        const int line = qdiv(task, f2, rf2), t = task - line * f2;
        C v[F1];
#pragma unroll
        for (int j = 0; j < F1; ++j) v[j] = load(line, t + f2 * j);
        SmallDft<R, F1, INV>::run(v);
#pragma unroll
        for (int k = 1; k < F1; ++k) {
            C w = tw[k * f2 + t];   // w_n^{t k}: lanes over t read consecutive values
            if (INV) w.y = -w.y;
            v[k] = cmul(v[k], w);
        }
        C* d = buf + line * lsa + t;
#pragma unroll
        for (int k = 0; k < F1; ++k) d[k * (f2 + 1)] = v[k];
    }
}

template <typename R, int F2, bool INV, typename Store>
__device__ __forceinline__ void fft2_phase_b(const typename Cx<R>::T* __restrict__ buf, int lsa, int nlines, int f1,
                                             Store& store) {
    using C = typename Cx<R>::T;
    const int total = nlines * f1;
    const float rf1 = 1.0f / (float)f1;
    for (int task = threadIdx.x; task < total; task += blockDim.x) {
        const int line = qdiv(task, f1, rf1), k1 = task - line * f1;
        const C* s = buf + line * lsa + k1 * (F2 + 1);
        C u[F2];
#pragma unroll
        for (int t = 0; t < F2; ++t) u[t] = s[t];
        SmallDft<R, F2, INV>::run(u);
#pragma unroll
        for (int k2 = 0; k2 < F2; ++k2) store(line, k1 + f1 * k2, u[k2]);
    }
}

// The twiddle table of phase A in shared memory, tw[k f2 + t] = w_n^{t k}
// (t < f2, k < f1; forward sign), from the table twg[m] = w_n^m: the lanes of
// a phase-A step read consecutive values (the natural table, read at t k,
// puts lanes of an even k on few banks).
template <typename C>
__device__ __forceinline__ void fft2_twiddles(C* __restrict__ tw, const C* __restrict__ twg, const FftPlanDev& fp) {
    const int f2 = fp.f2, n = fp.f1 * fp.f2;
    const float rf2 = 1.0f / (float)f2;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int k = qdiv(e, f2, rf2), t = e - k * f2;
        tw[e] = twg[t * k];
    }
}

// Row stride of a phase-A line buffer, and of a buffer of natural-order
// results. A two-factor pass with L lines per CTA holds the twiddle table (n
// values), L phase-A rows and L result rows in shared memory.
__host__ __device__ constexpr int fft2_lsa(int f1, int f2) { return f1 * (f2 + 1); }
__host__ __device__ constexpr int fft2_lsb(int n) { return n + 1; }

// The whole two-factor transform of nlines lines: load(line, m) gives element
// m of a line, store(line, k, X_k) takes the results; tw is the table that
// fft2_twiddles fills. buf holds nlines rows
// of fft2_lsa(f1, f2) values. Contains __syncthreads (call from all threads);
// the caller synchronises before reading what store wrote to shared memory.
template <typename R, bool INV, typename Load, typename Store>
__device__ __forceinline__ void fft2_lines(typename Cx<R>::T* __restrict__ buf, const typename Cx<R>::T* tw,
                                           const FftPlanDev& fp, int nlines, Load&& load, Store&& store) {
    const int f1 = fp.f1, f2 = fp.f2, lsa = fft2_lsa(f1, f2);
    switch (f1) {
        case 4: fft2_phase_a<R, 4, INV>(buf, lsa, nlines, f2, tw, load); break;
        case 5: fft2_phase_a<R, 5, INV>(buf, lsa, nlines, f2, tw, load); break;
        case 6: fft2_phase_a<R, 6, INV>(buf, lsa, nlines, f2, tw, load); break;
        case 8: fft2_phase_a<R, 8, INV>(buf, lsa, nlines, f2, tw, load); break;
        case 10: fft2_phase_a<R, 10, INV>(buf, lsa, nlines, f2, tw, load); break;
        case 12: fft2_phase_a<R, 12, INV>(buf, lsa, nlines, f2, tw, load); break;
        case 16: fft2_phase_a<R, 16, INV>(buf, lsa, nlines, f2, tw, load); break;
        case 20: fft2_phase_a<R, 20, INV>(buf, lsa, nlines, f2, tw, load); break;
        default: break;
    }
    __syncthreads();
    switch (f2) {
        case 4: fft2_phase_b<R, 4, INV>(buf, lsa, nlines, f1, store); break;
        case 5: fft2_phase_b<R, 5, INV>(buf, lsa, nlines, f1, store); break;
        case 6: fft2_phase_b<R, 6, INV>(buf, lsa, nlines, f1, store); break;
        case 8: fft2_phase_b<R, 8, INV>(buf, lsa, nlines, f1, store); break;
        case 10: fft2_phase_b<R, 10, INV>(buf, lsa, nlines, f1, store); break;
        case 12: fft2_phase_b<R, 12, INV>(buf, lsa, nlines, f1, store); break;
        case 16: fft2_phase_b<R, 16, INV>(buf, lsa, nlines, f1, store); break;
        case 20: fft2_phase_b<R, 20, INV>(buf, lsa, nlines, f1, store); break;
        default: break;
    }
}

}  // namespace enuf
