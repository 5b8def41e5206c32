// Batched mixed-radix FFTs for the pressure Poisson solve (paper Sec. 2.6.1,
// spectral solver p = DFT^-1 Lhat^-1 DFT r), and the FP64 Thomas solve along a
// wall-normal direction.
//
// Design: every pass moves a tile of whole lines into shared memory, runs a
// Stockham auto-sort FFT there (ping-pong buffers, one butterfly per work item,
// radices 2, 3, 4, 5, 7, 8), and writes the tile back. Tiles are TW lines wide:
//  - x pass: lines are contiguous in memory; pairs of real lines are packed
//    into one complex line (a + i b) and separated after the transform, giving
//    the half spectra of both (real-to-complex without a separate kernel);
//  - y and z passes: lines are strided; a tile holds TW neighbouring columns so
//    that every global access is a contiguous run of TW complex values;
//  - the last periodic pass does forward FFT, multiplies by the precomputed
//    table 1/(Lhat * Ntot) (Lhat(0) := 1), and the inverse FFT, in one visit.
// The inverse transform is conj(FFT(conj(x))) (unnormalised; 1/Ntot is in the table).
// The Stockham indexing (butterfly j of a stage with radix R reads j + r L/R,
// twiddles by W_{Ns R}^{r (j mod Ns)}, writes (j div Ns) Ns R + (j mod Ns) + r Ns)
// is the published auto-sort formulation (Stockham 1966; as used for GPUs by
// Govindaraju et al., SC 2008).
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace ins {

constexpr int FFT_MAX_STAGES = 16;
constexpr int FFT_THREADS = 256;

template <typename T>
struct FftLine {
    int L;                         // line length
    int nst;                       // number of stages
    int radix[FFT_MAX_STAGES];
    const cplx<T>* tw;             // tw[m] = exp(-2 pi i m / L), m in [0, L)
};

// ---------------------------------------------------------------- butterflies
template <typename T, int R>
struct Dft;

template <typename T>
struct Dft<T, 2> {
    static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>*, int) {
        cplx<T> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <typename T>
struct Dft<T, 4> {
    static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>*, int) {
        cplx<T> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        cplx<T> t2 = cadd(v[1], v[3]), t3 = cmul_mi(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <typename T>
struct Dft<T, 8> {
    static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>*, int) {
        const T s = (T)0.70710678118654752440;  // 1/sqrt(2)
        cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
        cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
        Dft<T, 4>::run(e, nullptr, 0);
        Dft<T, 4>::run(o, nullptr, 0);
        // o[m] *= W8^m, W8 = exp(-2 pi i / 8)
        cplx<T> o1 = {(o[1].re + o[1].im) * s, (o[1].im - o[1].re) * s};
        cplx<T> o2 = cmul_mi(o[2]);
        cplx<T> o3 = {(o[3].im - o[3].re) * s, -(o[3].re + o[3].im) * s};
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

// Odd radices: y_m = a_0 + sum_q (a_q + a_{R-q}) cos(2 pi q m/R) - i (a_q - a_{R-q}) sin(2 pi q m/R)
// with the cos/sin read from the line's twiddle table (tw[q L/R] = exp(-2 pi i q/R)).
template <typename T, int R>
struct DftOdd {
    static __device__ __forceinline__ void run(cplx<T>* v, const cplx<T>* tw, int L) {
        constexpr int H = (R - 1) / 2;
        cplx<T> s[H], d[H];
#pragma unroll
        for (int q = 1; q <= H; ++q) {
            s[q - 1] = cadd(v[q], v[R - q]);
            d[q - 1] = csub(v[q], v[R - q]);
        }
        cplx<T> y0 = v[0];
#pragma unroll
        for (int q = 0; q < H; ++q) y0 = cadd(y0, s[q]);
        const int step = L / R;
        cplx<T> out[R];
        out[0] = y0;
#pragma unroll
        for (int m = 1; m <= H; ++m) {
            cplx<T> X = v[0], Y = {(T)0, (T)0};
#pragma unroll
            for (int q = 1; q <= H; ++q) {
                cplx<T> w = ldg_c(&tw[((q * m) % R) * step]);   // cos - i sin
                T c = w.re, sn = -w.im;
                X.re = fma(c, s[q - 1].re, X.re);
                X.im = fma(c, s[q - 1].im, X.im);
                Y.re = fma(sn, d[q - 1].re, Y.re);
                Y.im = fma(sn, d[q - 1].im, Y.im);
            }
            // y_m = X - i Y, y_{R-m} = X + i Y
            out[m] = {X.re + Y.im, X.im - Y.re};
            out[R - m] = {X.re - Y.im, X.im + Y.re};
        }
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = out[m];
    }
};
template <typename T>
struct Dft<T, 3> : DftOdd<T, 3> {};
template <typename T>
struct Dft<T, 5> : DftOdd<T, 5> {};
template <typename T>
struct Dft<T, 7> : DftOdd<T, 7> {};

// One Stockham stage over a tile held as buf[m * SP + c], c in [0, TW).
template <typename T, int R>
__device__ __forceinline__ void fft_stage(const cplx<T>* __restrict__ A, cplx<T>* __restrict__ B, int SP,
                                          int lgTW, int L, int Ns, const cplx<T>* __restrict__ tw) {
    const int TW = 1 << lgTW;
    const int nb = L / R;
    const int twstride = L / (Ns * R);
    for (int item = threadIdx.x; item < (nb << lgTW); item += blockDim.x) {
        const int c = item & (TW - 1);
        const int j = item >> lgTW;
        const int k = j % Ns;
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = A[(j + r * nb) * SP + c];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], ldg_c(&tw[r * k * twstride]));
        }
        Dft<T, R>::run(v, tw, L);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) B[(base + r * Ns) * SP + c] = v[r];
    }
}

// Forward FFT of the TW lines of the tile in buf0 (buf1 is scratch). Returns
// the buffer holding the result in natural order. Ends with __syncthreads().
template <typename T>
__device__ cplx<T>* fft_tile(const FftLine<T>& pl, cplx<T>* buf0, cplx<T>* buf1, int SP, int lgTW) {
    cplx<T>* A = buf0;
    cplx<T>* B = buf1;
    int Ns = 1;
    for (int s = 0; s < pl.nst; ++s) {
        const int R = pl.radix[s];
        switch (R) {
            case 2: fft_stage<T, 2>(A, B, SP, lgTW, pl.L, Ns, pl.tw); break;
            case 3: fft_stage<T, 3>(A, B, SP, lgTW, pl.L, Ns, pl.tw); break;
            case 4: fft_stage<T, 4>(A, B, SP, lgTW, pl.L, Ns, pl.tw); break;
            case 5: fft_stage<T, 5>(A, B, SP, lgTW, pl.L, Ns, pl.tw); break;
            case 7: fft_stage<T, 7>(A, B, SP, lgTW, pl.L, Ns, pl.tw); break;
            default: fft_stage<T, 8>(A, B, SP, lgTW, pl.L, Ns, pl.tw); break;
        }
        __syncthreads();
        cplx<T>* t = A;
        A = B;
        B = t;
        Ns *= R;
    }
    return A;
}

// ------------------------------------------------------------------ x pass
// Real lines (contiguous, length L = nx) -> half spectra (nxh = L/2 + 1 each).
// CTA handles line pairs [p0, p0 + TW); lines 2p and 2p+1 share one complex FFT.
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_x_r2c(FftLine<T> pl, const T* __restrict__ in,
                                                           cplx<T>* __restrict__ S, int lines, int nxh, int lgTW) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TW = 1 << lgTW, SP = TW + 1, L = pl.L;
    cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf1 = buf0 + (size_t)L * SP;
    const long p0 = (long)blockIdx.x * TW;
    for (int item = threadIdx.x; item < L * TW; item += blockDim.x) {
        const int c = item / L, m = item - c * L;
        const long la = 2 * (p0 + c), lb = la + 1;
        cplx<T> z;
        z.re = la < lines ? in[la * L + m] : (T)0;
        z.im = lb < lines ? in[lb * L + m] : (T)0;
        buf0[m * SP + c] = z;
    }
    __syncthreads();
    cplx<T>* X = fft_tile(pl, buf0, buf1, SP, lgTW);
    for (int item = threadIdx.x; item < nxh * TW; item += blockDim.x) {
        const int c = item / nxh, kk = item - c * nxh;
        const long la = 2 * (p0 + c), lb = la + 1;
        const cplx<T> Z = X[kk * SP + c];
        const cplx<T> Zc = cconj(X[(kk == 0 ? 0 : L - kk) * SP + c]);
        const T h = (T)0.5;
        // A = (Z + conj Z_{-k})/2, B = (Z - conj Z_{-k})/(2i)
        if (la < lines) S[la * nxh + kk] = {h * (Z.re + Zc.re), h * (Z.im + Zc.im)};
        if (lb < lines) S[lb * nxh + kk] = {h * (Z.im - Zc.im), -h * (Z.re - Zc.re)};
    }
}

// Half spectra -> real lines (unnormalised inverse).
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_x_c2r(FftLine<T> pl, const cplx<T>* __restrict__ S,
                                                           T* __restrict__ out, int lines, int nxh, int lgTW) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TW = 1 << lgTW, SP = TW + 1, L = pl.L;
    cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf1 = buf0 + (size_t)L * SP;
    const long p0 = (long)blockIdx.x * TW;
    for (int item = threadIdx.x; item < L * TW; item += blockDim.x) {
        const int c = item / L, m = item - c * L;
        const long la = 2 * (p0 + c), lb = la + 1;
        const bool upper = m >= nxh;                 // use the Hermitian mirror L - m
        const int src = upper ? L - m : m;
        cplx<T> A = la < lines ? S[la * nxh + src] : cplx<T>{(T)0, (T)0};
        cplx<T> B = lb < lines ? S[lb * nxh + src] : cplx<T>{(T)0, (T)0};
        if (upper) {
            A = cconj(A);
            B = cconj(B);
        }
        if (m == 0 || 2 * m == L) {  // real-valued bins of a real line
            A.im = (T)0;
            B.im = (T)0;
        }
        // Z = A + i B, conjugated for the inverse transform
        buf0[m * SP + c] = {A.re - B.im, -(A.im + B.re)};
    }
    __syncthreads();
    cplx<T>* X = fft_tile(pl, buf0, buf1, SP, lgTW);
    for (int item = threadIdx.x; item < L * TW; item += blockDim.x) {
        const int c = item / L, m = item - c * L;
        const long la = 2 * (p0 + c), lb = la + 1;
        const cplx<T> z = X[m * SP + c];   // conj of the inverse: re -> line a, -im -> line b
        if (la < lines) out[la * L + m] = z.re;
        if (lb < lines) out[lb * L + m] = -z.im;
    }
}

// ------------------------------------------------------------- strided pass
// Columns col in [0, ncol): element (col, m) at
//   (col / cdiv) * outer + m * lstride + (col % cdiv).
// mode 0: forward, 1: inverse, 2: forward, times scale[addr], inverse.
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_strided(FftLine<T> pl, cplx<T>* __restrict__ S, long ncol,
                                                             long cdiv, long outer, long lstride, int mode,
                                                             const T* __restrict__ scale, int lgTW) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TW = 1 << lgTW, SP = TW + 1, L = pl.L;
    cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf1 = buf0 + (size_t)L * SP;
    const long c0 = (long)blockIdx.x * TW;
    for (int item = threadIdx.x; item < L * TW; item += blockDim.x) {
        const int c = item & (TW - 1), m = item >> lgTW;
        const long col = c0 + c;
        cplx<T> z = {(T)0, (T)0};
        if (col < ncol) {
            const long a = (col / cdiv) * outer + m * lstride + (col % cdiv);
            z = S[a];
            if (mode == 1) z = cconj(z);
        }
        buf0[m * SP + c] = z;
    }
    __syncthreads();
    cplx<T>* X = fft_tile(pl, buf0, buf1, SP, lgTW);
    if (mode == 2) {
        cplx<T>* Y = (X == buf0) ? buf1 : buf0;
        for (int item = threadIdx.x; item < L * TW; item += blockDim.x) {
            const int c = item & (TW - 1), m = item >> lgTW;
            const long col = c0 + c;
            T s = (T)0;
            if (col < ncol) s = ldg_t(&scale[(col / cdiv) * outer + m * lstride + (col % cdiv)]);
            const cplx<T> z = X[m * SP + c];
            Y[m * SP + c] = {z.re * s, -z.im * s};     // scaled and conjugated
        }
        __syncthreads();
        X = fft_tile(pl, Y, X, SP, lgTW);
    }
    for (int item = threadIdx.x; item < L * TW; item += blockDim.x) {
        const int c = item & (TW - 1), m = item >> lgTW;
        const long col = c0 + c;
        if (col < ncol) {
            cplx<T> z = X[m * SP + c];
            if (mode != 0) z = cconj(z);
            S[(col / cdiv) * outer + m * lstride + (col % cdiv)] = z;
        }
    }
}

// Spectral table s = 1 / ((lx + ly + lz) * ntot), entry (0,0,0) = 1/ntot, layout [kz][ky][kx].
template <typename T>
__global__ void k_make_scale(T* __restrict__ s, const double* __restrict__ lx, const double* __restrict__ ly,
                             const double* __restrict__ lz, int nxh, int ny, int nz, double ntot) {
    const long n = (long)nxh * ny * nz;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
        const int kx = idx % nxh;
        const long r = idx / nxh;
        const int ky = r % ny;
        const int kz = r / ny;
        double lam = lx[kx] + ly[ky] + lz[kz];
        if (kx == 0 && ky == 0 && kz == 0) lam = 1.0;
        s[idx] = (T)(1.0 / (lam * ntot));
    }
}

// ---------------------------------------------------------- wall direction
// FP64 solve of (D G along y + lambda_x + lambda_z) p = r for every (kx, kz) mode by a twisted
// (two-ended) factorisation with precomputed factors (they do not change in time). Rows
// lo_j x_{j-1} + b_j x_j + up_j x_{j+1} = r_j meet at m = ny / 2:
//   top    (j < m, downwards):  d_j = (r_j - lo_j d_{j-1}) * f_j,  row j: x_j + g_j x_{j+1} = d_j,
//   bottom (j > m, upwards):    e_j = (r_j - up_j e_{j+1}) * f_j,  row j: g_j x_{j-1} + x_j = e_j,
//   middle: x_m = (r_m - lo_m d_{m-1} - up_m e_{m+1}) * f_m,
// then x_j = d_j - g_j x_{j+1} upwards from m and x_j = e_j - g_j x_{j-1} downwards from m
// (f = th_invm, g = th_cp, per row and column). The normalisation s = 1/(nx nz) of the two
// inverse FFTs is folded into the factors (f' = s f, lo' = lo / s, up' = up / s give s x with
// the same operations). FP32 spectra are converted to and from FP64 by bit operations (the
// convert instructions would run on the FP64 pipe). Two threads per column, one per end, so twice
// the columns' parallelism of a one-sided sweep; the middle values pass through shared memory.
// col = kz * nxh + kx; element (col, j) at (col / nxh) * ny * nxh + j * nxh + col % nxh.
// The mean mode (col 0) has its first row replaced by p_0 = 0 (r_0 taken as 0).
// Block 2 * TH_COLS threads: threads [0, TH_COLS) the top ends, the rest the bottom ends of
// TH_COLS consecutive columns.
// FP32 spectra are solved in double-float arithmetic (pairs of FP32 numbers, about 48 significant
// bits: dfloat.cuh) on the FP32 pipe instead of FP64 arithmetic on the FP64 pipe; the FP64 factors
// are stored as double-float pairs (rounded from FP64 on the host, 2^-48 relative; no conversion
// in the sweeps) and the scratch holds double-float pairs. Double-float spectra (the double-float
// FP64 step on a channel) use the same arithmetic with the FP64 tables split by bits. FP64 spectra keep
// FP64 arithmetic.
constexpr int TH_COLS = 64;

// A: the arithmetic type; F: the stored factor type (the grid holds its factor tables as FP64 for
// FP64 spectra and as double-float pairs, rounded from the same FP64 values, for FP32 spectra).
template <typename T>
struct ThArith {
    using A = double;
    using F = double;
    static __device__ __forceinline__ A in(T x) { return as_f64(x); }
    static __device__ __forceinline__ A fac(F x) { return x; }
    static __device__ __forceinline__ F ld(const F* p) { return __ldg(p); }
    static __device__ __forceinline__ T out(A x) { return from_f64<T>(x); }
};
// double-float spectra (the double-float FP64 step on a wall-bounded grid): FP64 tables split by bits
template <>
struct ThArith<df> {
    using A = df;
    using F = double;
    static __device__ __forceinline__ A in(df x) { return x; }
    static __device__ __forceinline__ A fac(F x) { return df_split(x); }
    static __device__ __forceinline__ F ld(const F* p) { return __ldg(p); }
    static __device__ __forceinline__ df out(A x) { return x; }
};
template <>
struct ThArith<float> {
    using A = df;
    using F = df;
    static __device__ __forceinline__ A in(float x) { return df(x); }
    static __device__ __forceinline__ A fac(F x) { return x; }
    static __device__ __forceinline__ F ld(const F* p) { return ldg_t(p); }
    static __device__ __forceinline__ float out(A x) { return __fadd_rn(x.hi, x.lo); }
};

template <typename T>
__global__ void __launch_bounds__(2 * TH_COLS) k_thomas2(cplx<T>* __restrict__ S,
                                                         const typename ThArith<T>::F* __restrict__ lo,
                                                         const typename ThArith<T>::F* __restrict__ up,
                                                         const typename ThArith<T>::F* __restrict__ invm,
                                                         const typename ThArith<T>::F* __restrict__ cp,
                                                         cplx<typename ThArith<T>::A>* __restrict__ dscr, int nxh,
                                                         int ny, long ncol) {
    using Ar = ThArith<T>;
    using A = typename Ar::A;
    using Fc = typename Ar::F;
    // The loads do not depend on the recurrence: rows are fetched in batches of CH before
    // each CH-step stretch of the (sequential) sweep, so CH loads per array are in flight.
    constexpr int CH = 16;
    __shared__ cplx<A> mid[2][TH_COLS];   // d_{m-1} (top ends), e_{m+1} (bottom ends)
    const int lc = threadIdx.x % TH_COLS;
    const bool top = threadIdx.x < TH_COLS;
    const long col = blockIdx.x * (long)TH_COLS + lc;
    const bool ok = col < ncol;
    const long base = ok ? (col / nxh) * (long)ny * nxh + (col % nxh) : 0;
    const int m = ny / 2;
    // rows handled by this end, in elimination order: top 0 .. m-1, bottom ny-1 .. m+1
    const int nrows = top ? m : ny - 1 - m;
    const int dir = top ? 1 : -1;
    const int j0 = top ? 0 : ny - 1;
    const Fc* cpl = top ? lo : up;   // the coupling to the previous row of the sweep
    const A zero = A(0.0);
    cplx<A> dv = {zero, zero};
    if (ok) {
        for (int s0 = 0; s0 < nrows; s0 += CH) {
            cplx<T> r[CH];
            Fc a[CH], f[CH];
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                if (s0 + q < nrows) {
                    const int j = j0 + dir * (s0 + q);
                    r[q] = S[base + (long)j * nxh];
                    a[q] = Ar::ld(&cpl[j]);
                    f[q] = Ar::ld(&invm[(long)j * ncol + col]);
                }
            }
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                if (s0 + q < nrows) {
                    const int j = j0 + dir * (s0 + q);
                    A rre = Ar::in(r[q].re), rim = Ar::in(r[q].im);
                    if (j == 0 && col == 0) rre = rim = zero;
                    const A aq = Ar::fac(a[q]), fq = Ar::fac(f[q]);
                    if constexpr (std::is_same<A, df>::value) {
                        // (r - a d) f as r f - (a f) d: only one product and one difference on the
                        // sequential dependence from row to row (double-float; in FP64 the extra
                        // product costs the FP64 pipe more than the shorter chain saves)
                        const A bq = aq * fq;
                        const A are = rre * fq, aim = rim * fq;
                        dv.re = are - bq * dv.re;
                        dv.im = aim - bq * dv.im;
                    } else {
                        dv.re = (rre - aq * dv.re) * fq;
                        dv.im = (rim - aq * dv.im) * fq;
                    }
                    dscr[(long)j * ncol + col] = dv;
                }
            }
        }
    }
    mid[top ? 0 : 1][lc] = dv;   // 0 when this end has no rows
    // row m's right-hand side is read by both ends before the barrier (the top end rewrites it)
    cplx<T> rm = {(T)0, (T)0};
    Fc fm = Fc(0.0);
    if (ok) {
        rm = S[base + (long)m * nxh];
        if (m == 0 && col == 0) rm = {(T)0, (T)0};   // ny == 1: the mean mode's p_0 = 0 row is the middle
        fm = Ar::ld(&invm[(long)m * ncol + col]);
    }
    __syncthreads();
    if (!ok) return;
    // x_m, computed by both ends of the column
    const cplx<A> dm = mid[0][lc], em = mid[1][lc];
    const A lom = Ar::fac(Ar::ld(&lo[m])), upm = Ar::fac(Ar::ld(&up[m])), fmA = Ar::fac(fm);
    cplx<A> x;
    x.re = (Ar::in(rm.re) - lom * dm.re - upm * em.re) * fmA;
    x.im = (Ar::in(rm.im) - lom * dm.im - upm * em.im) * fmA;
    if (top) S[base + (long)m * nxh] = {Ar::out(x.re), Ar::out(x.im)};
    // back-substitution from the middle outwards: top m-1 .. 0, bottom m+1 .. ny-1
    const int jb = top ? m - 1 : m + 1;
    for (int s0 = 0; s0 < nrows; s0 += CH) {
        cplx<A> d[CH];
        Fc g[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            if (s0 + q < nrows) {
                const int j = jb - dir * (s0 + q);
                d[q] = dscr[(long)j * ncol + col];
                g[q] = Ar::ld(&cp[(long)j * ncol + col]);
            }
        }
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            if (s0 + q < nrows) {
                const int j = jb - dir * (s0 + q);
                const A gq = Ar::fac(g[q]);
                x.re = d[q].re - gq * x.re;
                x.im = d[q].im - gq * x.im;
                S[base + (long)j * nxh] = {Ar::out(x.re), Ar::out(x.im)};
            }
        }
    }
}

}  // namespace ins

namespace ins {

// ------------------------------------------------------ DCT-II wall-normal solve
// Uniform wall-normal spacing (paper Sec. 6: the channel DNS on a uniform grid solves the
// pressure with FFTs): with homogeneous Neumann rows the y operator is diagonalised by the
// DCT-II, X_k = sum_j x_j cos(pi k (2j+1) / (2N)), with eigenvalues mu_k = -4 sin^2(pi k/(2N)) / dy^2.
// One visit per tile of TW columns (after the x and z forward FFTs): the DCT-II by one complex
// FFT of the reordered line v = (x_0, x_2, ..., x_3, x_1) (Makhoul, IEEE TASSP 1980):
//   X_k = (w_k V_k + conj(w_k) V_{N-k}) / 2,  w_k = exp(-i pi k / (2N)),  V_N := V_0;
// division by lambda_x + lambda_z + mu_k (FP64; the mean mode is set to 0) times `norm`;
// and the inverse: V_k = conj(w_k) (X_k - i X_{N-k}) (X_N := 0), v = IDFT(V) (the 1/N is in
// `norm`), x_{2m} = v_m, x_{2(N-1-m)+1} = v_m for m >= ceil(N/2).
// Columns as in k_fft_strided: element (col, j) at (col / cdiv) * outer + j * lstride + col % cdiv,
// kx = col % cdiv, kz = col / cdiv.
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS) k_dct_solve_y(FftLine<T> pl, cplx<T>* __restrict__ S, long ncol,
                                                             long cdiv, long outer, long lstride,
                                                             const cplx<T>* __restrict__ qw,
                                                             const double* __restrict__ lamx,
                                                             const double* __restrict__ lamy,
                                                             const double* __restrict__ lamz, double norm, int lgTW) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TW = 1 << lgTW, SP = TW + 1, L = pl.L;
    const int hN = (L + 1) / 2;
    cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf1 = buf0 + (size_t)L * SP;
    const long c0 = (long)blockIdx.x * TW;
    auto src_row = [L, hN](int m) { return m < hN ? 2 * m : 2 * (L - 1 - m) + 1; };
    for (int item = threadIdx.x; item < L * TW; item += blockDim.x) {
        const int c = item & (TW - 1), m = item >> lgTW;
        const long col = c0 + c;
        cplx<T> z = {(T)0, (T)0};
        if (col < ncol) z = S[(col / cdiv) * outer + (long)src_row(m) * lstride + (col % cdiv)];
        buf0[m * SP + c] = z;
    }
    __syncthreads();
    cplx<T>* V = fft_tile(pl, buf0, buf1, SP, lgTW);
    cplx<T>* X = (V == buf0) ? buf1 : buf0;
    for (int item = threadIdx.x; item < L * TW; item += blockDim.x) {
        const int c = item & (TW - 1), k = item >> lgTW;
        const long col = c0 + c;
        const cplx<T> w = ldg_c(&qw[k]);
        const cplx<T> vk = V[k * SP + c];
        const cplx<T> vn = V[(k == 0 ? 0 : L - k) * SP + c];
        // (w vk + conj(w) vn) / 2
        cplx<T> d = {(T)0.5 * (w.re * (vk.re + vn.re) - w.im * (vk.im - vn.im)),
                     (T)0.5 * (w.re * (vk.im + vn.im) + w.im * (vk.re - vn.re))};
        double s = 0.0;
        if (col < ncol) {
            const long kx = col % cdiv, kz = col / cdiv;
            const double lam = lamx[kx] + lamz[kz] + lamy[k];
            s = lam != 0.0 ? norm / lam : 0.0;
        }
        X[k * SP + c] = {(T)(s * (double)d.re), (T)(s * (double)d.im)};
    }
    __syncthreads();
    for (int item = threadIdx.x; item < L * TW; item += blockDim.x) {
        const int c = item & (TW - 1), k = item >> lgTW;
        const cplx<T> w = ldg_c(&qw[k]);
        const cplx<T> xk = X[k * SP + c];
        const cplx<T> xn = k == 0 ? cplx<T>{(T)0, (T)0} : X[(L - k) * SP + c];
        // t = xk - i xn; V = conj(w) t; stored conjugated for the inverse by a forward FFT
        const cplx<T> t = {xk.re + xn.im, xk.im - xn.re};
        const cplx<T> vv = {w.re * t.re + w.im * t.im, w.re * t.im - w.im * t.re};
        V[k * SP + c] = cconj(vv);
    }
    __syncthreads();
    cplx<T>* Z = fft_tile(pl, V, X, SP, lgTW);
    for (int item = threadIdx.x; item < L * TW; item += blockDim.x) {
        const int c = item & (TW - 1), m = item >> lgTW;
        const long col = c0 + c;
        if (col < ncol) S[(col / cdiv) * outer + (long)src_row(m) * lstride + (col % cdiv)] = cconj(Z[m * SP + c]);
    }
}

}  // namespace ins
