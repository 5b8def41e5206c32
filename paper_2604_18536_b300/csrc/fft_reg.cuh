// Register-resident FFT passes for line lengths L = R1 * R2 with R1, R2 in
// {4, 8, 16} (L = 16 .. 256): the hot sizes of the periodic Poisson solve.
//
// Four-step decomposition (index m = j + R2 r, frequency k = k1 + R1 k2):
//   X[k1 + R1 k2] = sum_j W_R2^{j k2} ( W_L^{j k1} sum_r x[j + R2 r] W_R1^{r k1} ).
// Stage A: thread (column c, j) loads its R1 values x[j + R2 r] straight from
// global memory into registers, does a DFT of size R1 and the twiddles
// W_L^{j k1}. One exchange through shared memory. Stage B: thread (c, k1)
// gathers its R2 values, does a DFT of size R2 and holds X[k1 + R1 k2] for all
// k2, which it stores directly (or, in the fused forward/scale/inverse pass,
// feeds to the inverse transform: with the factors swapped, that data is
// already laid out for the inverse's stage A, so only one more exchange is
// needed). One shared buffer of L x (TW + 1) values, no ping-pong.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace ins {

template <typename T, int R>
struct DftR;

template <typename T>
struct DftR<T, 4> {
    static __device__ __forceinline__ void run(cplx<T>* v) { Dft<T, 4>::run(v, nullptr, 0); }
};
template <typename T>
struct DftR<T, 8> {
    static __device__ __forceinline__ void run(cplx<T>* v) { Dft<T, 8>::run(v, nullptr, 0); }
};

// 16-point DFT as 4 x 4 with the internal twiddles W16^{j k1}.
template <typename T>
struct DftR<T, 16> {
    static __device__ __forceinline__ void run(cplx<T>* v) {
        const T c1 = (T)0.92387953251128675613;   // cos(pi/8)
        const T s1 = (T)0.38268343236508977173;   // sin(pi/8)
        const T h = (T)0.70710678118654752440;    // 1/sqrt(2)
        cplx<T> y[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            cplx<T> t[4] = {v[j], v[j + 4], v[j + 8], v[j + 12]};
            Dft<T, 4>::run(t, nullptr, 0);
#pragma unroll
            for (int k = 0; k < 4; ++k) y[j][k] = t[k];
        }
        // twiddles W16^{j k1}, W16 = exp(-2 pi i / 16)
        y[1][1] = cmul(y[1][1], cplx<T>{c1, -s1});
        y[1][2] = {(y[1][2].re + y[1][2].im) * h, (y[1][2].im - y[1][2].re) * h};   // W16^2
        y[1][3] = cmul(y[1][3], cplx<T>{s1, -c1});
        y[2][1] = {(y[2][1].re + y[2][1].im) * h, (y[2][1].im - y[2][1].re) * h};   // W16^2
        y[2][2] = cmul_mi(y[2][2]);                                                  // W16^4
        y[2][3] = {(y[2][3].im - y[2][3].re) * h, -(y[2][3].re + y[2][3].im) * h};  // W16^6
        y[3][1] = cmul(y[3][1], cplx<T>{s1, -c1});                                    // W16^3
        y[3][2] = {(y[3][2].im - y[3][2].re) * h, -(y[3][2].re + y[3][2].im) * h};  // W16^6
        y[3][3] = cmul(y[3][3], cplx<T>{-c1, s1});                                    // W16^9
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            cplx<T> t[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
            Dft<T, 4>::run(t, nullptr, 0);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
        }
    }
};

// Stage A in registers: DFT_R1 over r of v[r] = x[j + R2 r], then v[k1] *= W_L^{j k1}.
template <typename T, int R1>
__device__ __forceinline__ void stage_a(cplx<T>* v, int j, const cplx<T>* __restrict__ tw) {
    DftR<T, R1>::run(v);
    if (j > 0) {
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], ldg_c(&tw[j * k1]));
    }
}

template <typename T, int R1, int R2>
struct RegShape {
    static constexpr int L = R1 * R2;
    static constexpr int RM = R1 > R2 ? R1 : R2;
    static constexpr int NT = sizeof(T) == 8 ? 128 : 256;   // keeps the exchange buffer under 48 KB
    static constexpr int TW = NT / RM;    // columns (or line pairs) per tile
    static constexpr int SP = TW + 1;     // padded row of the exchange buffer
};

// Strided pass, columns as in k_fft_strided: element (col, m) at
// (col / cdiv) * outer + m * lstride + (col % cdiv).
// mode 0: forward, 1: inverse, 2: forward, times scale[addr], inverse.
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2) k_fft_strided_reg(const cplx<T>* __restrict__ tw, cplx<T>* __restrict__ S,
                                                         long ncol, long cdiv, long outer, long lstride, int mode,
                                                         const T* __restrict__ scale) {
    using Sh = RegShape<T, R1, R2>;
    constexpr int L = Sh::L, TW = Sh::TW, SP = Sh::SP;
    __shared__ cplx<T> ex[L * SP];
    const int c = threadIdx.x % TW;
    const int q = threadIdx.x / TW;          // j in stage A, k1 in stage B
    const long col = (long)blockIdx.x * TW + c;
    const bool ok = col < ncol;
    const long cb = ok ? (col / cdiv) * outer + (col % cdiv) : 0;
    cplx<T> v[Sh::RM];
    // ---- forward stage A (R1 x R2): thread (c, j = q < R2)
    if (q < R2) {
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            cplx<T> z = {(T)0, (T)0};
            if (ok) z = S[cb + (long)(q + R2 * r) * lstride];
            if (mode == 1) z = cconj(z);
            v[r] = z;
        }
        stage_a<T, R1>(v, q, tw);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) ex[(q * R1 + k1) * SP + c] = v[k1];
    }
    __syncthreads();
    // ---- forward stage B: thread (c, k1 = q < R1) gathers Y_j[k1], j < R2
    if (q < R1) {
#pragma unroll
        for (int j = 0; j < R2; ++j) v[j] = ex[(j * R1 + q) * SP + c];
        DftR<T, R2>::run(v);       // v[k2] = X[q + R1 k2]
    }
    if (mode == 2) {
        // scale and conjugate, then the inverse with the factors swapped: thread (c, j' = q < R1)
        // holds x'[q + R1 k2] for k2 < R2, i.e. stage A input of an R2 x R1 transform.
        if (q < R1) {
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                const long m = q + R1 * k2;
                const T s = ok ? __ldg(&scale[cb + m * lstride]) : (T)0;
                v[k2] = {v[k2].re * s, -v[k2].im * s};
            }
            stage_a<T, R2>(v, q, tw);
        }
        __syncthreads();   // everyone finished reading ex
        if (q < R1) {
#pragma unroll
            for (int k1 = 0; k1 < R2; ++k1) ex[(q * R2 + k1) * SP + c] = v[k1];
        }
        __syncthreads();
        if (q < R2) {
#pragma unroll
            for (int j = 0; j < R1; ++j) v[j] = ex[(j * R2 + q) * SP + c];
            DftR<T, R1>::run(v);   // v[k2] = conj(result)[q + R2 k2]
            if (ok) {
#pragma unroll
                for (int k2 = 0; k2 < R1; ++k2) S[cb + (long)(q + R2 * k2) * lstride] = cconj(v[k2]);
            }
        }
        return;
    }
    if (q < R1 && ok) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
            cplx<T> z = v[k2];
            if (mode == 1) z = cconj(z);
            S[cb + (long)(q + R1 * k2) * lstride] = z;
        }
    }
}

// x pass, real lines -> half spectra. CTA handles TW line pairs packed as a + i b.
// Thread mapping (j fastest) keeps the loads along a line contiguous.
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2) k_fft_x_r2c_reg(const cplx<T>* __restrict__ tw, const T* __restrict__ in,
                                                       cplx<T>* __restrict__ S, int lines, int nxh) {
    using Sh = RegShape<T, R1, R2>;
    constexpr int L = Sh::L, TW = Sh::TW, RM = Sh::RM;
    constexpr int SR = L + L / 16 + 1;   // padded row per pair (breaks power-of-two strides)
    __shared__ cplx<T> ex[TW * SR];
    const int q = threadIdx.x % RM;      // j (stage A) / k1 (stage B)
    const int c = threadIdx.x / RM;
    const long la = 2 * ((long)blockIdx.x * TW + c), lb = la + 1;
    auto sidx = [](int m) { return m + (m >> 4); };
    cplx<T> v[RM];
    if (q < R2) {
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const int m = q + R2 * r;
            v[r] = {la < lines ? in[la * L + m] : (T)0, lb < lines ? in[lb * L + m] : (T)0};
        }
        stage_a<T, R1>(v, q, tw);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) ex[c * SR + sidx(q * R1 + k1)] = v[k1];
    }
    __syncthreads();
    if (q < R1) {
#pragma unroll
        for (int j = 0; j < R2; ++j) v[j] = ex[c * SR + sidx(j * R1 + q)];
        DftR<T, R2>::run(v);
    }
    __syncthreads();
    if (q < R1) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) ex[c * SR + sidx(q + R1 * k2)] = v[k2];   // natural order
    }
    __syncthreads();
    const T h = (T)0.5;
    for (int item = threadIdx.x; item < TW * nxh; item += blockDim.x) {
        const int cc = item / nxh, kk = item - cc * nxh;
        const long a = 2 * ((long)blockIdx.x * TW + cc), b = a + 1;
        const cplx<T> Z = ex[cc * SR + sidx(kk)];
        const cplx<T> Zc = cconj(ex[cc * SR + sidx(kk == 0 ? 0 : L - kk)]);
        if (a < lines) S[a * nxh + kk] = {h * (Z.re + Zc.re), h * (Z.im + Zc.im)};
        if (b < lines) S[b * nxh + kk] = {h * (Z.im - Zc.im), -h * (Z.re - Zc.re)};
    }
}

// x pass, half spectra -> real lines (unnormalised inverse).
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2) k_fft_x_c2r_reg(const cplx<T>* __restrict__ tw, const cplx<T>* __restrict__ S,
                                                       T* __restrict__ out, int lines, int nxh) {
    using Sh = RegShape<T, R1, R2>;
    constexpr int L = Sh::L, TW = Sh::TW, RM = Sh::RM;
    constexpr int SR = L + L / 16 + 1;
    __shared__ cplx<T> ex[TW * SR];
    auto sidx = [](int m) { return m + (m >> 4); };
    // Z = A + i B over the full line (Hermitian extension), conjugated for the inverse
    for (int item = threadIdx.x; item < TW * L; item += blockDim.x) {
        const int cc = item / L, m = item - cc * L;
        const long a = 2 * ((long)blockIdx.x * TW + cc), b = a + 1;
        const bool upper = m >= nxh;
        const int src = upper ? L - m : m;
        cplx<T> A = a < lines ? S[a * nxh + src] : cplx<T>{(T)0, (T)0};
        cplx<T> B = b < lines ? S[b * nxh + src] : cplx<T>{(T)0, (T)0};
        if (upper) {
            A = cconj(A);
            B = cconj(B);
        }
        if (m == 0 || 2 * m == L) {
            A.im = (T)0;
            B.im = (T)0;
        }
        ex[cc * SR + sidx(m)] = {A.re - B.im, -(A.im + B.re)};
    }
    __syncthreads();
    const int q = threadIdx.x % RM;
    const int c = threadIdx.x / RM;
    cplx<T> v[RM];
    if (q < R2) {
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = ex[c * SR + sidx(q + R2 * r)];
        stage_a<T, R1>(v, q, tw);
    }
    __syncthreads();
    if (q < R2) {
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) ex[c * SR + sidx(q * R1 + k1)] = v[k1];
    }
    __syncthreads();
    if (q < R1) {
        const long la = 2 * ((long)blockIdx.x * TW + c), lb = la + 1;
#pragma unroll
        for (int j = 0; j < R2; ++j) v[j] = ex[c * SR + sidx(j * R1 + q)];
        DftR<T, R2>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
            const int m = q + R1 * k2;
            if (la < lines) out[la * L + m] = v[k2].re;
            if (lb < lines) out[lb * L + m] = -v[k2].im;
        }
    }
}

}  // namespace ins
