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

// CTAs per SM of the double-float strided pass (its register cap: three CTAs of 128 threads
// measured 16 % faster at 256^3 than two, despite a few spilled registers)
#ifndef FFT_DF_MINB
#define FFT_DF_MINB 3
#endif

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

// 3-point DFT with constants: s = a1 + a2, d = a1 - a2, y0 = a0 + s, y1,2 = a0 - s/2 -+ i (sqrt3/2) d.
template <typename T>
struct DftR<T, 3> {
    static __device__ __forceinline__ void run(cplx<T>* v) {
        const T h3 = (T)0.86602540378443864676;   // sqrt(3)/2
        const cplx<T> s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
        const cplx<T> t = {v[0].re - (T)0.5 * s.re, v[0].im - (T)0.5 * s.im};
        const cplx<T> e = {h3 * d.im, -h3 * d.re};   // -i (sqrt3/2) d
        v[0] = cadd(v[0], s);
        v[1] = cadd(t, e);
        v[2] = csub(t, e);
    }
};

// 6-point DFT as 3 x 2: DFT3 of (x[n2], x[n2+2], x[n2+4]) for n2 = 0, 1, twiddles W6^{n2 k1},
// DFT2 over n2: X[k1 + 3 k2].
template <typename T>
struct DftR<T, 6> {
    static __device__ __forceinline__ void run(cplx<T>* v) {
        const T h3 = (T)0.86602540378443864676;
        cplx<T> a[3] = {v[0], v[2], v[4]}, b[3] = {v[1], v[3], v[5]};
        DftR<T, 3>::run(a);
        DftR<T, 3>::run(b);
        const cplx<T> b1 = cmul(b[1], cplx<T>{(T)0.5, -h3});    // W6
        const cplx<T> b2 = cmul(b[2], cplx<T>{(T)-0.5, -h3});   // W6^2
        v[0] = cadd(a[0], b[0]);
        v[3] = csub(a[0], b[0]);
        v[1] = cadd(a[1], b1);
        v[4] = csub(a[1], b1);
        v[2] = cadd(a[2], b2);
        v[5] = csub(a[2], b2);
    }
};

// 12-point DFT as 4 x 3: DFT4 of (x[n2], x[n2+3], x[n2+6], x[n2+9]) for n2 < 3, twiddles
// W12^{n2 k1}, DFT3 over n2: X[k1 + 4 k2].
template <typename T>
struct DftR<T, 12> {
    static __device__ __forceinline__ void run(cplx<T>* v) {
        const T h3 = (T)0.86602540378443864676;
        cplx<T> y[3][4];
#pragma unroll
        for (int n2 = 0; n2 < 3; ++n2) {
            cplx<T> t[4] = {v[n2], v[n2 + 3], v[n2 + 6], v[n2 + 9]};
            Dft<T, 4>::run(t, nullptr, 0);
#pragma unroll
            for (int k = 0; k < 4; ++k) y[n2][k] = t[k];
        }
        y[1][1] = cmul(y[1][1], cplx<T>{h3, (T)-0.5});      // W12
        y[1][2] = cmul(y[1][2], cplx<T>{(T)0.5, -h3});      // W12^2
        y[1][3] = cmul_mi(y[1][3]);                           // W12^3 = -i
        y[2][1] = cmul(y[2][1], cplx<T>{(T)0.5, -h3});      // W12^2
        y[2][2] = cmul(y[2][2], cplx<T>{(T)-0.5, -h3});     // W12^4
        y[2][3] = {-y[2][3].re, -y[2][3].im};                 // W12^6 = -1
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            cplx<T> t[3] = {y[0][k1], y[1][k1], y[2][k1]};
            DftR<T, 3>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) v[k1 + 4 * k2] = t[k2];
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

// The same with the twiddles W_L^{j k1} already in registers (w[k1], k1 < R1).
template <typename T, int R1>
__device__ __forceinline__ void stage_a_w(cplx<T>* v, int j, const cplx<T>* w) {
    DftR<T, R1>::run(v);
    if (j > 0) {
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], w[k1]);
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
__global__ void __launch_bounds__(sizeof(T) == 8 ? 128 : 256, std::is_same<T, df>::value ? FFT_DF_MINB : 2) k_fft_strided_reg(const cplx<T>* __restrict__ tw, cplx<T>* __restrict__ S,
                                                         long ncol, long cdiv, long outer, long lstride, int mode,
                                                         const T* __restrict__ scale) {
    using Sh = RegShape<T, R1, R2>;
    constexpr int L = Sh::L, TW = Sh::TW, SP = Sh::SP;
    __shared__ cplx<T> ex[L * SP];
    const int c = threadIdx.x % TW;
    const int q = threadIdx.x / TW;          // j in stage A, k1 in stage B
    cplx<T> v[Sh::RM];
    if constexpr (R1 == R2 && std::is_same<T, df>::value) {
        // Square factorisation, double-float: the inverse half of mode 2 has the same thread roles,
        // layouts and twiddles as the forward half, so both run through one copy of the code (a
        // loop that is not unrolled): the fused pass then fits the instruction cache. Written as a
        // loop over tiles (the launch gives one CTA per tile): compiled so, it spills 8 instead of 24
        // bytes and runs 113 against 119 us per pass at 256^3.
        constexpr int R = R1;
        const long ntiles = (ncol + TW - 1) / TW;
#pragma unroll 1
        for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long col = tile * TW + c;
        const bool ok = col < ncol;
        const long cb = ok ? (col / cdiv) * outer + (col % cdiv) : 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cplx<T> z = {(T)0, (T)0};
            if (ok) z = S[cb + (long)(q + R * r) * lstride];
            if (mode == 1) z = cconj(z);
            v[r] = z;
        }
        const int npass = mode == 2 ? 2 : 1;
#pragma unroll 1
        for (int pass = 0; pass < npass; ++pass) {
            if (pass == 1) {
                // scale and conjugate: v[k2] = X[q + R k2] becomes the inverse's stage-A input
#pragma unroll
                for (int k2 = 0; k2 < R; ++k2) {
                    const T sc = ok ? ldg_t(&scale[cb + (long)(q + R * k2) * lstride]) : (T)0;
                    v[k2] = {v[k2].re * sc, -v[k2].im * sc};
                }
                __syncthreads();   // everyone finished reading ex
            }
            stage_a<T, R>(v, q, tw);
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) ex[(q * R + k1) * SP + c] = v[k1];
            __syncthreads();
#pragma unroll
            for (int j = 0; j < R; ++j) v[j] = ex[(j * R + q) * SP + c];
            DftR<T, R>::run(v);   // v[k2] = X[q + R k2] (pass 1: the conjugated inverse)
        }
        if (ok) {
#pragma unroll
            for (int k2 = 0; k2 < R; ++k2) {
                cplx<T> z = v[k2];
                if (mode != 0) z = cconj(z);
                S[cb + (long)(q + R * k2) * lstride] = z;
            }
        }
        __syncthreads();   // ex is rewritten by the next tile
        }
        return;
    }
    const long col = (long)blockIdx.x * TW + c;
    const bool ok = col < ncol;
    const long cb = ok ? (col / cdiv) * outer + (col % cdiv) : 0;
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
                const T s = ok ? ldg_t(&scale[cb + m * lstride]) : (T)0;
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

// ---------------------------------------------------------------------------------------
// Pipelined strided pass: persistent CTAs walk the tiles of TW columns; the tile
// after the current one is copied global -> shared with cp.async while the current one is
// transformed, so the HBM latency is hidden behind the butterflies. The tile's shared
// buffer (L rows of TW padded columns) also serves as the exchange buffer once stage A has
// read it. Mode 2 computes the spectral factor from eigenvalue sums (one value per column,
// the line's values in shared memory), so it reads nothing more than the spectrum.
template <int BYTES>
__device__ __forceinline__ void fr_cp_async(void* smem, const void* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
    else if constexpr (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void fr_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void fr_cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void fr_cp_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ float fr_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double fr_rcp(double x) { return 1.0 / x; }

template <typename T, int R1, int R2>
struct PipeShape {
    static constexpr int L = R1 * R2;
    static constexpr int RM = R1 > R2 ? R1 : R2;
    static constexpr int NT = sizeof(T) == 8 ? 128 : 256;   // 128-byte rows of TW complex values
    static constexpr int TW = NT / RM;
    static constexpr int SP = TW + 1;
    static constexpr int PER = L * TW / NT;   // copies per thread per tile
    static constexpr size_t smem(bool scaled) {
        return 2 * (size_t)L * SP * sizeof(cplx<T>) + (scaled ? (size_t)L * sizeof(T) : 0);
    }
    static constexpr size_t smem_max() { return smem(true) > smem(false) ? smem(true) : smem(false); }
};

// Same modes and addressing as k_fft_strided_reg<T, R1, R2>; grid = any number of CTAs
// (persistent), dynamic shared memory PipeShape::smem(mode == 2). Mode 2 forms the spectral
// factor 1 / (N (lambda_col + lambda_line[m])) from N-scaled eigenvalue sums instead of
// reading a table: eig[col] for the ncol columns, eig[ncol + m] along the line (L values),
// eig[ncol + L] for the mean mode (column 0, m = 0); the factor's rounding differs from the
// FP64-built table by about one unit in the last place.
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(PipeShape<T, R1, R2>::NT, 2) k_fft_strided_pipe(const cplx<T>* __restrict__ tw,
                                                                                cplx<T>* __restrict__ S, long ncol,
                                                                                long cdiv, long outer, long lstride,
                                                                                int mode, const T* __restrict__ eig) {
    using Sh = PipeShape<T, R1, R2>;
    constexpr int L = Sh::L, TW = Sh::TW, SP = Sh::SP;
    extern __shared__ __align__(16) unsigned char fr_smem[];
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(fr_smem);              // [2][L * SP]
    T* sl = reinterpret_cast<T*>(buf + 2 * L * SP);                    // [L] line eigenvalues (mode 2)
    const long ntiles = (ncol + TW - 1) / TW;
    const int c = threadIdx.x % TW;
    const int q = threadIdx.x / TW;
    // copy e = threadIdx.x + NT t of a tile is element (column e % TW, row e / TW); NT is a
    // multiple of TW, so a thread's column is the same for all its copies: one address
    // computation per tile, then row steps of (NT / TW) lstride
    static_assert(Sh::NT % TW == 0, "tile columns must divide the CTA size");
    constexpr int MSTEP = Sh::NT / TW;
    auto issue = [&](long tile, int b) {
        cplx<T>* dst = buf + b * L * SP;
        const long col = tile * TW + c;
        const bool ok = col < ncol;
        const int nb = ok ? (int)sizeof(cplx<T>) : 0;
        const long base = ok ? (col / cdiv) * outer + (col % cdiv) + (long)q * lstride : 0;
        const long step = ok ? (long)MSTEP * lstride : 0;
#pragma unroll
        for (int t = 0; t < Sh::PER; ++t) {
            const int m = q + MSTEP * t;
            fr_cp_async<sizeof(cplx<T>)>(dst + m * SP + c, S + base + t * step, nb);
        }
        fr_cp_commit();
    };
    // a thread's stage-A index j = q is the same for every tile (and for the inverse's stage A
    // in mode 2): its twiddles W_L^{q k1} are loaded once. k1 < max(R1, R2) where q < min(R1, R2)
    // (both stages), else k1 < min(R1, R2); q k1 < L in both cases.
    constexpr int RMIN = R1 < R2 ? R1 : R2;
    cplx<T> twr[Sh::RM];
    {
        const int kmax = q < RMIN ? Sh::RM : RMIN;
#pragma unroll
        for (int k1 = 0; k1 < Sh::RM; ++k1) twr[k1] = (k1 > 0 && k1 < kmax) ? ldg_c(&tw[q * k1]) : cplx<T>{(T)1, (T)0};
    }
    T inv_n = (T)0;
    if (mode == 2) {
        for (int m = threadIdx.x; m < L; m += Sh::NT) sl[m] = eig[ncol + m];   // visible after the first barrier
        inv_n = eig[ncol + L];
    }
    long tile = blockIdx.x;
    int b = 0;
    if (tile < ntiles) issue(tile, 0);
    for (; tile < ntiles; tile += gridDim.x, b ^= 1) {
        const long next = tile + gridDim.x;
        if (next < ntiles) issue(next, b ^ 1);
        else fr_cp_commit();   // empty group: the wait below always leaves one group pending
        fr_cp_wait1();
        __syncthreads();
        cplx<T>* X = buf + b * L * SP;
        const long col = tile * TW + c;
        const bool ok = col < ncol;
        const long cb = ok ? (col / cdiv) * outer + (col % cdiv) : 0;
        const T lc = (mode == 2 && ok) ? __ldg(&eig[col]) : (T)1;
        cplx<T> v[Sh::RM];
        // forward stage A: thread (c, j = q < R2)
        if (q < R2) {
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                cplx<T> z = X[(q + R2 * r) * SP + c];
                if (mode == 1) z = cconj(z);
                v[r] = z;
            }
            stage_a_w<T, R1>(v, q, twr);
        }
        __syncthreads();   // the tile has been read: X becomes the exchange buffer
        if (q < R2) {
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) X[(q * R1 + k1) * SP + c] = v[k1];
        }
        __syncthreads();
        if (q < R1) {
#pragma unroll
            for (int j = 0; j < R2; ++j) v[j] = X[(j * R1 + q) * SP + c];
            DftR<T, R2>::run(v);   // v[k2] = X[q + R1 k2]
        }
        if (mode == 2) {
            if (q < R1) {
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) {
                    const int m = q + R1 * k2;
                    const T s = (col == 0 && m == 0) ? inv_n : fr_rcp(lc + sl[m]);
                    v[k2] = {v[k2].re * s, -v[k2].im * s};
                }
                stage_a_w<T, R2>(v, q, twr);
            }
            __syncthreads();
            if (q < R1) {
#pragma unroll
                for (int k1 = 0; k1 < R2; ++k1) X[(q * R2 + k1) * SP + c] = v[k1];
            }
            __syncthreads();
            if (q < R2) {
#pragma unroll
                for (int j = 0; j < R1; ++j) v[j] = X[(j * R2 + q) * SP + c];
                DftR<T, R1>::run(v);
                if (ok) {
#pragma unroll
                    for (int k2 = 0; k2 < R1; ++k2) S[cb + (long)(q + R2 * k2) * lstride] = cconj(v[k2]);
                }
            }
        } else if (q < R1 && ok) {
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                cplx<T> z = v[k2];
                if (mode == 1) z = cconj(z);
                S[cb + (long)(q + R1 * k2) * lstride] = z;
            }
        }
        __syncthreads();   // buffer b is refilled two tiles ahead
    }
    fr_cp_wait0();
}

// Pipelined inverse x pass: a tile of TW line pairs is one contiguous block of the
// half spectrum (2 TW rows of nxh complex), copied with 16-byte cp.async into a double
// buffer while the previous tile is transformed. Needs a 16-byte aligned spectrum (checked
// by the caller); the tail of the last tile is zero-filled (src-size operand). (The same
// staging for the forward pass measured slower than its direct register loads.)
__device__ __forceinline__ void fr_cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}

template <typename T, int R1, int R2>
struct PipeX {
    static constexpr int L = R1 * R2;
    static constexpr int RM = R1 > R2 ? R1 : R2;
    static constexpr int NT = sizeof(T) == 8 ? 128 : 256;
    static constexpr int TW = NT / RM;          // line pairs per tile
    static constexpr int SR = L + L / 16 + 1;   // padded exchange row
    static constexpr int EPC = 16 / (int)sizeof(cplx<T>);   // complex values per 16-byte chunk
    static constexpr size_t smem_c2r(int nxh) {
        return 2 * (((size_t)2 * TW * nxh * sizeof(cplx<T>) + 15) & ~size_t(15)) + (size_t)TW * SR * sizeof(cplx<T>);
    }
};

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(PipeX<T, R1, R2>::NT, 2) k_fft_x_c2r_pipe(const cplx<T>* __restrict__ tw,
                                                                          const cplx<T>* __restrict__ S,
                                                                          T* __restrict__ out, int lines, int nxh) {
    using Sh = PipeX<T, R1, R2>;
    constexpr int L = Sh::L, TW = Sh::TW, RM = Sh::RM, SR = Sh::SR;
    extern __shared__ __align__(16) unsigned char fx_smem[];
    const int rawc = (int)(((size_t)2 * TW * nxh * sizeof(cplx<T>) + 15) / 16) * Sh::EPC;   // complex per buffer
    cplx<T>* raw = reinterpret_cast<cplx<T>*>(fx_smem);           // [2][rawc]
    cplx<T>* ex = raw + 2 * rawc;                                 // [TW][SR]
    const long npairs = ((long)lines + 1) / 2;
    const long ntiles = (npairs + TW - 1) / TW;
    const long total = (long)lines * nxh;      // complex values in the half spectrum
    const int nch = (2 * TW * nxh + Sh::EPC - 1) / Sh::EPC;   // 16-byte chunks per tile
    auto sidx = [](int m) { return m + (m >> 4); };
    auto issue = [&](long tile, int b) {
        const long c0 = tile * 2 * TW * nxh;
        for (int ch = threadIdx.x; ch < nch; ch += Sh::NT) {
            const long e = c0 + (long)Sh::EPC * ch;
            const long left = total - e;
            const int nb = left >= Sh::EPC ? 16 : (left > 0 ? (int)(left * sizeof(cplx<T>)) : 0);
            fr_cp_async16(raw + b * rawc + Sh::EPC * ch, nb > 0 ? S + e : S, nb);
        }
        fr_cp_commit();
    };
    const int q = threadIdx.x % RM;
    const int c = threadIdx.x / RM;
    cplx<T> twr[R1];   // W_L^{q k1}: the same for every tile
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) twr[k1] = (k1 > 0 && q < R2) ? ldg_c(&tw[q * k1]) : cplx<T>{(T)1, (T)0};
    long tile = blockIdx.x;
    int b = 0;
    if (tile < ntiles) issue(tile, 0);
    for (; tile < ntiles; tile += gridDim.x, b ^= 1) {
        const long next = tile + gridDim.x;
        if (next < ntiles) issue(next, b ^ 1);
        else fr_cp_commit();
        fr_cp_wait1();
        __syncthreads();
        const cplx<T>* rw = raw + b * rawc;
        // Z = A + i B over the full line (Hermitian extension), conjugated for the inverse
        for (int item = threadIdx.x; item < TW * L; item += Sh::NT) {
            const int cc = item / L, m = item - cc * L;
            const bool upper = m >= nxh;
            const int src = upper ? L - m : m;
            cplx<T> A = rw[(2 * cc) * nxh + src];
            cplx<T> B = rw[(2 * cc + 1) * nxh + src];
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
        cplx<T> v[RM];
        if (q < R2) {
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = ex[c * SR + sidx(q + R2 * r)];
            stage_a_w<T, R1>(v, q, twr);
        }
        __syncthreads();
        if (q < R2) {
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) ex[c * SR + sidx(q * R1 + k1)] = v[k1];
        }
        __syncthreads();
        if (q < R1) {
            const long la = 2 * (tile * TW + c), lb = la + 1;
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
        __syncthreads();   // ex and raw[b] are free
    }
    fr_cp_wait0();
}

// x pass, real lines -> half spectra. CTA handles TW line pairs packed as a + i b per tile and
// walks the tiles (grid = tiles, or fewer CTAs that stay resident; the twiddles of a thread's
// stage-A index are loaded once). Thread mapping (j fastest) keeps the loads along a line contiguous.
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 128 : 256, 3) k_fft_x_r2c_reg(const cplx<T>* __restrict__ tw, const T* __restrict__ in,
                                                       cplx<T>* __restrict__ S, int lines, int nxh) {
    using Sh = RegShape<T, R1, R2>;
    constexpr int L = Sh::L, TW = Sh::TW, RM = Sh::RM;
    constexpr int SR = L + L / 16 + 1;   // padded row per pair (breaks power-of-two strides)
    __shared__ cplx<T> ex[TW * SR];
    const int q = threadIdx.x % RM;      // j (stage A) / k1 (stage B)
    const int c = threadIdx.x / RM;
    auto sidx = [](int m) { return m + (m >> 4); };
    // FP32: the twiddles stay in registers; FP64 (one tile per CTA, register-heavy) loads them per use
    constexpr int NTW = sizeof(T) == 4 ? R1 : 1;
    cplx<T> twr[NTW];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) twr[k1] = (k1 > 0 && q < R2) ? ldg_c(&tw[q * k1]) : cplx<T>{(T)1, (T)0};
    }
    const long ntiles = (((long)lines + 1) / 2 + TW - 1) / TW;
    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long la = 2 * (tile * TW + c), lb = la + 1;
        cplx<T> v[RM];
        if (q < R2) {
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                const int m = q + R2 * r;
                v[r] = {la < lines ? in[la * L + m] : (T)0, lb < lines ? in[lb * L + m] : (T)0};
            }
            if constexpr (sizeof(T) == 4)
                stage_a_w<T, R1>(v, q, twr);
            else
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
        // split Z = A + i B into the half spectra of a and b (nxh = L / 2 + 1): thread (pair cs,
        // frequency kk < L / 2), PPI pairs per sweep; the kk = 0 thread also writes kk = L / 2
        const T h = (T)0.5;
        constexpr int LH = L / 2, PPI = Sh::NT / LH;   // threads >= PPI LH idle here (LH not dividing NT)
        const int kk = threadIdx.x % LH, cs = threadIdx.x / LH;
#pragma unroll
        for (int it = 0; it < (TW + PPI - 1) / PPI; ++it) {
            const int cc = it * PPI + cs;
            if (cs >= PPI || cc >= TW) break;
            const long a = 2 * (tile * TW + cc), b = a + 1;
            const cplx<T> Z = ex[cc * SR + sidx(kk)];
            const cplx<T> Zc = cconj(ex[cc * SR + sidx(kk == 0 ? 0 : L - kk)]);
            if (a < lines) S[a * nxh + kk] = {h * (Z.re + Zc.re), h * (Z.im + Zc.im)};
            if (b < lines) S[b * nxh + kk] = {h * (Z.im - Zc.im), -h * (Z.re - Zc.re)};
            if (kk == 0) {
                const cplx<T> Zn = ex[cc * SR + sidx(LH)];
                const cplx<T> Znc = cconj(Zn);
                if (a < lines) S[a * nxh + LH] = {h * (Zn.re + Znc.re), h * (Zn.im + Znc.im)};
                if (b < lines) S[b * nxh + LH] = {h * (Zn.im - Znc.im), -h * (Zn.re - Znc.re)};
            }
        }
        __syncthreads();   // ex is rewritten by the next tile
    }
}

// x pass, half spectra -> real lines (unnormalised inverse).
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 128 : 256, sizeof(T) == 8 ? 3 : 2) k_fft_x_c2r_reg(const cplx<T>* __restrict__ tw, const cplx<T>* __restrict__ S,
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
