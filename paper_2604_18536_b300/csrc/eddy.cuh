// Eddy-viscosity closure models (paper App. "Eddy-viscosity models"; constants of Sec. 6.3)
// on 3-D periodic uniform grids: the LES baselines of the learned closure.
//
// The term added to F is e^a = sum_b delta_b (2 nu_t S_ab) (the eddy-viscous stress
// divergence; dissipative). Staggered points:
//   S_aa at cell I:           (u^a_I - u^a_{I-e_a}) / d_a
//   S_ab on the (a, b) edge of I (face a of I, face b of I):
//                             ((u^a_{I+e_b} - u^a_I) / d_b + (u^b_{I+e_a} - u^b_I) / d_a) / 2
//   A_ab at cell I (a != b):  mean of delta_b u^a on the four (a, b) edges around I; the
//                             edge differences telescope to
//                             (u^a_{I+e_b} - u^a_{I-e_b} + u^a_{I-e_a+e_b} - u^a_{I-e_a-e_b}) / (4 d_b)
//   nu_t at cell I from A(I) by the model; on the (a, b) edge of I the mean of nu_t at I,
//   I + e_a, I + e_b, I + e_a + e_b.
// Models (D the filter width, S = sym A):
//   Smagorinsky (C D)^2 sqrt(2 S:S); WALE (C D)^2 (Sd:Sd)^(3/2) / ((S:S)^(5/2) + (Sd:Sd)^(5/4)),
//   Sd = sym(A A) - tr(A A)/3 I; QR (C D)^2 |tr(S^3)/3| / (S:S/2); Vreman
//   C^2 sqrt(B_beta / (tr(A A^T)/2)), beta_ij = sum_m d_m^2 A_im A_jm; constant: nu_t = C.
// Divisions by a vanishing invariant give nu_t = 0. Two kernels, one thread per cell:
// k_eddy_nut (reads u, writes nu_t), k_eddy_div (reads u and nu_t, writes e); neighbour
// values come through the read-only cache (LES sizes; not a bandwidth-critical path).
#pragma once

#include "common.cuh"

namespace ins {

enum EddyKind { EDDY_NONE = 0, EDDY_SMAGORINSKY = 1, EDDY_WALE = 2, EDDY_QR = 3, EDDY_VREMAN = 4, EDDY_CONSTANT = 5 };

template <typename T>
struct EddyCoef {
    int nx, ny, nz;
    T id[3];       // 1 / d_a (uniform spacing)
    T w2[3];       // d_a^2 (Vreman)
    T CD2;         // (C D)^2
    T C2;          // C^2 (Vreman), C (constant model)
};

template <typename T>
struct Idx3 {
    int nx, ny, nz;
    __device__ __forceinline__ int at(int i, int j, int k) const {
        i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
        j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
        k = k < 0 ? k + nz : (k >= nz ? k - nz : k);
        return (k * ny + j) * nx + i;
    }
};

template <typename T, int MODEL>
__device__ __forceinline__ T eddy_model(const EddyCoef<T>& c, const T (&A)[3][3]) {
    T S[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) S[a][b] = (T)0.5 * (A[a][b] + A[b][a]);
    T ss = (T)0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) ss = fma(S[a][b], S[a][b], ss);
    if constexpr (MODEL == EDDY_CONSTANT) {
        return c.C2;
    } else if constexpr (MODEL == EDDY_SMAGORINSKY) {
        return c.CD2 * sqrt((T)2 * ss);
    } else if constexpr (MODEL == EDDY_WALE) {
        T A2[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) A2[a][b] = A[a][0] * A[0][b] + A[a][1] * A[1][b] + A[a][2] * A[2][b];
        const T tr3 = (A2[0][0] + A2[1][1] + A2[2][2]) / (T)3;
        T sd = (T)0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                T v = (T)0.5 * (A2[a][b] + A2[b][a]);
                if (a == b) v -= tr3;
                sd = fma(v, v, sd);
            }
        const T den = ss * ss * sqrt(ss) + sd * sqrt(sqrt(sd));
        return den > (T)0 ? c.CD2 * sd * sqrt(sd) / den : (T)0;
    } else if constexpr (MODEL == EDDY_QR) {
        T rs = (T)0;   // tr(S^3)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) rs = fma(S[a][b], S[b][0] * S[0][a] + S[b][1] * S[1][a] + S[b][2] * S[2][a], rs);
        rs = rs / (T)3;
        return ss > (T)0 ? c.CD2 * fabs(rs) / ((T)0.5 * ss) : (T)0;
    } else {   // Vreman
        T beta[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                beta[i][j] = c.w2[0] * A[i][0] * A[j][0] + c.w2[1] * A[i][1] * A[j][1] + c.w2[2] * A[i][2] * A[j][2];
        T B = beta[0][0] * beta[1][1] - beta[0][1] * beta[0][1] + beta[0][0] * beta[2][2] - beta[0][2] * beta[0][2] +
              beta[1][1] * beta[2][2] - beta[1][2] * beta[1][2];
        T aa = (T)0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) aa = fma(A[a][b], A[a][b], aa);
        const T den = (T)0.5 * aa;
        return den > (T)0 ? c.C2 * sqrt(fmax(B, (T)0) / den) : (T)0;
    }
}

// nu_t at every cell. Block (32, 8), grid (ceil(nx/32), ceil(ny/8), nz).
template <typename T, int MODEL>
__global__ void __launch_bounds__(256) k_eddy_nut(EddyCoef<T> c, const T* __restrict__ u, T* __restrict__ nut) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= c.nx || j >= c.ny) return;
    const Idx3<T> X{c.nx, c.ny, c.nz};
    const size_t N = (size_t)c.nx * c.ny * c.nz;
    const int o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    T A[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T* ua = u + a * N;
        A[a][a] = (__ldg(&ua[X.at(i, j, k)]) - __ldg(&ua[X.at(i - o[a][0], j - o[a][1], k - o[a][2])])) * c.id[a];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b == a) continue;
            const int bi = o[b][0], bj = o[b][1], bk = o[b][2];
            const int ai = o[a][0], aj = o[a][1], ak = o[a][2];
            const T s = __ldg(&ua[X.at(i + bi, j + bj, k + bk)]) - __ldg(&ua[X.at(i - bi, j - bj, k - bk)]) +
                        __ldg(&ua[X.at(i - ai + bi, j - aj + bj, k - ak + bk)]) -
                        __ldg(&ua[X.at(i - ai - bi, j - aj - bj, k - ak - bk)]);
            A[a][b] = (T)0.25 * s * c.id[b];
        }
    }
    nut[X.at(i, j, k)] = eddy_model<T, MODEL>(c, A);
}

// e^a = sum_b delta_b (2 nu_t S_ab) on the a-faces of every cell. Same launch shape.
template <typename T>
__global__ void __launch_bounds__(256) k_eddy_div(EddyCoef<T> c, const T* __restrict__ u, const T* __restrict__ nut,
                                                  T* __restrict__ e) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= c.nx || j >= c.ny) return;
    const Idx3<T> X{c.nx, c.ny, c.nz};
    const size_t N = (size_t)c.nx * c.ny * c.nz;
    const int o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    auto U = [&](int a, int di, int dj, int dk) { return __ldg(&u[a * N + X.at(i + di, j + dj, k + dk)]); };
    auto V = [&](int di, int dj, int dk) { return __ldg(&nut[X.at(i + di, j + dj, k + dk)]); };
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int ai = o[a][0], aj = o[a][1], ak = o[a][2];
        // b == a: (T_aa(I + e_a) - T_aa(I)) / d_a
        const T Saa_p = (U(a, ai, aj, ak) - U(a, 0, 0, 0)) * c.id[a];
        const T Saa_0 = (U(a, 0, 0, 0) - U(a, -ai, -aj, -ak)) * c.id[a];
        T acc = (T)2 * (V(ai, aj, ak) * Saa_p - V(0, 0, 0) * Saa_0) * c.id[a];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b == a) continue;
            const int bi = o[b][0], bj = o[b][1], bk = o[b][2];
            // T_ab on the (a, b) edge of J = I + s e_b, s = 0 (upper) and -1 (lower)
            T t[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int si = -q * bi, sj = -q * bj, sk = -q * bk;
                const T Sab = (T)0.5 * ((U(a, si + bi, sj + bj, sk + bk) - U(a, si, sj, sk)) * c.id[b] +
                                        (U(b, si + ai, sj + aj, sk + ak) - U(b, si, sj, sk)) * c.id[a]);
                const T nue = (T)0.25 * (V(si, sj, sk) + V(si + ai, sj + aj, sk + ak) + V(si + bi, sj + bj, sk + bk) +
                                         V(si + ai + bi, sj + aj + bj, sk + ak + bk));
                t[q] = (T)2 * nue * Sab;
            }
            acc += (t[0] - t[1]) * c.id[b];
        }
        e[a * N + X.at(i, j, k)] = acc;
    }
}

}  // namespace ins
