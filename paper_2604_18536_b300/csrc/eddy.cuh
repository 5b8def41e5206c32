// Eddy-viscosity closure models (paper App. "Eddy-viscosity models"; constants of Sec. 6.3)
// on 3-D grids with x and z periodic and uniform and y periodic-uniform or a no-slip wall
// direction (possibly stretched): the LES baselines of the learned closure and the channel LES.
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
// Walls in y (WALL): across a wall u^x, u^z take the odd ghost and u^y is 0 (the forward
// operator's rules), nu_t takes the even ghost (the mirrored cell); the spacings are per row
// (d_y[j], h_y[j], and h_y[-1] = d_y[0]); the filter width is (d_x d_y[j] d_z)^(1/3).
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
    // wall-normal y (WALL): per-row arrays of ny values
    const T* idy;  // 1 / d_y[j]
    const T* ihy;  // 1 / h_y[j] (h_y[ny-1] = d_y[ny-1])
    const T* cd2y; // (C D_j)^2
    const T* w2y;  // d_y[j]^2
};

// u^c at (i, j, k): x, z wrap; beyond a wall in y u^y is 0 and u^x, u^z take the odd ghost.
template <typename T, bool WALL>
__device__ __forceinline__ T eval_u(const T* __restrict__ u, size_t N, int c, int i, int j, int k, int nx, int ny,
                                    int nz) {
    i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
    k = k < 0 ? k + nz : (k >= nz ? k - nz : k);
    T s = (T)1;
    if (WALL) {
        if (j < 0 || j >= ny) {
            if (c == 1) return (T)0;
            j = j < 0 ? 0 : ny - 1;
            s = (T)-1;
        }
    } else {
        j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
    }
    return s * __ldg(&u[c * N + ((size_t)k * ny + j) * nx + i]);
}

// nu_t at (i, j, k): x, z wrap; beyond a wall in y the even ghost.
template <typename T, bool WALL>
__device__ __forceinline__ T eval_nu(const T* __restrict__ nu, int i, int j, int k, int nx, int ny, int nz) {
    i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
    k = k < 0 ? k + nz : (k >= nz ? k - nz : k);
    if (WALL) j = j < 0 ? 0 : (j >= ny ? ny - 1 : j);
    else j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
    return __ldg(&nu[((size_t)k * ny + j) * nx + i]);
}

// 1 / h_b at index m of direction b (m = -1: the spacing below the first cell).
template <typename T, bool WALL>
__device__ __forceinline__ T inv_h(const EddyCoef<T>& c, int b, int m) {
    if (WALL && b == 1) return m < 0 ? __ldg(&c.idy[0]) : __ldg(&c.ihy[m]);
    return c.id[b];
}
template <typename T, bool WALL>
__device__ __forceinline__ T inv_d(const EddyCoef<T>& c, int b, int m) {
    if (WALL && b == 1) return __ldg(&c.idy[m]);
    return c.id[b];
}

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
__device__ __forceinline__ T eddy_model(const EddyCoef<T>& c, const T (&A)[3][3], T CD2, T w2y) {
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
        return CD2 * sqrt((T)2 * ss);
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
        return den > (T)0 ? CD2 * sd * sqrt(sd) / den : (T)0;
    } else if constexpr (MODEL == EDDY_QR) {
        T rs = (T)0;   // tr(S^3)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) rs = fma(S[a][b], S[b][0] * S[0][a] + S[b][1] * S[1][a] + S[b][2] * S[2][a], rs);
        rs = rs / (T)3;
        return ss > (T)0 ? CD2 * fabs(rs) / ((T)0.5 * ss) : (T)0;
    } else {   // Vreman
        T beta[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                beta[i][j] = c.w2[0] * A[i][0] * A[j][0] + w2y * A[i][1] * A[j][1] + c.w2[2] * A[i][2] * A[j][2];
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
template <typename T, int MODEL, bool WALL>
__global__ void __launch_bounds__(256) k_eddy_nut(EddyCoef<T> c, const T* __restrict__ u, T* __restrict__ nut) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    if (i >= nx || j >= ny) return;
    const size_t N = (size_t)nx * ny * nz;
    const int o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    const int I3[3] = {i, j, k};
    auto U = [&](int comp, int di, int dj, int dk) { return eval_u<T, WALL>(u, N, comp, i + di, j + dj, k + dk, nx, ny, nz); };
    T A[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        A[a][a] = (U(a, 0, 0, 0) - U(a, -o[a][0], -o[a][1], -o[a][2])) * inv_d<T, WALL>(c, a, I3[a]);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b == a) continue;
            // mean of E_ab over the edges (I), (I - e_b), (I - e_a), (I - e_a - e_b):
            // E_ab(J) = (u^a_{J+e_b} - u^a_J) / h_b[J_b]
            T sum = (T)0;
#pragma unroll
            for (int sa = 0; sa < 2; ++sa)
#pragma unroll
                for (int sb = 0; sb < 2; ++sb) {
                    const int ji = -sa * o[a][0] - sb * o[b][0], jj = -sa * o[a][1] - sb * o[b][1],
                              jk = -sa * o[a][2] - sb * o[b][2];
                    const T e = (U(a, ji + o[b][0], jj + o[b][1], jk + o[b][2]) - U(a, ji, jj, jk)) *
                                inv_h<T, WALL>(c, b, I3[b] - sb);
                    // the edge below a wall in a carries u^a = 0 on both ends when a is y
                    sum += (WALL && a == 1 && sa == 1 && j == 0) ? (T)0 : e;
                }
            A[a][b] = (T)0.25 * sum;
        }
    }
    const T cd2 = WALL ? __ldg(&c.cd2y[j]) : c.CD2;
    const T w2y = WALL ? __ldg(&c.w2y[j]) : c.w2[1];
    nut[((size_t)k * ny + j) * nx + i] = eddy_model<T, MODEL>(c, A, cd2, w2y);
}

// e^a = sum_b delta_b (2 nu_t S_ab) on the a-faces of every cell (stored top wall faces of u^y:
// 0). Same launch shape.
template <typename T, bool WALL>
__global__ void __launch_bounds__(256) k_eddy_div(EddyCoef<T> c, const T* __restrict__ u, const T* __restrict__ nut,
                                                  T* __restrict__ e) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    if (i >= nx || j >= ny) return;
    const size_t N = (size_t)nx * ny * nz;
    const size_t I = ((size_t)k * ny + j) * nx + i;
    const int o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    const int I3[3] = {i, j, k};
    auto U = [&](int comp, int di, int dj, int dk) { return eval_u<T, WALL>(u, N, comp, i + di, j + dj, k + dk, nx, ny, nz); };
    auto V = [&](int di, int dj, int dk) { return eval_nu<T, WALL>(nut, i + di, j + dj, k + dk, nx, ny, nz); };
    // E_ab on the (a, b) edge of cell I + (di, dj, dk), its b index m
    auto E = [&](int a, int b, int di, int dj, int dk, int m) {
        return (U(a, di + o[b][0], dj + o[b][1], dk + o[b][2]) - U(a, di, dj, dk)) * inv_h<T, WALL>(c, b, m);
    };
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (WALL && a == 1 && j == ny - 1) {
            e[N + I] = (T)0;
            continue;
        }
        const int ai = o[a][0], aj = o[a][1], ak = o[a][2];
        // b == a: (T_aa(I + e_a) - T_aa(I)) / h_a
        const T Saa_p = (U(a, ai, aj, ak) - U(a, 0, 0, 0)) * inv_d<T, WALL>(c, a, I3[a] + 1);
        const T Saa_0 = (U(a, 0, 0, 0) - U(a, -ai, -aj, -ak)) * inv_d<T, WALL>(c, a, I3[a]);
        T acc = (T)2 * (V(ai, aj, ak) * Saa_p - V(0, 0, 0) * Saa_0) * inv_h<T, WALL>(c, a, I3[a]);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b == a) continue;
            const int bi = o[b][0], bj = o[b][1], bk = o[b][2];
            // upper edge (I; a, b) and lower edge (I - e_b; a, b)
            const T Sup = (T)0.5 * (E(a, b, 0, 0, 0, I3[b]) + E(b, a, 0, 0, 0, I3[a]));
            const T nup = (T)0.25 * (V(0, 0, 0) + V(ai, aj, ak) + V(bi, bj, bk) + V(ai + bi, aj + bj, ak + bk));
            T Elo_ba = E(b, a, -bi, -bj, -bk, I3[a]);
            if (WALL && b == 1 && j == 0) Elo_ba = (T)0;      // u^y below the bottom wall
            const T Slo = (T)0.5 * (E(a, b, -bi, -bj, -bk, I3[b] - 1) + Elo_ba);
            const T nlo = (T)0.25 * (V(-bi, -bj, -bk) + V(ai - bi, aj - bj, ak - bk) + V(0, 0, 0) + V(ai, aj, ak));
            acc += (T)2 * (nup * Sup - nlo * Slo) * inv_d<T, WALL>(c, b, I3[b]);
        }
        e[a * N + I] = acc;
    }
}

}  // namespace ins
