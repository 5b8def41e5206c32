// Pullback of F on wall-bounded grids (channel: x, z periodic and uniform, y a no-slip wall,
// possibly stretched) for the step VJP (paper Sec. 3.4 and App. B pullbacks).
//
// k_adj_rhs_wall_g: J_F^T w in gather form. Every face output F^a_I is the sum of the App. A /
// App. B terms, convection as flux differences of products of two interpolations of u and
// diffusion nu (c+ u_{I+e_b} + c- u_{I-e_b} - (c+ + c-) u_I); the transposes follow the
// forward boundary rules: x and z wrap; across a wall in y, u^y is 0 (wall-normal velocity)
// and u^x, u^z take the odd ghost (minus the first or last stored value), so a ghost's
// derivative lands on that stored value with a minus sign. The stored top wall faces of u^y
// are not unknowns (cotangent 0, value 0).
//
// Also: the projection pullback P^T = M Omega P Omega^-1 M (Omega the face volumes, whose
// x/z factors cancel: rows of u^x, u^z are scaled by d_y[j], rows of u^y by h_y[j]) as two
// passes around the Poisson solve; the stage finish ubar0 += q, kbar = dt (b ybar + a q) is
// fused into k_adj_rhs_wall_g.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace ins {

// J_F^T w in gather form (one thread per cell, no atomics), fused with the stage finish.
// Every convective term of F is a flux difference -k_I (phi(I) - phi(I - e)) over an
// edge flux phi = A B (a product of two sums of u); summing by parts, an edge E carries the
// flux cotangent phibar(E) = k_{E+e} w(E + e) - k_E w(E), and u gathers phibar(E) times the
// other factor over the edges whose factors contain it. Fluxes (E = (i, j, k), rows j):
//   xx = (u^x_E + u^x_{E+x})^2, k = 1/(4 d_x) in F^x        yy, zz likewise (k_yy = 1/(4 h_y[j]))
//   xy = (u^y_E + u^y_{E+x})(u^x_E + u^x_{E+y}), k = 1/(4 d_y[j]) in F^x along y
//   xz = (u^z_E + u^z_{E+x})(u^x_E + u^x_{E+z}), k = 1/(4 d_z) in F^x along z and 1/(4 d_x)
//        in F^z along x (the same product)
//   zy = (u^y_E + u^y_{E+z})(u^z_E + u^z_{E+y}), k = 1/(4 d_y[j]) in F^z along y
//   yx = (wl_j u^x_E + wr_j u^x_{E+y})(u^y_E + u^y_{E+x}), k = 1/(2 d_x) in F^y along x
//   yz = (wl_j u^z_E + wr_j u^z_{E+y})(u^y_E + u^y_{E+z}), k = 1/(2 d_z) in F^y along z
// (wl, wr the volume weights of the y interpolation). Cotangents of faces that are not
// unknowns are 0 (rows outside the grid, the top wall faces of u^y); u^y is 0 below the
// bottom wall and on the top wall faces. Every flux that reaches a wall ghost of u^x or u^z is
// multiplied by a zero wall-normal velocity, so only the diffusion terms fold ghost
// derivatives back: -c_- w at the first row and -c_+ w at the last (odd ghosts).
// The finish: ubar0 += q, kbar = dt (bn y + an q) (kbar null: none), y = ybar or (null) the
// old ubar0; the stored top wall faces of u^y keep q = 0. nu_part: one FP64 partial of
// <w, diffusion(u) / nu> per CTA. The grid has fewer than 2^31 / 3 cells (the caller checks).

// Coefficients of wall_adj_cell for cell (i, j): x and z are uniform, so they depend on the row
// only; a z march computes them once.
template <typename T>
struct WallRowCoef {
    T fym, fy0, fyp;      // 1/(4 d_y) at rows j - 1, j, j + 1 (clamped)
    T sym, sy0, syp;      // 1/(4 h_y) at rows j - 1, j, j + 1 (clamped)
    T wl, wr, wrm;        // volume weights of row j, wr of row j - 1 (0 at j = 0)
    T cx, cx2, cz, cz2;   // 1/(4 d), 1/(2 d) of x and z
    T lx, lz;             // 1/d^2 of x and z
    T bp, bm, bpm, bmp;   // tangential y diffusion: c+_j, c-_j, c+_{j-1} (0 at j = 0), c-_{j+1} (0 at the top)
    T ap, am, apm, amp;   // u^y diffusion: a+_j, a-_j, a+_{j-1} (0 at j = 0), a-_{j+1} (0 unless j + 1 < ny - 1)
};

template <typename T, int DIM>
__device__ __forceinline__ WallRowCoef<T> wall_row_coef(const Geo<T>& G, int i, int j) {
    const int ny = G.ny;
    auto cl = [ny](int jj) { return jj < 0 ? 0 : (jj >= ny ? ny - 1 : jj); };
    auto bpy = [&](int jj) { return G.coef(1, C_INV_H, jj) * G.coef(1, C_INV_D, jj); };
    auto bmy = [&](int jj) {
        return (jj == 0 ? G.coef(1, C_INV_D, 0) : G.coef(1, C_INV_H, jj - 1)) * G.coef(1, C_INV_D, jj);
    };
    auto apy = [&](int jj) { return G.coef(1, C_INV_D, jj + 1) * G.coef(1, C_INV_H, jj); };
    auto amy = [&](int jj) { return G.coef(1, C_INV_D, jj) * G.coef(1, C_INV_H, jj); };
    WallRowCoef<T> R;
    R.fym = (T)0.25 * G.coef(1, C_INV_D, cl(j - 1));
    R.fy0 = (T)0.25 * G.coef(1, C_INV_D, j);
    R.fyp = (T)0.25 * G.coef(1, C_INV_D, cl(j + 1));
    R.sym = G.coef(1, C_CONV_AA, cl(j - 1));
    R.sy0 = G.coef(1, C_CONV_AA, j);
    R.syp = G.coef(1, C_CONV_AA, cl(j + 1));
    R.wl = G.coef(1, C_WL, j);
    R.wr = G.coef(1, C_WR, j);
    R.wrm = j > 0 ? G.coef(1, C_WR, j - 1) : (T)0;
    R.cx = G.coef(0, C_CONV_AA, i);
    R.cx2 = G.coef(0, C_CONV_AB, i);
    R.cz = DIM == 3 ? G.coef(2, C_CONV_AA, 0) : (T)0;
    R.cz2 = DIM == 3 ? G.coef(2, C_CONV_AB, 0) : (T)0;
    R.lx = G.coef(0, C_INV_H, i) * G.coef(0, C_INV_D, i);
    R.lz = DIM == 3 ? G.coef(2, C_INV_H, 0) * G.coef(2, C_INV_D, 0) : (T)0;
    R.bp = bpy(j);
    R.bm = bmy(j);
    R.bpm = j > 0 ? bpy(j - 1) : (T)0;
    R.bmp = j + 1 < ny ? bmy(j + 1) : (T)0;
    if (j < ny - 1) {
        R.ap = apy(j);
        R.am = amy(j);
    } else {
        R.ap = R.am = (T)0;
    }
    R.apm = j > 0 ? apy(j - 1) : (T)0;
    R.amp = j + 1 < ny - 1 ? amy(j + 1) : (T)0;
    return R;
}

// J_F^T w of the three faces of cell (i, j) (z index implicit in the accessor). A.u(c, di,
// dj, dk) and A.w(c, di, dj, dk) give u^c and w^c at the offset with the wall rules applied:
// u^x, u^z odd ghosts beyond the walls; u^y 0 beyond the walls and on the top wall faces; w^x,
// w^z 0 beyond the walls; w^y 0 beyond the walls and on the top wall faces. q: the pullback of
// each face (q[1] = 0 on the top wall faces), nup += w . (diffusion of u / nu) on the faces.
template <typename T, int DIM, typename Acc>
__device__ __forceinline__ void wall_adj_cell(const WallRowCoef<T>& R, int ny, T nu, int j, const Acc& A, T (&q)[3],
                                              double& nup) {
    const T fym = R.fym, fy0 = R.fy0, fyp = R.fyp, sym = R.sym, sy0 = R.sy0, syp = R.syp;
    const T wl = R.wl, wr = R.wr, wrm = R.wrm, cx = R.cx, cx2 = R.cx2, cz = R.cz, cz2 = R.cz2, lx = R.lx, lz = R.lz;
    T lpart = (T)0;   // w . (diffusion of u / nu) over the three faces
    // ---- u^x
    {
        const T u0 = A.u(0, 0, 0, 0), ue = A.u(0, 1, 0, 0), uw = A.u(0, -1, 0, 0);
        const T w0 = A.w(0, 0, 0, 0), we = A.w(0, 1, 0, 0), ww = A.w(0, -1, 0, 0);
        const T wn = A.w(0, 0, 1, 0), ws = A.w(0, 0, -1, 0);
        T a = (T)2 * cx * ((u0 + ue) * (we - w0) + (uw + u0) * (w0 - ww));
        // xy: edges P and P - y; V = u^y_E + u^y_{E+x}
        const T V0 = A.u(1, 0, 0, 0) + A.u(1, 1, 0, 0), Vs = A.u(1, 0, -1, 0) + A.u(1, 1, -1, 0);
        a += (fyp * wn - fy0 * w0) * V0 + (fy0 * w0 - fym * ws) * Vs;
        // yx: edges P (wl) and P - y (wr)
        a += cx2 * (A.w(1, 1, 0, 0) - A.w(1, 0, 0, 0)) * wl * V0 + cx2 * (A.w(1, 1, -1, 0) - A.w(1, 0, -1, 0)) * wrm * Vs;
        // diffusion (x, y; z below), ghost folds at the walls
        const T bp = R.bp, bm = R.bm;
        T d = lx * (we + ww - (T)2 * w0) + R.bpm * ws + R.bmp * wn -
              (bp + bm) * w0;
        if (j == 0) d -= bm * w0;
        if (j == ny - 1) d -= bp * w0;
        T lap = lx * (ue + uw - (T)2 * u0) + bp * A.u(0, 0, 1, 0) + bm * A.u(0, 0, -1, 0) - (bp + bm) * u0;
        if constexpr (DIM == 3) {
            const T wt = A.w(0, 0, 0, 1), wb = A.w(0, 0, 0, -1);
            const T ut = A.u(0, 0, 0, 1), ub = A.u(0, 0, 0, -1);
            // xz: edges P and P - z; V = u^z_E + u^z_{E+x}
            const T Vz0 = A.u(2, 0, 0, 0) + A.u(2, 1, 0, 0), Vzb = A.u(2, 0, 0, -1) + A.u(2, 1, 0, -1);
            const T pb0 = cz * (wt - w0) + cx * (A.w(2, 1, 0, 0) - A.w(2, 0, 0, 0));
            const T pbb = cz * (w0 - wb) + cx * (A.w(2, 1, 0, -1) - A.w(2, 0, 0, -1));
            a += pb0 * Vz0 + pbb * Vzb;
            d += lz * (wt + wb - (T)2 * w0);
            lap += lz * (ut + ub - (T)2 * u0);
        }
        q[0] = a + nu * d;
        lpart = fma(w0, lap, lpart);
    }
    // ---- u^y (not an unknown on the top wall faces)
    if (j < ny - 1) {
        const T u0 = A.u(1, 0, 0, 0), un = A.u(1, 0, 1, 0), us = A.u(1, 0, -1, 0);
        const T w0 = A.w(1, 0, 0, 0), wn = A.w(1, 0, 1, 0), ws = A.w(1, 0, -1, 0);
        const T we = A.w(1, 1, 0, 0), ww = A.w(1, -1, 0, 0);
        T a = (T)2 * ((u0 + un) * (syp * wn - sy0 * w0) + (us + u0) * (sy0 * w0 - sym * ws));
        // xy: edges P and P - x; T = u^x_E + u^x_{E+y}
        const T x0 = A.u(0, 0, 0, 0), xn = A.u(0, 0, 1, 0), xw = A.u(0, -1, 0, 0), xwn = A.u(0, -1, 1, 0);
        a += (fyp * A.w(0, 0, 1, 0) - fy0 * A.w(0, 0, 0, 0)) * (x0 + xn) +
             (fyp * A.w(0, -1, 1, 0) - fy0 * A.w(0, -1, 0, 0)) * (xw + xwn);
        // yx: edges P and P - x; A = wl u^x_E + wr u^x_{E+y}
        a += cx2 * (we - w0) * (wl * x0 + wr * xn) + cx2 * (w0 - ww) * (wl * xw + wr * xwn);
        const T ap = R.ap, am = R.am;
        T d = lx * (we + ww - (T)2 * w0) + R.apm * ws + R.amp * wn -
              (ap + am) * w0;
        T lap = lx * (A.u(1, 1, 0, 0) + A.u(1, -1, 0, 0) - (T)2 * u0) + ap * un + am * us - (ap + am) * u0;
        if constexpr (DIM == 3) {
            const T wt = A.w(1, 0, 0, 1), wb = A.w(1, 0, 0, -1);
            const T z0 = A.u(2, 0, 0, 0), zn = A.u(2, 0, 1, 0), zb = A.u(2, 0, 0, -1), zbn = A.u(2, 0, 1, -1);
            // zy: edges P and P - z; T = u^z_E + u^z_{E+y}
            a += (fyp * A.w(2, 0, 1, 0) - fy0 * A.w(2, 0, 0, 0)) * (z0 + zn) +
                 (fyp * A.w(2, 0, 1, -1) - fy0 * A.w(2, 0, 0, -1)) * (zb + zbn);
            // yz: edges P and P - z; A = wl u^z_E + wr u^z_{E+y}
            a += cz2 * (wt - w0) * (wl * z0 + wr * zn) + cz2 * (w0 - wb) * (wl * zb + wr * zbn);
            d += lz * (wt + wb - (T)2 * w0);
            lap += lz * (A.u(1, 0, 0, 1) + A.u(1, 0, 0, -1) - (T)2 * u0);
        }
        q[1] = a + nu * d;
        lpart = fma(w0, lap, lpart);
    } else {
        q[1] = (T)0;
    }
    // ---- u^z
    if constexpr (DIM == 3) {
        const T u0 = A.u(2, 0, 0, 0), ut = A.u(2, 0, 0, 1), ub = A.u(2, 0, 0, -1);
        const T w0 = A.w(2, 0, 0, 0), wt = A.w(2, 0, 0, 1), wb = A.w(2, 0, 0, -1);
        const T wn = A.w(2, 0, 1, 0), ws = A.w(2, 0, -1, 0);
        const T we = A.w(2, 1, 0, 0), ww = A.w(2, -1, 0, 0);
        T a = (T)2 * cz * ((u0 + ut) * (wt - w0) + (ub + u0) * (w0 - wb));
        // xz: edges P and P - x; T = u^x_E + u^x_{E+z}
        const T pb0 = cz * (A.w(0, 0, 0, 1) - A.w(0, 0, 0, 0)) + cx * (we - w0);
        const T pbw = cz * (A.w(0, -1, 0, 1) - A.w(0, -1, 0, 0)) + cx * (w0 - ww);
        a += pb0 * (A.u(0, 0, 0, 0) + A.u(0, 0, 0, 1)) + pbw * (A.u(0, -1, 0, 0) + A.u(0, -1, 0, 1));
        // zy: edges P and P - y; V = u^y_E + u^y_{E+z}
        const T V0 = A.u(1, 0, 0, 0) + A.u(1, 0, 0, 1), Vs = A.u(1, 0, -1, 0) + A.u(1, 0, -1, 1);
        a += (fyp * wn - fy0 * w0) * V0 + (fy0 * w0 - fym * ws) * Vs;
        // yz: edges P (wl) and P - y (wr)
        a += cz2 * (A.w(1, 0, 0, 1) - A.w(1, 0, 0, 0)) * wl * V0 + cz2 * (A.w(1, 0, -1, 1) - A.w(1, 0, -1, 0)) * wrm * Vs;
        const T bp = R.bp, bm = R.bm;
        T d = lx * (we + ww - (T)2 * w0) + lz * (wt + wb - (T)2 * w0) + R.bpm * ws +
              R.bmp * wn - (bp + bm) * w0;
        if (j == 0) d -= bm * w0;
        if (j == ny - 1) d -= bp * w0;
        const T lap = lx * (A.u(2, 1, 0, 0) + A.u(2, -1, 0, 0) - (T)2 * u0) + lz * (ut + ub - (T)2 * u0) +
                      bp * A.u(2, 0, 1, 0) + bm * A.u(2, 0, -1, 0) - (bp + bm) * u0;
        q[2] = a + nu * d;
        lpart = fma(w0, lap, lpart);
    }
    if constexpr (std::is_same<T, df>::value)
        nup += df_to_double(lpart);
    else
        nup += (double)lpart;
}

// Accessor of wall_adj_cell on global memory (x, z wrap; the wall rules by row). US: the storage
// type of u (the double-float pullback reads the FP64 step input and double-float stage states).
template <typename T, typename US = T>
struct GlobalWallAcc {
    const US* uu;
    const T* ww;
    int nx, ny, N, i, j, ip, im, k, kp, km;
    __device__ __forceinline__ int at(int di, int jj, int dk) const {
        const int ii = di == 0 ? i : (di > 0 ? ip : im);
        const int kk = dk == 0 ? k : (dk > 0 ? kp : km);
        return (kk * ny + jj) * nx + ii;
    }
    __device__ __forceinline__ T u(int c, int di, int dj, int dk) const {
        const int jj = j + dj;
        if (c == 1) return (jj < 0 || jj >= ny - 1) ? (T)0 : cvt_in<T>(uu[N + at(di, jj, dk)]);
        if (jj < 0) return -cvt_in<T>(uu[c * N + at(di, 0, dk)]);
        if (jj >= ny) return -cvt_in<T>(uu[c * N + at(di, ny - 1, dk)]);
        return cvt_in<T>(uu[c * N + at(di, jj, dk)]);
    }
    __device__ __forceinline__ T w(int c, int di, int dj, int dk) const {
        const int jj = j + dj;
        if (c == 1) return (jj < 0 || jj >= ny - 1) ? (T)0 : ww[N + at(di, jj, dk)];
        return (jj < 0 || jj >= ny) ? (T)0 : ww[c * N + at(di, jj, dk)];
    }
};

template <typename T>
struct WallAdjG {
    Geo<T> g;
    T nu;
    const double* dt_dev;
    double dt_host;
    double bn, an;
};

// finish of one cell: ubar0 += q, kbar = dt (bn y + an q). UB: the storage type of the state
// cotangents (FP64 in the double-float pullback: q is added to ubar0 in FP64).
template <typename T, int DIM, typename UB = T>
__device__ __forceinline__ void wall_adj_finish(const WallAdjG<T>& c, int N, int P, const T (&q)[3],
                                                const UB* __restrict__ ybar, UB* __restrict__ ubar0,
                                                T* __restrict__ kbar, T dtb, T dta) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const int t = a * N + P;
        const UB old = ubar0[t];
        if constexpr (std::is_same<T, UB>::value) {
            ubar0[t] = old + q[a];
            if (kbar) kbar[t] = fma(dtb, ybar ? ybar[t] : old, dta * q[a]);
        } else {
            ubar0[t] = old + df_to_double(q[a]);
            if (kbar) kbar[t] = fma(dtb, cvt_in<T>(ybar ? ybar[t] : old), dta * q[a]);
        }
    }
}

__device__ __forceinline__ void block_partial(double nup, double* __restrict__ nu_part) {
    for (int o = 16; o > 0; o >>= 1) nup += __shfl_xor_sync(0xffffffffu, nup, o);
    __shared__ double red[8];
    if (threadIdx.x == 0) red[threadIdx.y] = nup;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double sum = 0.0;
        for (int r = 0; r < 8; ++r) sum += red[r];
        nu_part[((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = sum;
    }
}

// One thread per cell, neighbours from global memory (2-D grids and FP64). Block (32, 8),
// grid (ceil(nx/32), ceil(ny/8), nz).
// US, UB: storage types of u and of the state cotangents (the double-float pullback of an FP64
// channel: T = df, u FP64 in the first stage and double-float after it, ybar and ubar0 FP64).
template <typename T, int DIM, typename US = T, typename UB = T>
__global__ void __launch_bounds__(256) k_adj_rhs_wall_g(WallAdjG<T> c, const US* __restrict__ u,
                                                        const T* __restrict__ w, const UB* __restrict__ ybar,
                                                        UB* __restrict__ ubar0, T* __restrict__ kbar,
                                                        double* __restrict__ nu_part) {
    const Geo<T>& G = c.g;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int N = nx * ny * nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    double nup = 0.0;
    if (i < nx && j < ny) {
        GlobalWallAcc<T, US> A;
        A.uu = u;
        A.ww = w;
        A.nx = nx;
        A.ny = ny;
        A.N = N;
        A.i = i;
        A.j = j;
        A.ip = i + 1 == nx ? 0 : i + 1;
        A.im = i == 0 ? nx - 1 : i - 1;
        A.k = k;
        A.kp = DIM == 3 ? (k + 1 == nz ? 0 : k + 1) : k;
        A.km = DIM == 3 ? (k == 0 ? nz - 1 : k - 1) : k;
        T q[3];
        wall_adj_cell<T, DIM>(wall_row_coef<T, DIM>(G, i, j), ny, c.nu, j, A, q, nup);
        const double dt = c.dt_dev ? *c.dt_dev : c.dt_host;
        wall_adj_finish<T, DIM, UB>(c, N, (k * ny + j) * nx + i, q, ybar, ubar0, kbar, cvt_in<T>(dt * c.bn),
                                    cvt_in<T>(dt * c.an));
    }
    block_partial(nup, nu_part);
}

// 3-D (FP32): z march over a chunk of planes per CTA; u and w of planes k - 1 .. k + 2 in a
// four-slot shared ring (34 x 10 cells: the 32 x 8 tile and a one-cell halo), stored with the
// wall rules applied, so the cell arithmetic reads shared memory without branches. Plane k + 2
// is loaded into registers at the top of iteration k and stored into the slot of plane k - 2
// before the iteration's barrier. Block (32, 8), grid (ceil(nx/32), ceil(ny/8),
// ceil(nz/kchunk)), dynamic shared memory wall_adj_smem<T>().
constexpr int WZX = 34, WZY = 10, WZP = WZX * WZY;
constexpr int WZH = WZP - 256;   // halo cells of a plane (staged by threads 0 .. 83)
template <typename T>
constexpr int wall_adj_smem() { return 4 * 6 * WZP * (int)sizeof(T); }

template <typename T>
struct SharedWallAcc {
    const T* s;     // ring base
    int so[3];      // slot offsets of planes k - 1, k, k + 1
    int c0;         // own cell in a plane
    __device__ __forceinline__ T u(int c, int di, int dj, int dk) const {
        return s[so[dk + 1] + c * WZP + c0 + dj * WZX + di];
    }
    __device__ __forceinline__ T w(int c, int di, int dj, int dk) const {
        return s[so[dk + 1] + (3 + c) * WZP + c0 + dj * WZX + di];
    }
};

// UIN: the accumulator's previous value comes from uin (the first stage of the pullback reads
// ybar there); otherwise from ubar0 itself (uin unused). US, UB: storage types of u and of the
// state cotangents (the double-float pullback of an FP64 channel: T = df, u FP64 in the first stage
// and double-float after it, ybar and ubar0 FP64 with q added in FP64).
template <typename T, bool UIN = false, typename US = T, typename UB = T>
__global__ void __launch_bounds__(256, 2) k_adj_rhs_wall_z(WallAdjG<T> c, const US* __restrict__ u,
                                                        const T* __restrict__ w, const UB* __restrict__ ybar,
                                                        UB* __restrict__ ubar0, T* __restrict__ kbar,
                                                        double* __restrict__ nu_part, int kchunk,
                                                        const UB* __restrict__ uin) {
    extern __shared__ __align__(16) unsigned char wz_smem[];
    T* const ring = reinterpret_cast<T*>(wz_smem);
    const Geo<T>& G = c.g;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int N = nx * ny * nz;
    const int tx = threadIdx.x, ty = threadIdx.y, t = tx + ty * 32;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8;
    const int i = i0 + tx, j = j0 + ty;
    const int kb = blockIdx.z * kchunk, ke = min(kb + kchunk, nz);
    const bool own = i < nx && j < ny;
    // staged cells of this thread: its own and (t < WZH) one halo cell (rows 0 and WZY - 1,
    // then columns 0 and WZX - 1 of rows 1 .. WZY - 2)
    int sidx[2], off[2], gjr[2];
    bool has[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        int li = tx + 1, lj = ty + 1;
        has[e] = e == 0 || t < WZH;
        if (e == 1 && has[1]) {
            if (t < 2 * WZX) {
                lj = t < WZX ? 0 : WZY - 1;
                li = t < WZX ? t : t - WZX;
            } else {
                const int h = t - 2 * WZX;
                lj = 1 + (h >> 1);
                li = (h & 1) ? WZX - 1 : 0;
            }
        }
        sidx[e] = lj * WZX + li;
        int gi = (i0 - 1 + li) % nx;   // a full modulo: the tile may be wider than the grid
        if (gi < 0) gi += nx;
        const int gj = j0 - 1 + lj;
        gjr[e] = gj;
        off[e] = (gj < 0 ? 0 : (gj >= ny ? ny - 1 : gj)) * nx + gi;
    }
    auto wrapz = [nz](int kk) { return kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk); };
    auto slot = [kb](int q) { return ((q - kb + 1) & 3) * 6 * WZP; };
    T v[2][6];
    auto load = [&](int q) {
        const int base = wrapz(q) * nx * ny;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (!has[e]) continue;
            const int a = base + off[e], gj = gjr[e];
            const bool in = gj >= 0 && gj < ny, top = gj >= ny - 1;
            const T sg = in ? (T)1 : (T)-1;   // odd ghost of u^x, u^z beyond a wall
            v[e][0] = sg * cvt_in<T>(u[a]);
            v[e][1] = (in && !top) ? cvt_in<T>(u[N + a]) : (T)0;
            v[e][2] = sg * cvt_in<T>(u[2 * N + a]);
            v[e][3] = in ? w[a] : (T)0;
            v[e][4] = (in && !top) ? w[N + a] : (T)0;
            v[e][5] = in ? w[2 * N + a] : (T)0;
        }
    };
    auto store = [&](int q) {
        T* const s = ring + slot(q);
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (has[e]) {
#pragma unroll
                for (int f = 0; f < 6; ++f) s[f * WZP + sidx[e]] = v[e][f];
            }
    };
    for (int q = kb - 1; q <= kb + 1 && q <= ke; ++q) {
        load(q);
        store(q);
    }
    __syncthreads();
    const double dt = c.dt_dev ? *c.dt_dev : c.dt_host;
    const T dtb = cvt_in<T>(dt * c.bn), dta = cvt_in<T>(dt * c.an);
    double nup = 0.0;
    SharedWallAcc<T> A;
    A.s = ring;
    A.c0 = (ty + 1) * WZX + tx + 1;
    const WallRowCoef<T> rc = wall_row_coef<T, 3>(G, own ? i : 0, own ? j : 0);
    for (int k = kb; k < ke; ++k) {
        const bool more = k + 2 <= ke;
        if (more) load(k + 2);
        if (own) {
            // the finish's own-cell values first, so their loads overlap the stencil arithmetic
            const int P = (k * ny + j) * nx + i;
            UB old[3], yv[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                old[a] = UIN ? uin[a * N + P] : ubar0[a * N + P];   // the accumulator's previous value
                yv[a] = ybar ? ybar[a * N + P] : old[a];
            }
            A.so[0] = slot(k - 1);
            A.so[1] = slot(k);
            A.so[2] = slot(k + 1);
            T q[3];
            wall_adj_cell<T, 3>(rc, ny, c.nu, j, A, q, nup);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if constexpr (std::is_same<T, UB>::value) {
                    ubar0[a * N + P] = old[a] + q[a];
                    if (kbar) kbar[a * N + P] = fma(dtb, yv[a], dta * q[a]);
                } else {
                    ubar0[a * N + P] = old[a] + df_to_double(q[a]);
                    if (kbar) kbar[a * N + P] = fma(dtb, cvt_in<T>(yv[a]), dta * q[a]);
                }
            }
        }
        if (more) store(k + 2);
        __syncthreads();
    }
    block_partial(nup, nu_part);
}

// The projection pullback P^T kbar = M Omega P Omega^-1 M kbar as two passes around the
// Poisson solve, the row scalings folded in. Rows of u^x, u^z carry the factor d_y[j], rows of
// u^y the factor h_y[j] (the x/z factors of Omega cancel); the stored top wall faces of u^y
// are 0. Block (32, 8), grid (ceil(nx/32), ceil(ny/8), nz).
// phi = D (Omega^-1 M kbar).
template <typename T, int DIM>
__global__ void k_wall_div_scaled(Geo<T> g, const T* __restrict__ kb, T* __restrict__ phi) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long N = (long)nx * ny * nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long a = ((long)k * ny + j) * nx + i;
    const int im = i == 0 ? nx - 1 : i - 1;
    const T idy = g.coef(1, C_INV_D, j);
    T d = (kb[a] * idy - kb[a - i + im] * idy) * g.coef(0, C_INV_D, i);
    const T wy = j == ny - 1 ? (T)0 : kb[N + a] * g.coef(1, C_INV_H, j);
    const T wym = j == 0 ? (T)0 : kb[N + a - nx] * g.coef(1, C_INV_H, j - 1);
    d += (wy - wym) * idy;
    if (DIM == 3) {
        const long az = k == 0 ? a + (long)(nz - 1) * nx * ny : a - (long)nx * ny;
        d += (kb[2 * N + a] * idy - kb[2 * N + az] * idy) * g.coef(2, C_INV_D, k);
    }
    phi[a] = d;
}

// w = M Omega (Omega^-1 M kbar - G p), hy / dy: the FP64 spacings h_y, d_y.
template <typename T, int DIM>
__global__ void k_wall_sub_scaled(Geo<T> g, const T* __restrict__ kb, const T* __restrict__ p, T* __restrict__ w,
                                  const double* __restrict__ hy, const double* __restrict__ dy) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long N = (long)nx * ny * nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long a = ((long)k * ny + j) * nx + i;
    const T idy = g.coef(1, C_INV_D, j), sd = cvt_in<T>(dy[j]);
    const T p0 = p[a];
    const T pe = p[a - i + (i + 1 == nx ? 0 : i + 1)];
    w[a] = (kb[a] * idy - (pe - p0) * g.coef(0, C_INV_H, i)) * sd;
    if (j == ny - 1) {
        w[N + a] = (T)0;
    } else {
        const T pn = p[a + nx];
        w[N + a] = (kb[N + a] * g.coef(1, C_INV_H, j) - (pn - p0) * g.coef(1, C_INV_H, j)) * cvt_in<T>(hy[j]);
    }
    if (DIM == 3) {
        const long plane = (long)nx * ny;
        const T pt = p[k + 1 == nz ? a - (long)(nz - 1) * plane : a + plane];
        w[2 * N + a] = (kb[2 * N + a] * idy - (pt - p0) * g.coef(2, C_INV_H, k)) * sd;
    }
}

// Zero the stored top wall faces of u^y.
template <typename T>
__global__ void k_mask_top(T* __restrict__ x, int nx, int ny, int nz, long N) {
    const long n = (long)nx * nz;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nx), k = (int)(t / nx);
        x[N + ((long)k * ny + (ny - 1)) * nx + i] = (T)0;
    }
}

}  // namespace ins
