// F(u) = C(u) + nu diffusion(u) + f on every velocity face and r = D F(u) in
// every cell (paper App. A discrete momentum equation, App. B kernels), one
// pass over u.
//
// Layout of the work: a CTA of 32 x 8 threads owns a 32 x 8 column of cells
// and marches up z through a chunk of planes. Three planes (k-1, k, k+1) of
// every velocity component, with a halo of 2 cells below and 1 above in x and
// y, sit in shared memory as a ring; plane k+2 is loaded into registers while
// plane k is computed and committed to the ring afterwards. Each thread
// computes F at its own three faces. The divergence also needs F^x one cell to
// the left of the tile and F^y one row below it: warp 1 (8 lanes) and warp 0
// compute those, so only two of the eight warps do one extra evaluation, and
// F^z one plane below is carried in a register from the previous plane.
//
// Coefficients: x and z are periodic and uniform, so their coefficients are
// kernel parameters; y is uniform too unless it is a wall direction, where the
// per-row coefficients of the stretched grid are read once per thread (they
// do not change along the z march). With uniform interpolation directions the
// interpolation weights 1/2 are folded into the coefficients:
//   self term   b == a: -((u_i + u_{i+1})^2 - (u_{i-1} + u_i)^2) * 0.25/h_a
//   cross term  b != a: -(V+ T+ - V- T-) * 0.5/d_b with V = w_l u^b + w_r u^b_{+a}
//               (volume weights along a) and T = sums of the transported u^a;
//               when a is uniform V+ = u^b + u^b_{+a} and the factor is 0.25/d_b.
// Boundary rules are applied while loading: periodic wrap, or at a no-slip
// wall in y the odd ghost for u^x, u^z and 0 for u^y (paper Sec. 2.4).
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace ins {

constexpr int RBX = 32;
constexpr int RBY = 8;
constexpr int RSX = RBX + 3;   // plane covers i0-2 .. i0+RBX
constexpr int RSY = RBY + 3;   //              j0-2 .. j0+RBY
constexpr int RSPL = RSX * RSY;
constexpr int RNT = RBX * RBY;
constexpr int RPF = (RSPL + RNT - 1) / RNT;   // plane elements per thread

// per-row y coefficients of a wall (stretched) direction, arrays over j
enum YCoef { CY_F = 0, CY_S, CY_WL, CY_WR, CY_AP, CY_AM, CY_BP, CY_BM, CY_I, CY_COUNT };
//  CY_F  0.25/d_y[j]          cross terms with flux direction y (uniform interpolation direction)
//  CY_S  0.25/h_y[j]          self term of u^y
//  CY_WL, CY_WR               volume weights d_j/(d_j+d_{j+1}), d_{j+1}/(d_j+d_{j+1})
//  CY_AP nu/(d_{j+1} h_j), CY_AM nu/(d_j h_j)        diffusion of u^y along y
//  CY_BP nu/(h_j d_j),     CY_BM nu/(h_{j-1} d_j)    diffusion of u^x, u^z along y
//  CY_I  1/d_y[j]                                    divergence

template <typename T>
struct RhsCoef {
    int nx, ny, nz;
    T cx, cy, cz;   // 0.25/D
    T dx, dy, dz;   // nu/D^2
    T ix, iy, iz;   // 1/D
    T fx, fy, fz;   // body force
    const T* yc;    // wall: CY_COUNT arrays of ny values
    const double* yc64;   // double-float arithmetic: the FP64 arrays, split by bits when a row is read
};

template <typename T>
struct YRow {
    T f, s, wl, wr, ap, am, bp, bm, i;
};

template <typename T, bool WALL>
__device__ __forceinline__ YRow<T> yrow(const RhsCoef<T>& c, int j) {
    YRow<T> r;
    if constexpr (WALL && std::is_same<T, df>::value) {
        // the FP64 row coefficients, split once per row (a thread's row stays fixed along its march)
        const double* y = c.yc64;
        const int n = c.ny;
        r.f = df_split(__ldg(y + CY_F * n + j));
        r.s = df_split(__ldg(y + CY_S * n + j));
        r.wl = df_split(__ldg(y + CY_WL * n + j));
        r.wr = df_split(__ldg(y + CY_WR * n + j));
        r.ap = df_split(__ldg(y + CY_AP * n + j));
        r.am = df_split(__ldg(y + CY_AM * n + j));
        r.bp = df_split(__ldg(y + CY_BP * n + j));
        r.bm = df_split(__ldg(y + CY_BM * n + j));
        r.i = df_split(__ldg(y + CY_I * n + j));
    } else if constexpr (WALL) {
        const T* y = c.yc;
        const int n = c.ny;
        r.f = __ldg(y + CY_F * n + j);
        r.s = __ldg(y + CY_S * n + j);
        r.wl = __ldg(y + CY_WL * n + j);
        r.wr = __ldg(y + CY_WR * n + j);
        r.ap = __ldg(y + CY_AP * n + j);
        r.am = __ldg(y + CY_AM * n + j);
        r.bp = __ldg(y + CY_BP * n + j);
        r.bm = __ldg(y + CY_BM * n + j);
        r.i = __ldg(y + CY_I * n + j);
    } else {
        r.f = c.cy;
        r.s = c.cy;
        r.wl = r.wr = (T)0.5;
        r.ap = r.am = r.bp = r.bm = c.dy;
        r.i = c.iy;
    }
    return r;
}

// Plane arrays in shared memory: P[comp][lj * RSX + li].
template <typename T>
using Plane = T (*)[RSPL];
template <typename T>
using CPlane = const T (*)[RSPL];

// Plane arguments: PL indexes [component][row * SX + column] (the ring planes of k_rhs_div by
// default; other kernels pass their own row stride and plane type).
template <typename T, int DIM, bool WALL, int SX = RSX, typename PL = CPlane<T>>
__device__ __forceinline__ T eval_Fx(const RhsCoef<T>& c, const YRow<T>& y, PL m, PL o, PL p, int c0) {
    const T uc = o[0][c0], ue = o[0][c0 + 1], uw = o[0][c0 - 1], un = o[0][c0 + SX], us = o[0][c0 - SX];
    const T s1 = uc + ue, s2 = uw + uc;
    const T X = fma(s1, s1, -s2 * s2);
    // u^y interpolated along x (uniform): weights folded into y.f
    const T vp = o[1][c0] + o[1][c0 + 1], vm = o[1][c0 - SX] + o[1][c0 + 1 - SX];
    const T Y = fma(vp, uc + un, -vm * (us + uc));
    T acc = fma(c.dx, ue + uw, c.fx);
    acc = fma(y.bp, un, acc);
    acc = fma(y.bm, us, acc);
    T dsum = (T)2 * c.dx + y.bp + y.bm;
    if constexpr (DIM == 3) {
        const T ut = p[0][c0], ub = m[0][c0];
        const T wp = o[2][c0] + o[2][c0 + 1], wm = m[2][c0] + m[2][c0 + 1];
        const T Z = fma(wp, uc + ut, -wm * (ub + uc));
        acc = fma(c.dz, ut + ub, acc);
        dsum += (T)2 * c.dz;
        acc = fma(-c.cz, Z, acc);
    }
    acc = fma(-dsum, uc, acc);
    acc = fma(-c.cx, X, acc);
    return fma(-y.f, Y, acc);
}

template <typename T, int DIM, bool WALL, int SX = RSX, typename PL = CPlane<T>>
__device__ __forceinline__ T eval_Fy(const RhsCoef<T>& c, const YRow<T>& y, PL m, PL o, PL p, int c0) {
    const T uc = o[1][c0], un = o[1][c0 + SX], us = o[1][c0 - SX], ue = o[1][c0 + 1], uw = o[1][c0 - 1];
    const T s1 = uc + un, s2 = us + uc;
    const T Ys = fma(s1, s1, -s2 * s2);
    T vp, vm, cxf;
    if constexpr (WALL) {   // u^x interpolated along the stretched y with volume weights
        vp = fma(y.wl, o[0][c0], y.wr * o[0][c0 + SX]);
        vm = fma(y.wl, o[0][c0 - 1], y.wr * o[0][c0 - 1 + SX]);
        cxf = (T)2 * c.cx;
    } else {
        vp = o[0][c0] + o[0][c0 + SX];
        vm = o[0][c0 - 1] + o[0][c0 - 1 + SX];
        cxf = c.cx;
    }
    const T X = fma(vp, uc + ue, -vm * (uw + uc));
    T acc = fma(c.dx, ue + uw, c.fy);
    acc = fma(y.ap, un, acc);
    acc = fma(y.am, us, acc);
    T dsum = (T)2 * c.dx + y.ap + y.am;
    if constexpr (DIM == 3) {
        const T ut = p[1][c0], ub = m[1][c0];
        T wp, wm, czf;
        if constexpr (WALL) {
            wp = fma(y.wl, o[2][c0], y.wr * o[2][c0 + SX]);
            wm = fma(y.wl, m[2][c0], y.wr * m[2][c0 + SX]);
            czf = (T)2 * c.cz;
        } else {
            wp = o[2][c0] + o[2][c0 + SX];
            wm = m[2][c0] + m[2][c0 + SX];
            czf = c.cz;
        }
        const T Z = fma(wp, uc + ut, -wm * (ub + uc));
        acc = fma(c.dz, ut + ub, acc);
        dsum += (T)2 * c.dz;
        acc = fma(-czf, Z, acc);
    }
    acc = fma(-dsum, uc, acc);
    acc = fma(-y.s, Ys, acc);
    return fma(-cxf, X, acc);
}

template <typename T, bool WALL, int SX = RSX, typename PL = CPlane<T>>
__device__ __forceinline__ T eval_Fz(const RhsCoef<T>& c, const YRow<T>& y, PL m, PL o, PL p, int c0) {
    const T uc = o[2][c0], ut = p[2][c0], ub = m[2][c0], ue = o[2][c0 + 1], uw = o[2][c0 - 1], un = o[2][c0 + SX],
            us = o[2][c0 - SX];
    const T s1 = uc + ut, s2 = ub + uc;
    const T Zs = fma(s1, s1, -s2 * s2);
    const T vp = o[0][c0] + p[0][c0], vm = o[0][c0 - 1] + p[0][c0 - 1];
    const T X = fma(vp, uc + ue, -vm * (uw + uc));
    const T wp = o[1][c0] + p[1][c0], wm = o[1][c0 - SX] + p[1][c0 - SX];
    const T Y = fma(wp, uc + un, -wm * (us + uc));
    T acc = fma(c.dx, ue + uw, c.fz);
    acc = fma(c.dz, ut + ub, acc);
    acc = fma(y.bp, un, acc);
    acc = fma(y.bm, us, acc);
    acc = fma(-((T)2 * (c.dx + c.dz) + y.bp + y.bm), uc, acc);
    acc = fma(-c.cz, Zs, acc);
    acc = fma(-c.cx, X, acc);
    return fma(-y.f, Y, acc);
}

// The 27 values the three F evaluations of one cell read in 3-D (planes m = k-1, o = k,
// p = k+1; suffixes e/w/n/s = +x/-x/+y/-y). Along the z march, the m values and five of the
// o values are the previous iteration's o and p values, kept in registers, so each plane
// costs 17 shared loads per cell instead of 27.
template <typename T>
struct Nb {
    T X0, X0e, X0w, X0n, X0s, X0wn;       // u^x, plane o
    T Y0, Y0e, Y0w, Y0n, Y0s, Y0es;       // u^y, plane o
    T Z0, Z0e, Z0w, Z0n, Z0s;             // u^z, plane o
    T Xp, Xpw, Yp, Yps, Zp;               // plane p
    T Xm, Ym, Zm, Zme, Zmn;               // plane m
    // z-face products shared by consecutive planes: the lower-face product of plane k is the
    // upper-face product of plane k-1 (same operands, so carrying it changes no bit)
    T cx, cy, cz;                         // F^x: w-interp * (u^x+u^x)_z, F^y: likewise, F^z: (u^z+u^z)^2
};

// carried products for the first plane of a march (from the m and o values)
template <typename T, bool WALL>
__device__ __forceinline__ void nb_carry_init(Nb<T>& v, const YRow<T>& y) {
    v.cx = (v.Zm + v.Zme) * (v.Xm + v.X0);
    const T wm = WALL ? fma(y.wl, v.Zm, y.wr * v.Zmn) : v.Zm + v.Zmn;
    v.cy = wm * (v.Ym + v.Y0);
    const T s2 = v.Zm + v.Z0;
    v.cz = s2 * s2;
}

// o-plane values not carried over from the previous iteration's p plane
template <typename T>
__device__ __forceinline__ void nb_load_o(Nb<T>& v, CPlane<T> o, int c0) {
    v.X0e = o[0][c0 + 1];
    v.X0n = o[0][c0 + RSX];
    v.X0s = o[0][c0 - RSX];
    v.X0wn = o[0][c0 - 1 + RSX];
    v.Y0e = o[1][c0 + 1];
    v.Y0w = o[1][c0 - 1];
    v.Y0n = o[1][c0 + RSX];
    v.Y0es = o[1][c0 + 1 - RSX];
    v.Z0e = o[2][c0 + 1];
    v.Z0w = o[2][c0 - 1];
    v.Z0n = o[2][c0 + RSX];
    v.Z0s = o[2][c0 - RSX];
}

template <typename T>
__device__ __forceinline__ void nb_load_p(Nb<T>& v, CPlane<T> p, int c0) {
    v.Xp = p[0][c0];
    v.Xpw = p[0][c0 - 1];
    v.Yp = p[1][c0];
    v.Yps = p[1][c0 - RSX];
    v.Zp = p[2][c0];
}

// end of an iteration: o -> m, p -> o (the carried part)
template <typename T>
__device__ __forceinline__ void nb_rotate(Nb<T>& v) {
    v.Xm = v.X0;
    v.Ym = v.Y0;
    v.Zm = v.Z0;
    v.Zme = v.Z0e;
    v.Zmn = v.Z0n;
    v.X0 = v.Xp;
    v.X0w = v.Xpw;
    v.Y0 = v.Yp;
    v.Y0s = v.Yps;
    v.Z0 = v.Zp;
}

// Same arithmetic as eval_Fx / eval_Fy / eval_Fz (DIM = 3) on register values.
template <typename T, bool WALL>
__device__ __forceinline__ T nb_Fx(const RhsCoef<T>& c, const YRow<T>& y, Nb<T>& v) {
    const T uc = v.X0, ue = v.X0e, uw = v.X0w, un = v.X0n, us = v.X0s;
    const T s1 = uc + ue, s2 = uw + uc;
    const T X = fma(s1, s1, -s2 * s2);
    const T vp = v.Y0 + v.Y0e, vm = v.Y0s + v.Y0es;
    const T Y = fma(vp, uc + un, -vm * (us + uc));
    T acc = fma(c.dx, ue + uw, c.fx);
    acc = fma(y.bp, un, acc);
    acc = fma(y.bm, us, acc);
    T dsum = (T)2 * c.dx + y.bp + y.bm;
    const T ut = v.Xp, ub = v.Xm;
    const T wp = v.Z0 + v.Z0e, sup = uc + ut;
    const T Z = fma(wp, sup, -v.cx);
    v.cx = wp * sup;
    acc = fma(c.dz, ut + ub, acc);
    dsum += (T)2 * c.dz;
    acc = fma(-c.cz, Z, acc);
    acc = fma(-dsum, uc, acc);
    acc = fma(-c.cx, X, acc);
    return fma(-y.f, Y, acc);
}

template <typename T, bool WALL>
__device__ __forceinline__ T nb_Fy(const RhsCoef<T>& c, const YRow<T>& y, Nb<T>& v) {
    const T uc = v.Y0, un = v.Y0n, us = v.Y0s, ue = v.Y0e, uw = v.Y0w;
    const T s1 = uc + un, s2 = us + uc;
    const T Ys = fma(s1, s1, -s2 * s2);
    T vp, vm, cxf, wp, czf;
    if constexpr (WALL) {
        vp = fma(y.wl, v.X0, y.wr * v.X0n);
        vm = fma(y.wl, v.X0w, y.wr * v.X0wn);
        cxf = (T)2 * c.cx;
        wp = fma(y.wl, v.Z0, y.wr * v.Z0n);
        czf = (T)2 * c.cz;
    } else {
        vp = v.X0 + v.X0n;
        vm = v.X0w + v.X0wn;
        cxf = c.cx;
        wp = v.Z0 + v.Z0n;
        czf = c.cz;
    }
    const T X = fma(vp, uc + ue, -vm * (uw + uc));
    T acc = fma(c.dx, ue + uw, c.fy);
    acc = fma(y.ap, un, acc);
    acc = fma(y.am, us, acc);
    T dsum = (T)2 * c.dx + y.ap + y.am;
    const T ut = v.Yp, ub = v.Ym;
    const T sup = uc + ut;
    const T Z = fma(wp, sup, -v.cy);
    v.cy = wp * sup;
    acc = fma(c.dz, ut + ub, acc);
    dsum += (T)2 * c.dz;
    acc = fma(-czf, Z, acc);
    acc = fma(-dsum, uc, acc);
    acc = fma(-y.s, Ys, acc);
    return fma(-cxf, X, acc);
}

template <typename T, bool WALL>
__device__ __forceinline__ T nb_Fz(const RhsCoef<T>& c, const YRow<T>& y, Nb<T>& v) {
    const T uc = v.Z0, ut = v.Zp, ub = v.Zm, ue = v.Z0e, uw = v.Z0w, un = v.Z0n, us = v.Z0s;
    const T s1 = uc + ut;
    const T Zs = fma(s1, s1, -v.cz);
    v.cz = s1 * s1;
    const T vp = v.X0 + v.Xp, vm = v.X0w + v.Xpw;
    const T X = fma(vp, uc + ue, -vm * (uw + uc));
    const T wp = v.Y0 + v.Yp, wm = v.Y0s + v.Yps;
    const T Y = fma(wp, uc + un, -wm * (us + uc));
    T acc = fma(c.dx, ue + uw, c.fz);
    acc = fma(c.dz, ut + ub, acc);
    acc = fma(y.bp, un, acc);
    acc = fma(y.bm, us, acc);
    acc = fma(-((T)2 * (c.dx + c.dz) + y.bp + y.bm), uc, acc);
    acc = fma(-c.cz, Zs, acc);
    acc = fma(-c.cx, X, acc);
    return fma(-y.f, Y, acc);
}

// Where each thread's share of a plane comes from (the same for every plane).
template <bool WALL>
struct PlaneMap {
    int off[RPF];       // in-plane offset (row * nx + column), -1 when the thread has no element
    bool ghost[RPF];    // wall ghost: negate u^x, u^z; u^y is 0
};

template <bool WALL>
__device__ __forceinline__ PlaneMap<WALL> plane_map(int nx, int ny, int i0, int j0) {
    PlaneMap<WALL> pm;
    const int tid = threadIdx.x + threadIdx.y * RBX;
#pragma unroll
    for (int q = 0; q < RPF; ++q) {
        const int idx = tid + q * RNT;
        pm.off[q] = -1;
        pm.ghost[q] = false;
        if (idx < RSPL) {
            const int li = idx % RSX, lj = idx / RSX;
            int gi = (i0 - 2 + li) % nx;
            if (gi < 0) gi += nx;
            int gj = j0 - 2 + lj;
            if (!WALL) {
                gj %= ny;
                if (gj < 0) gj += ny;
            } else if (gj < 0 || gj >= ny) {
                int mj = gj < 0 ? -gj - 1 : 2 * ny - 1 - gj;
                gj = mj < 0 ? 0 : (mj >= ny ? ny - 1 : mj);
                pm.ghost[q] = true;
            }
            pm.off[q] = gj * nx + gi;
        }
    }
    return pm;
}

// Offsets are 32-bit: grids hold fewer than 2^31 cells, so every in-component index fits.
// S: the storage type of u (FP64 fields read by the double-float kernel are split on load).
template <typename T, int DIM, bool WALL, typename S = T>
__device__ __forceinline__ void plane_fetch(const PlaneMap<WALL>& pm, const S* __restrict__ u0, const S* __restrict__ u1,
                                            const S* __restrict__ u2, int base, T (&v)[DIM][RPF]) {
#pragma unroll
    for (int q = 0; q < RPF; ++q) {
        if (pm.off[q] >= 0) {
            const int o = base + pm.off[q];
            T x0 = cvt_in<T>(u0[o]), x1 = cvt_in<T>(u1[o]);
            if (WALL && pm.ghost[q]) {
                x0 = -x0;
                x1 = (T)0;
            }
            v[0][q] = x0;
            v[1][q] = x1;
            if constexpr (DIM == 3) {
                T x2 = cvt_in<T>(u2[o]);
                if (WALL && pm.ghost[q]) x2 = -x2;
                v[2][q] = x2;
            }
        }
    }
}

template <typename T, int DIM, bool WALL>
__device__ __forceinline__ void plane_commit(const PlaneMap<WALL>& pm, Plane<T> s, const T (&v)[DIM][RPF]) {
    const int tid = threadIdx.x + threadIdx.y * RBX;
#pragma unroll
    for (int q = 0; q < RPF; ++q)
        if (pm.off[q] >= 0) {
#pragma unroll
            for (int cc = 0; cc < DIM; ++cc) s[cc][tid + q * RNT] = v[cc][q];
        }
}

// F (dim fields, may be null) and r = D F. Grid: (ceil(nx/32), ceil(ny/8), ceil(nz/kchunk)), block (32, 8).
// m (dim fields, may be null): a closure term added to F on every face, including the halo
// faces the divergence reads.
// UI: storage type of u (T, or double for the double-float kernel reading an FP64 field).
template <typename T, int DIM, bool WALL, typename UI = T>
__global__ void __launch_bounds__(RNT) k_rhs_div(RhsCoef<T> c, const UI* __restrict__ u, T* __restrict__ F,
                                                 T* __restrict__ r, int kchunk, const T* __restrict__ mc) {
    __shared__ T su[3][DIM][RSPL];
    __shared__ T sFx[RBY][RBX + 1];
    __shared__ T sFy[RBY + 1][RBX];
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    const long N = (long)nx * ny * nz;
    const long plane = (long)nx * ny;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * RBX, j0 = blockIdx.y * RBY;
    const int i = i0 + tx, j = j0 + ty;
    const bool inside = i < nx && j < ny;
    const int c0 = (ty + 2) * RSX + (tx + 2);
    const YRow<T> yr = yrow<T, WALL>(c, j < ny ? j : ny - 1);
    // halo work: warp 0 computes F^y one row below the tile, warp 1 (lanes 0..7) F^x left of it
    const bool hy = ty == 0;
    const bool hx = ty == 1 && tx < RBY;
    const bool hy_wall = WALL && j0 == 0;   // the row below is the bottom wall: F^y = 0
    const int jhy = j0 - 1 < 0 ? ny - 1 : j0 - 1;
    const int jhx = j0 + tx < ny ? j0 + tx : ny - 1;
    const int c0hy = 1 * RSX + (tx + 2);
    const int c0hx = (tx + 2) * RSX + 1;
    const PlaneMap<WALL> pm = plane_map<WALL>(nx, ny, i0, j0);
    T v[DIM][RPF];

    if constexpr (DIM == 2) {
        plane_fetch<T, DIM, WALL, UI>(pm, u, u + N, u, 0, v);   // 2-D: no third component
        plane_commit<T, DIM, WALL>(pm, su[0], v);
        __syncthreads();
        CPlane<T> o = su[0];
        const int ic = i < nx ? i : nx - 1;
        const long am = (long)(j < ny ? j : ny - 1) * nx + ic;
        T fx = eval_Fx<T, 2, WALL>(c, yr, o, o, o, c0);
        T fy = eval_Fy<T, 2, WALL>(c, yr, o, o, o, c0);
        if (mc) {
            fx += mc[am];
            fy += mc[N + am];
        }
        if (WALL && j == ny - 1) fy = (T)0;
        sFx[ty][tx + 1] = fx;
        sFy[ty + 1][tx] = fy;
        if (hy) {
            T h = hy_wall ? (T)0 : eval_Fy<T, 2, WALL>(c, yrow<T, WALL>(c, jhy), o, o, o, c0hy);
            if (mc && !hy_wall) h += mc[N + (long)jhy * nx + ic];
            sFy[0][tx] = h;
        }
        if (hx) {
            T h = eval_Fx<T, 2, WALL>(c, yrow<T, WALL>(c, jhx), o, o, o, c0hx);
            if (mc) h += mc[(long)jhx * nx + (i0 - 1 < 0 ? nx - 1 : i0 - 1)];
            sFx[tx][0] = h;
        }
        __syncthreads();
        if (inside) {
            const long a = (long)j * nx + i;
            if (F) {
                F[a] = fx;
                F[N + a] = fy;
            }
            r[a] = (fx - sFx[ty][tx]) * c.ix + (fy - sFy[ty][tx]) * yr.i;
        }
        return;
    } else {
        const int kb = blockIdx.z * kchunk;
        const int ke = min(kb + kchunk, nz);
        const int iplane = nx * ny;
        T* const F1 = F ? F + N : nullptr;
        T* const F2 = F ? F + 2 * N : nullptr;
        auto wrapz = [nz](int k) { return k < 0 ? k + nz : (k >= nz ? k - nz : k); };
        int sm = 0, so = 1, sp = 2;
        plane_fetch<T, DIM, WALL, UI>(pm, u, u + N, u + 2 * N, wrapz(kb - 2) * iplane, v);
        plane_commit<T, DIM, WALL>(pm, su[sm], v);
        plane_fetch<T, DIM, WALL, UI>(pm, u, u + N, u + 2 * N, wrapz(kb - 1) * iplane, v);
        plane_commit<T, DIM, WALL>(pm, su[so], v);
        plane_fetch<T, DIM, WALL, UI>(pm, u, u + N, u + 2 * N, wrapz(kb) * iplane, v);
        plane_commit<T, DIM, WALL>(pm, su[sp], v);
        plane_fetch<T, DIM, WALL, UI>(pm, u, u + N, u + 2 * N, wrapz(kb + 1) * iplane, v);
        __syncthreads();
        const int ic = i < nx ? i : nx - 1;
        const int jc = j < ny ? j : ny - 1;
        const int ihm = i0 - 1 < 0 ? nx - 1 : i0 - 1;
        T fz_prev = eval_Fz<T, WALL>(c, yr, su[sm], su[so], su[sp], c0);
        if (mc) fz_prev += mc[2 * N + (long)wrapz(kb - 1) * plane + (long)jc * nx + ic];
        __syncthreads();
        plane_commit<T, DIM, WALL>(pm, su[sm], v);
        {
            const int t = sm;
            sm = so;
            so = sp;
            sp = t;
        }
        __syncthreads();
        // register neighbourhood: m plane and the carried o values of the first iteration
        Nb<T> nb;
        {
            CPlane<T> m = su[sm];
            CPlane<T> o = su[so];
            nb.Xm = m[0][c0];
            nb.Ym = m[1][c0];
            nb.Zm = m[2][c0];
            nb.Zme = m[2][c0 + 1];
            nb.Zmn = m[2][c0 + RSX];
            nb.X0 = o[0][c0];
            nb.X0w = o[0][c0 - 1];
            nb.Y0 = o[1][c0];
            nb.Y0s = o[1][c0 - RSX];
            nb.Z0 = o[2][c0];
        }
        nb_carry_init<T, WALL>(nb, yr);
        for (int k = kb; k < ke; ++k) {
            const bool more = k + 1 < ke;
            if (more) plane_fetch<T, DIM, WALL, UI>(pm, u, u + N, u + 2 * N, wrapz(k + 2) * iplane, v);
            CPlane<T> m = su[sm];
            CPlane<T> o = su[so];
            CPlane<T> p = su[sp];
            nb_load_o<T>(nb, o, c0);
            nb_load_p<T>(nb, p, c0);
            T fx = nb_Fx<T, WALL>(c, yr, nb);
            T fy = nb_Fy<T, WALL>(c, yr, nb);
            T fz = nb_Fz<T, WALL>(c, yr, nb);
            if (mc) {
                const long am = (long)k * plane + (long)jc * nx + ic;
                fx += mc[am];
                fy += mc[N + am];
                fz += mc[2 * N + am];
            }
            if (WALL && j == ny - 1) fy = (T)0;
            sFx[ty][tx + 1] = fx;
            sFy[ty + 1][tx] = fy;
            if (hy) {
                T h = hy_wall ? (T)0 : eval_Fy<T, 3, WALL>(c, yrow<T, WALL>(c, jhy), m, o, p, c0hy);
                if (mc && !hy_wall) h += mc[N + (long)k * plane + (long)jhy * nx + ic];
                sFy[0][tx] = h;
            }
            if (hx) {
                T h = eval_Fx<T, 3, WALL>(c, yrow<T, WALL>(c, jhx), m, o, p, c0hx);
                if (mc) h += mc[(long)k * plane + (long)jhx * nx + ihm];
                sFx[tx][0] = h;
            }
            __syncthreads();
            if (inside) {
                const int a = k * iplane + j * nx + i;
                if (F) {
                    F[a] = fx;
                    F1[a] = fy;
                    F2[a] = fz;
                }
                r[a] = (fx - sFx[ty][tx]) * c.ix + (fy - sFy[ty][tx]) * yr.i + (fz - fz_prev) * c.iz;
            }
            fz_prev = fz;
            nb_rotate<T>(nb);
            if (more) plane_commit<T, DIM, WALL>(pm, su[sm], v);
            {
                const int t = sm;
                sm = so;
                so = sp;
                sp = t;
            }
            __syncthreads();
        }
    }
}

}  // namespace ins

namespace ins {

// ---------------------------------------------------------------------------------------
// Fused RK stage boundary (3-D): the update of stage s and the F / D F evaluation of stage
// s + 1 in one z march, so the stage state u_{s+1} never goes to memory.
//
// Each plane of the halo'd tile is staged from the previous stage's F_s, p_s and u_0:
//   k^a = F_s^a - (p_{I+e_a} - p_I) / h_a   (k^y = 0 on the stored top wall face),
//   u_{s+1}^a = u_0^a + dt a_{s+1,s} k^a,
// with the wall ghosts of u_{s+1} taken from the mirrored cell as in k_rhs_div. Thread t
// stages its own cell and, for t < 129, one halo cell; at its own cell (planes of its
// chunk only) it also updates the RK accumulator, acc = b_s k (s = 0) or acc += b_s k.
// The evaluation of F_{s+1} and r = D F_{s+1} on the staged ring is that of k_rhs_div.
// Reads F_s, p_s, u_0, acc and writes acc, F_{s+1}, r: 17 values per cell instead of the
// 23 of a separate update (16) and evaluation (7).
// The halo cells are staged by the upper four warps, so that the halo evaluations of warps 0
// and 1 do not fall on the same warps as a second staged cell; the three corner cells of
// column 0 that no stencil reads ((0, 0), (0, 1) and (0, RSY - 1) of the plane) are left out,
// which leaves 126 halo cells.
constexpr int FH = 126;          // halo cells of a plane that are staged

struct FusedMap {
    int off[2];       // in-plane offset of the source cell (mirror cell for a wall ghost)
    int sidx[2];      // position in the shared plane
    int dxp[2];       // offset of the +x neighbour (periodic wrap)
    int dyp[2];       // offset of the +y neighbour (periodic wrap; unused on the top wall row)
    int gj[2];        // row of the source cell
    bool ghost[2];    // wall ghost: u^x, u^z negated, u^y = 0
    bool has[2];      // element 1 exists only for t < FH
};

template <bool WALL>
__device__ __forceinline__ FusedMap fused_map(int nx, int ny, int i0, int j0) {
    FusedMap fm;
    const int t = threadIdx.x + threadIdx.y * RBX;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        int li, lj;
        const int h = t - RNT / 2;        // halo index of thread t >= 128
        if (e == 0) {
            li = threadIdx.x + 2;
            lj = threadIdx.y + 2;
        } else if (h >= 0 && h < 102) {   // rows 0, 1 and RSY - 1, columns 1 .. RSX - 1
            const int r = h / (RSX - 1);
            lj = r == 2 ? RSY - 1 : r;
            li = 1 + h - r * (RSX - 1);
        } else {                          // columns 0, 1 and RSX - 1 of rows 2 .. RSY - 2
            const int hh = h < 0 ? 0 : h - 102;
            lj = 2 + hh / 3;
            const int cc = hh % 3;
            li = cc == 2 ? RSX - 1 : cc;
        }
        fm.has[e] = e == 0 || (h >= 0 && h < FH);
        fm.sidx[e] = lj * RSX + li;
        int gi = (i0 - 2 + li) % nx;
        if (gi < 0) gi += nx;
        int gj = j0 - 2 + lj;
        fm.ghost[e] = false;
        if (!WALL) {
            gj %= ny;
            if (gj < 0) gj += ny;
        } else if (gj < 0 || gj >= ny) {
            const int mj = gj < 0 ? -gj - 1 : 2 * ny - 1 - gj;
            gj = mj < 0 ? 0 : (mj >= ny ? ny - 1 : mj);
            fm.ghost[e] = true;
        }
        fm.gj[e] = gj;
        fm.off[e] = gj * nx + gi;
        fm.dxp[e] = gi + 1 == nx ? -(nx - 1) : 1;
        fm.dyp[e] = gj + 1 == ny ? -(ny - 1) * nx : nx;
    }
    return fm;
}

struct FusedArgs {
    const double* dt_dev;
    double dt_host;
    double a_next;   // a_{s+1,s}
    double b;        // b_s
    int stage;       // s (0, 1 or 2)
    float* ust = nullptr;   // pair kernel, STS: the staged u_{s+1} of the own cells
};

template <typename T, bool WALL>
__global__ void __launch_bounds__(RNT, WALL ? 2 : 3) k_update_rhs_div(RhsCoef<T> c, T ihx, T ihz, const T* __restrict__ ihy,
                                                        const T* __restrict__ Fs, const T* __restrict__ p,
                                                        const T* __restrict__ u0, T* __restrict__ acc,
                                                        T* __restrict__ F, T* __restrict__ r, FusedArgs fa, int kchunk) {
    __shared__ T su[3][3][RSPL];
    __shared__ T sFx[RBY][RBX + 1];
    __shared__ T sFy[RBY + 1][RBX];
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    const size_t N = (size_t)nx * ny * nz;   // component stride (in-component offsets are 32-bit)
    const int iplane = nx * ny;
    const T* const Fs1 = Fs + N;
    const T* const Fs2 = Fs + 2 * N;
    const T* const u01 = u0 + N;
    const T* const u02 = u0 + 2 * N;
    T* const acc1 = acc + N;
    T* const acc2 = acc + 2 * N;
    T* const F1 = F + N;
    T* const F2 = F + 2 * N;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * RBX, j0 = blockIdx.y * RBY;
    const int i = i0 + tx, j = j0 + ty;
    const bool inside = i < nx && j < ny;
    const int c0 = (ty + 2) * RSX + (tx + 2);
    const YRow<T> yr = yrow<T, WALL>(c, j < ny ? j : ny - 1);
    const bool hy = ty == 0;
    const bool hx = ty == 1 && tx < RBY;
    const bool hy_wall = WALL && j0 == 0;
    const int jhy = j0 - 1 < 0 ? ny - 1 : j0 - 1;
    const int jhx = j0 + tx < ny ? j0 + tx : ny - 1;
    const int c0hy = 1 * RSX + (tx + 2);
    const int c0hx = (tx + 2) * RSX + 1;
    const FusedMap fm = fused_map<WALL>(nx, ny, i0, j0);
    const double dt = fa.dt_dev ? *fa.dt_dev : fa.dt_host;
    const T dta = (T)(dt * fa.a_next), bb = (T)fa.b;
    T ihy_e[2];
    bool top_e[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        ihy_e[e] = __ldg(&ihy[fm.gj[e]]);
        top_e[e] = WALL && fm.gj[e] == ny - 1;
    }
    const int kb = blockIdx.z * kchunk;
    const int ke = min(kb + kchunk, nz);
    auto wrapz = [nz](int k) { return k < 0 ? k + nz : (k >= nz ? k - nz : k); };
    T pself[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) pself[e] = fm.has[e] ? p[wrapz(kb - 2) * iplane + fm.off[e]] : (T)0;
    T v[3][2];
    // staging of plane q in two halves, so the global loads of plane k + 2 are in flight
    // while plane k is evaluated: stage_load issues them, stage_finish forms u_{s+1} in v
    // (and the accumulator at the own cell)
    T lF[3][2], lU[3][2], lpx[2], lpy[2], lpz[2], lA[3];
    int la[2];
    bool lown = false;
    auto stage_load = [&](int q) {
        const int base = wrapz(q) * iplane;
        const int basez = wrapz(q + 1) * iplane;
        lown = q >= kb && q < ke && inside;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (!fm.has[e]) continue;
            const int a = base + fm.off[e];
            la[e] = a;
            lF[0][e] = Fs[a];
            lF[1][e] = Fs1[a];
            lF[2][e] = Fs2[a];
            lU[0][e] = u0[a];
            lU[1][e] = u01[a];
            lU[2][e] = u02[a];
            lpx[e] = p[a + fm.dxp[e]];
            lpy[e] = p[a + fm.dyp[e]];
            lpz[e] = p[basez + fm.off[e]];
        }
        if (lown && fa.stage > 0) {
            lA[0] = acc[la[0]];
            lA[1] = acc1[la[0]];
            lA[2] = acc2[la[0]];
        }
    };
    auto stage_finish = [&]() {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (!fm.has[e]) continue;
            const T p0 = pself[e];
            pself[e] = lpz[e];
            const T kx = fma(p0 - lpx[e], ihx, lF[0][e]);
            const T ky = top_e[e] ? (T)0 : fma(p0 - lpy[e], ihy_e[e], lF[1][e]);
            const T kz = fma(p0 - lpz[e], ihz, lF[2][e]);
            T ux = fma(dta, kx, lU[0][e]);
            T uy = fma(dta, ky, lU[1][e]);
            T uz = fma(dta, kz, lU[2][e]);
            if (e == 0 && lown) {
                const int a = la[0];
                if (fa.stage == 0) {
                    acc[a] = bb * kx;
                    acc1[a] = bb * ky;
                    acc2[a] = bb * kz;
                } else {
                    acc[a] = fma(bb, kx, lA[0]);
                    acc1[a] = fma(bb, ky, lA[1]);
                    acc2[a] = fma(bb, kz, lA[2]);
                }
            }
            if (WALL && fm.ghost[e]) {
                ux = -ux;
                uy = (T)0;
                uz = -uz;
            }
            v[0][e] = ux;
            v[1][e] = uy;
            v[2][e] = uz;
        }
    };
    auto stage = [&](int q) {
        stage_load(q);
        stage_finish();
    };
    auto commit = [&](Plane<T> s) {
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (fm.has[e]) {
                s[0][fm.sidx[e]] = v[0][e];
                s[1][fm.sidx[e]] = v[1][e];
                s[2][fm.sidx[e]] = v[2][e];
            }
    };
    int sm = 0, so = 1, sp = 2;
    stage(kb - 2);
    commit(su[sm]);
    stage(kb - 1);
    commit(su[so]);
    stage(kb);
    commit(su[sp]);
    stage(kb + 1);
    __syncthreads();
    T fz_prev = eval_Fz<T, WALL>(c, yr, su[sm], su[so], su[sp], c0);
    __syncthreads();
    commit(su[sm]);
    {
        const int t = sm;
        sm = so;
        so = sp;
        sp = t;
    }
    __syncthreads();
    Nb<T> nb;
    {
        CPlane<T> m = su[sm];
        CPlane<T> o = su[so];
        nb.Xm = m[0][c0];
        nb.Ym = m[1][c0];
        nb.Zm = m[2][c0];
        nb.Zme = m[2][c0 + 1];
        nb.Zmn = m[2][c0 + RSX];
        nb.X0 = o[0][c0];
        nb.X0w = o[0][c0 - 1];
        nb.Y0 = o[1][c0];
        nb.Y0s = o[1][c0 - RSX];
        nb.Z0 = o[2][c0];
    }
    nb_carry_init<T, WALL>(nb, yr);
    for (int k = kb; k < ke; ++k) {
        const bool more = k + 1 < ke;
        if (more) stage_load(k + 2);
        CPlane<T> m = su[sm];
        CPlane<T> o = su[so];
        CPlane<T> pp = su[sp];
        nb_load_o<T>(nb, o, c0);
        nb_load_p<T>(nb, pp, c0);
        const T fx = nb_Fx<T, WALL>(c, yr, nb);
        T fy = nb_Fy<T, WALL>(c, yr, nb);
        const T fz = nb_Fz<T, WALL>(c, yr, nb);
        if (WALL && j == ny - 1) fy = (T)0;
        sFx[ty][tx + 1] = fx;
        sFy[ty + 1][tx] = fy;
        if (hy) sFy[0][tx] = hy_wall ? (T)0 : eval_Fy<T, 3, WALL>(c, yrow<T, WALL>(c, jhy), m, o, pp, c0hy);
        if (hx) sFx[tx][0] = eval_Fx<T, 3, WALL>(c, yrow<T, WALL>(c, jhx), m, o, pp, c0hx);
        __syncthreads();
        if (inside) {
            const int a = k * iplane + j * nx + i;
            F[a] = fx;
            F1[a] = fy;
            F2[a] = fz;
            r[a] = (fx - sFx[ty][tx]) * c.ix + (fy - sFy[ty][tx]) * yr.i + (fz - fz_prev) * c.iz;
        }
        fz_prev = fz;
        nb_rotate<T>(nb);
        if (more) {
            stage_finish();
            commit(su[sm]);
        }
        {
            const int t = sm;
            sm = so;
            so = sp;
            sp = t;
        }
        __syncthreads();
    }
}

}  // namespace ins
