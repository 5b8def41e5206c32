// Projection + RK stage update with 16-byte vector accesses and a z march
// (paper Sec. 2.6.2; pressure gradient of App. B).
//
// k = F - G p, (G p)^a = (p_{I+e_a} - p_I) / h_a, then for the classic RK4 scheme
//   stage 0: acc = b0 k;    us = u0 + dt a1 k
//   stage 1,2: acc += b k;  us = u0 + dt a k
//   stage 3: u0 = u0 + dt (acc + b3 k) in place, the CFL per-index maxima of
//            |u_{n+1}| and the non-finite flag;
//   stage -1 (projection only): us = F - G p (u0 and acc are not touched);
// and for the low-storage Wray scheme (LS; two registers u and k_{s-1}, Sec. 3.3)
//   u0 = u0 + dt (gamma_s k + zeta_s acc) in place (into us instead when us is not null),
//   acc = k (not on the last stage), the maxima and the flag on the last stage.
// Each thread owns VEC consecutive cells in x (one float4 / double2) of one row
// j and marches through a chunk of z planes: the pressure of plane k+1 loaded
// for G p in z is the centre pressure of the next plane, and the x neighbour of
// the last cell of a vector comes from the next lane by a warp shuffle.
// x and z are periodic and uniform (constant 1/h); y may be a stretched wall
// direction (1/h_y[j] is constant along the march).
#pragma once

#include "common.cuh"
#include "stencil.cuh"

namespace ins {

template <typename T>
struct VecT;
template <>
struct VecT<float> {
    using V = float4;
    static constexpr int N = 4;
    static __device__ __forceinline__ void ld(const float* p, float (&x)[4]) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
    static __device__ __forceinline__ void st(float* p, const float (&x)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
};
template <>
struct VecT<double> {
    using V = double2;
    static constexpr int N = 2;
    static __device__ __forceinline__ void ld(const double* p, double (&x)[2]) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        x[0] = v.x; x[1] = v.y;
    }
    static __device__ __forceinline__ void st(double* p, const double (&x)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
    }
};

// The same accesses with half the width (float2 / one double): rows whose 16-byte vector count
// would leave a warp partly idle (nx = 192 in FP32: 48 float4 per row, 96 float2) run with these.
template <typename T, int N>
struct VecIO : VecT<T> {};
template <>
struct VecIO<float, 2> {
    static constexpr int N = 2;
    static __device__ __forceinline__ void ld(const float* p, float (&x)[2]) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        x[0] = v.x; x[1] = v.y;
    }
    static __device__ __forceinline__ void st(float* p, const float (&x)[2]) {
        *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
    }
};
template <>
struct VecIO<double, 1> {
    static constexpr int N = 1;
    static __device__ __forceinline__ void ld(const double* p, double (&x)[1]) { x[0] = *p; }
    static __device__ __forceinline__ void st(double* p, const double (&x)[1]) { *p = x[0]; }
};

template <typename T>
struct RkCoef {
    int nx, ny, nz;
    T ihx, ihz;          // 1/h of the uniform x and z directions
    const T* ihy;        // 1/h_y[j]
    // SC (row-scaled projection of the wall-bounded step VJP): 1/d_y[j], and the FP64 d_y, h_y
    const T* idy = nullptr;
    const double* dy = nullptr;
    const double* hy = nullptr;
};

// Block (32, 8); grid (ceil(nx/VEC/32), ceil(ny/8), ceil(nz/kchunk)). Needs nx % VEC == 0 and
// 16-byte aligned field pointers.
// SC (with stage -1 only): the wall-bounded pullback's M Omega (Omega^-1 M F - G p): F^x, F^z
// scaled by 1/d_y[j] and F^y by 1/h_y[j] before the gradient, the result by d_y[j] (x, z) and
// h_y[j] (y) after it; the stored top wall faces of u^y are 0.
// SCL (with stage -1 only): F is read as (dt b) F (the step VJP's first cotangent dt b_last ybar,
// formed here instead of in a separate pass).
template <typename T, int DIM, bool WALL, bool LS = false, int VW = VecT<T>::N, bool SC = false, bool SCL = false>
__global__ void __launch_bounds__(256) k_rk_update_vec(RkCoef<T> c, const T* __restrict__ F, const T* __restrict__ p,
                                                       T* __restrict__ u0, T* __restrict__ acc, T* __restrict__ us,
                                                       RkArgs ra, int kchunk) {
    using VT = VecIO<T, VW>;
    constexpr int VEC = VW;
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    const long N = (long)nx * ny * nz;
    const long plane = (long)nx * ny;
    const int nvx = nx / VEC;
    const int lane = threadIdx.x, row = threadIdx.y;
    const int iv = blockIdx.x * 32 + lane;
    const int i0 = iv * VEC;
    const int j = blockIdx.y * 8 + row;
    const bool ok = iv < nvx && j < ny;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(kb + kchunk, nz);
    const double dt = ra.dt_dev ? *ra.dt_dev : ra.dt_host;
    const T dta = (T)(dt * ra.a_next), bb = (T)ra.b, dtt = (T)dt;
    const T dtz = (T)(dt * ra.b);
    const bool fin = LS ? ra.last != 0 : ra.stage == 3;
    const T ihy = __ldg(&c.ihy[j < ny ? j : ny - 1]);
    const bool top = WALL && j == ny - 1;
    const bool last_vec = iv == nvx - 1;
    const bool need_global_next = last_vec || lane == 31;
    const long jrow = (long)(j < ny ? j : 0) * nx;
    const long jnext = (long)(j + 1 < ny ? j + 1 : 0) * nx;   // periodic wrap in y
    // maxima of |u| in the field's own type (exact; one conversion to FP64 per reduction, so
    // the FP32 path does not load the FP64 pipe)
    T mxx[VEC], mxy = (T)0;
#pragma unroll
    for (int e = 0; e < VEC; ++e) mxx[e] = (T)0;
    bool bad = false;
    T P0[VEC], Pt[VEC];
    if (ok) VT::ld(p + (long)kb * plane + jrow + i0, P0);
    else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) P0[e] = (T)0;
    }
    for (int k = kb; k < ke; ++k) {
        const long base = (long)k * plane;
        const long a = base + jrow + i0;
        const long kt = (k + 1 < nz ? (long)(k + 1) : 0) * plane;
        // x neighbour of the last element: first element of the next vector (next lane or wrap)
        T pnext = __shfl_down_sync(0xffffffffu, P0[0], 1);
        T Pn[VEC];
        T qz = (T)0;
        if (ok) {
            if (need_global_next) pnext = p[base + jrow + (last_vec ? 0 : i0 + VEC)];
            if (DIM == 3) VT::ld(p + kt + jrow + i0, Pt);
            if (!top) VT::ld(p + base + jnext + i0, Pn);
            T f[3][VEC], kk[3][VEC];
            VT::ld(F + a, f[0]);
            VT::ld(F + N + a, f[1]);
            if (DIM == 3) VT::ld(F + 2 * N + a, f[2]);
            if constexpr (SCL) {
                const T al = (T)(dt * ra.b);
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    f[0][e] *= al;
                    f[1][e] *= al;
                    if (DIM == 3) f[2][e] *= al;
                }
            }
            if constexpr (SC) {
                const T sd = __ldg(&c.idy[j]);
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    f[0][e] *= sd;
                    f[1][e] *= ihy;
                    if (DIM == 3) f[2][e] *= sd;
                }
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const T pe = e + 1 < VEC ? P0[e + 1] : pnext;
                kk[0][e] = fma(P0[e] - pe, c.ihx, f[0][e]);
                kk[1][e] = top ? (T)0 : fma(P0[e] - Pn[e], ihy, f[1][e]);
                if (DIM == 3) kk[2][e] = fma(P0[e] - Pt[e], c.ihz, f[2][e]);
            }
#pragma unroll
            for (int cc = 0; cc < DIM; ++cc) {
                const long ea = cc * N + a;
                if (!LS && ra.stage < 0) {   // projection only: us = F - G p
                    if constexpr (SC) {
                        const T post = (T)(cc == 1 ? c.hy[j] : c.dy[j]);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) kk[cc][e] *= post;
                    }
                    VT::st(us + ea, kk[cc]);
                    continue;
                }
                T uv[VEC], av[VEC];
                VT::ld(u0 + ea, uv);
                if (LS) {
                    if (ra.stage > 0) {
                        VT::ld(acc + ea, av);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) uv[e] += fma(dtz, av[e], dta * kk[cc][e]);
                    } else {
#pragma unroll
                        for (int e = 0; e < VEC; ++e) uv[e] += dta * kk[cc][e];
                    }
                    if (!ra.last) VT::st(acc + ea, kk[cc]);
                    if (ra.last) {
#pragma unroll
                        for (int e = 0; e < VEC; ++e) {
                            bad |= !isfinite(uv[e]);
                            const T q = fabs(uv[e]);
                            if (cc == 0) mxx[e] = fmax(mxx[e], q);
                            else if (cc == 1) mxy = fmax(mxy, q);
                            else qz = fmax(qz, q);
                        }
                    }
                    VT::st((us ? us : u0) + ea, uv);
                } else if (ra.stage == 0) {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        av[e] = bb * kk[cc][e];
                        uv[e] = fma(dta, kk[cc][e], uv[e]);
                    }
                    if (acc) VT::st(acc + ea, av);   // null: stage state only (the step VJP's recompute)
                    VT::st(us + ea, uv);
                } else if (ra.stage < 3) {
                    VT::ld(acc + ea, av);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        av[e] = fma(bb, kk[cc][e], av[e]);
                        uv[e] = fma(dta, kk[cc][e], uv[e]);
                    }
                    VT::st(acc + ea, av);
                    VT::st(us + ea, uv);
                } else {
                    VT::ld(acc + ea, av);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        uv[e] = fma(dtt, fma(bb, kk[cc][e], av[e]), uv[e]);
                        bad |= !isfinite(uv[e]);
                        const T q = fabs(uv[e]);
                        if (cc == 0) mxx[e] = fmax(mxx[e], q);
                        else if (cc == 1) mxy = fmax(mxy, q);
                        else qz = fmax(qz, q);
                    }
                    VT::st(u0 + ea, uv);
                }
            }
        } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) Pt[e] = (T)0;
        }
        if (fin && ra.mx && DIM == 3) {
            for (int o = 16; o > 0; o >>= 1) qz = fmax(qz, __shfl_xor_sync(0xffffffffu, qz, o));
            if (lane == 0 && qz > (T)0) atomicMax(&ra.mx[nx + ny + k], (unsigned long long)__double_as_longlong((double)qz));
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) P0[e] = Pt[e];
    }
    if (fin) {
        if (ra.mx) {
            __shared__ T sx[8][32 * VEC + 1];
#pragma unroll
            for (int e = 0; e < VEC; ++e) sx[row][lane * VEC + e] = mxx[e];
            for (int o = 16; o > 0; o >>= 1) mxy = fmax(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
            if (lane == 0 && j < ny && mxy > (T)0)
                atomicMax(&ra.mx[nx + j], (unsigned long long)__double_as_longlong((double)mxy));
            __syncthreads();
            if (row == 0 && iv < nvx) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    T m = sx[0][lane * VEC + e];
                    for (int r = 1; r < 8; ++r) m = fmax(m, sx[r][lane * VEC + e]);
                    if (m > (T)0) atomicMax(&ra.mx[i0 + e], (unsigned long long)__double_as_longlong((double)m));
                }
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(ra.err_flag, 1u);
    }
}

// phi = D u (App. B divergence kernel) with the same thread layout and z march: VEC cells in x
// per thread, the x neighbour u^x_{i-1} of the first cell from the previous lane (or global
// memory at a warp or row start), u^z of plane k - 1 carried along the march. x and z uniform
// and periodic; y periodic or a wall (u^y below the bottom wall is 0), 1/d_y[j] per row.
template <typename T>
struct DivCoef {
    int nx, ny, nz;
    T idx, idz;          // 1/d of the uniform x and z directions
    const T* idy;        // 1/d_y[j]
    const T* ihy = nullptr;   // SC: 1/h_y[j]
    const double* sdt = nullptr;   // SCL: u is read as (dt beta) u, dt from sdt or sdt_host
    double sdt_host = 0.0, sbeta = 0.0;
};

// Block (32, 8); grid (ceil(nx/VEC/32), ceil(ny/8), ceil(nz/kchunk)). Needs nx % VEC == 0 and
// 16-byte aligned u and phi.
// SC: the divergence of Omega^-1 M u of the wall-bounded pullback (u^x, u^z scaled by 1/d_y[j],
// u^y by 1/h_y[j], the stored top wall faces of u^y taken as 0).
// SCL: the divergence of (dt beta) u (the step VJP's first cotangent).
template <typename T, int DIM, bool WALL, int VW = VecT<T>::N, bool SC = false, bool SCL = false>
__global__ void __launch_bounds__(256) k_divergence_vec(DivCoef<T> c, const T* __restrict__ u, T* __restrict__ phi,
                                                        int kchunk) {
    using VT = VecIO<T, VW>;
    constexpr int VEC = VW;
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    const long N = (long)nx * ny * nz;
    const long plane = (long)nx * ny;
    const int nvx = nx / VEC;
    const int lane = threadIdx.x, row = threadIdx.y;
    const int iv = blockIdx.x * 32 + lane;
    const int i0 = iv * VEC;
    const int j = blockIdx.y * 8 + row;
    const bool ok = iv < nvx && j < ny;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(kb + kchunk, nz);
    const T idy = __ldg(&c.idy[j < ny ? j : ny - 1]);
    const bool need_global_prev = iv == 0 || lane == 0;
    const long jrow = (long)(j < ny ? j : 0) * nx;
    const long jprev = (long)(j > 0 ? j - 1 : ny - 1) * nx;   // periodic wrap in y
    const bool bottom = WALL && j == 0;
    T Zm[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) Zm[e] = (T)0;
    if (DIM == 3 && ok) VT::ld(u + 2 * N + (long)(kb == 0 ? nz - 1 : kb - 1) * plane + jrow + i0, Zm);
    // SC row factors: x and z faces of row j, y faces of rows j and j - 1; SCL: times dt beta
    T sxz = (T)1, sy = (T)1, sym = (T)1;
    if constexpr (SC || SCL) {
        const T al = SCL ? (T)((c.sdt ? *c.sdt : c.sdt_host) * c.sbeta) : (T)1;
        if constexpr (SC) {
            const int jc = j < ny ? j : ny - 1;
            sxz = idy * al;
            sy = jc == ny - 1 ? (T)0 : __ldg(&c.ihy[jc]) * al;
            sym = jc > 0 ? __ldg(&c.ihy[jc - 1]) * al : (T)0;
        } else {
            sxz = sy = sym = al;
        }
        if (DIM == 3) {
#pragma unroll
            for (int e = 0; e < VEC; ++e) Zm[e] *= sxz;
        }
    }
    for (int k = kb; k < ke; ++k) {
        const long base = (long)k * plane;
        const long a = base + jrow + i0;
        T ux[VEC], uy[VEC], uym[VEC], uz[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) ux[e] = uy[e] = uym[e] = uz[e] = (T)0;
        if (ok) {
            VT::ld(u + a, ux);
            VT::ld(u + N + a, uy);
            if (!bottom) VT::ld(u + N + base + jprev + i0, uym);
            if (DIM == 3) VT::ld(u + 2 * N + a, uz);
            if constexpr (SC || SCL) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    ux[e] *= sxz;
                    uy[e] *= sy;
                    uym[e] *= sym;
                    uz[e] *= sxz;
                }
            }
        }
        T xprev = __shfl_up_sync(0xffffffffu, ux[VEC - 1], 1);
        if (ok && need_global_prev) xprev = u[base + jrow + (iv == 0 ? nx - 1 : i0 - 1)] * sxz;
        if (ok) {
            T d[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const T xm = e > 0 ? ux[e - 1] : xprev;
                T v = (ux[e] - xm) * c.idx;
                v += (uy[e] - uym[e]) * idy;
                if (DIM == 3) v += (uz[e] - Zm[e]) * c.idz;
                d[e] = v;
            }
            VT::st(phi + a, d);
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) Zm[e] = uz[e];
    }
}

}  // namespace ins
