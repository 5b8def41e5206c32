// Projection + classic RK4 stage update of the double-float FP64 step (periodic grids).
//
// The same update as k_rk_update_vec (paper Sec. 2.6.2; pressure gradient of App. B),
//   k = F - G p, (G p)^a = (p_{I+e_a} - p_I) / h_a,
//   stage 0: acc = b0 k;  stages 1, 2: acc += b k;  us = u0 + dt a k;
//   stage 3: u0 = u0 + dt (acc + b3 k) in place, the CFL per-index maxima of |u_{n+1}| and
//            the non-finite flag,
//   stage -1 (projection only, the step pullback's P^T): us = F - G p (u0 and acc untouched),
// and for Wray's low-storage scheme (LS; two registers u and k_{s-1})
//   u0 = u0 + dt (gamma_s k + zeta_s acc) in place (the increment added in FP64; into uto instead when
//   uto is given, the stage recompute of the pullback), acc = k (not on the last stage), the maxima and
//   the flag on the last stage,
// with F, p, acc and the stage state us stored as double-float pairs and u0 the caller's FP64
// field. The arithmetic is double-float (FP32 pipe); u0 is split by bits when it is read, and
// the last stage adds the double-float increment dt (acc + b3 k) to the FP64 u0 in FP64, so the
// stored velocity keeps its full precision and only the increment carries double-float
// rounding. The maxima compare the FP64 bit patterns of |u| as integers (non-negative doubles
// order like their bit patterns), which keeps them exact and off the FP64 pipe.
// Each thread owns two consecutive cells in x (16-byte accesses) of one row and marches through a
// chunk of z planes; the x neighbour of the second cell comes from the next lane.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"
#include "stencil.cuh"

namespace ins {

struct RkCoefDf {
    int nx, ny, nz;
    df ihx, ihy, ihz;   // 1/h of the uniform periodic directions
    const double* ihy_row;   // WALL: 1/h_y per row (FP64, split by bits once per thread)
};

__device__ __forceinline__ void ld2(const df* p, df (&x)[2]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = df(v.x, v.y);
    x[1] = df(v.z, v.w);
}
__device__ __forceinline__ void st2(df* p, const df (&x)[2]) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0].hi, x[0].lo, x[1].hi, x[1].lo);
}
__device__ __forceinline__ void ld2(const double* p, double (&x)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    x[0] = v.x;
    x[1] = v.y;
}
__device__ __forceinline__ void st2(double* p, const double (&x)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
}
// |x| as the bit pattern of an FP64 value (ordered like the values for non-negative doubles)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Block (32, 8); grid (ceil(nx/2/32), ceil(ny/8), ceil(nz/kchunk)). Needs nx even and 16-byte
// aligned fields. WALL: y is a no-slip wall direction with a stretched spacing (1/h_y per row); the
// stored top wall face of u^y (row ny - 1) is no unknown: its k is 0, so it keeps its value.
template <int DIM, bool LS = false, bool WALL = false>
__global__ void __launch_bounds__(256) k_rk_update_df(RkCoefDf c, const df* __restrict__ F, const df* __restrict__ p,
                                                      double* __restrict__ u0, df* __restrict__ acc,
                                                      df* __restrict__ us, RkArgs ra, int kchunk,
                                                      double* __restrict__ uto = nullptr) {
    constexpr int VEC = 2;
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
    const df dta = df(dt * ra.a_next), bb = df(ra.b), dtt = df(dt), dtz = df(dt * ra.b);
    const bool fin = LS ? ra.last != 0 : ra.stage == 3;
    const bool last_vec = iv == nvx - 1;
    const bool need_global_next = last_vec || lane == 31;
    const long jrow = (long)(j < ny ? j : 0) * nx;
    const df ihy = WALL ? (j < ny ? df_split(__ldg(&c.ihy_row[j])) : df(0.0f, 0.0f)) : c.ihy;
    const bool ytop = WALL && j == ny - 1;   // the top wall face of u^y
    const long jnext = (long)(j + 1 < ny ? j + 1 : 0) * nx;   // periodic wrap in y
    unsigned long long mxx[VEC] = {0ull, 0ull}, mxy = 0ull;
    bool bad = false;
    df P0[VEC], Pt[VEC];
    if (ok) ld2(p + (long)kb * plane + jrow + i0, P0);
    else P0[0] = P0[1] = df(0.0f, 0.0f);
    for (int k = kb; k < ke; ++k) {
        const long base = (long)k * plane;
        const long a = base + jrow + i0;
        const long kt = (k + 1 < nz ? (long)(k + 1) : 0) * plane;
        // x neighbour of the second cell: first cell of the next vector (next lane or wrap)
        df pnext;
        pnext.hi = __shfl_down_sync(0xffffffffu, P0[0].hi, 1);
        pnext.lo = __shfl_down_sync(0xffffffffu, P0[0].lo, 1);
        unsigned long long qz = 0ull;
        if (ok) {
            if (need_global_next) pnext = p[base + jrow + (last_vec ? 0 : i0 + VEC)];
            df Pn[VEC];
            if (DIM == 3) ld2(p + kt + jrow + i0, Pt);
            ld2(p + base + jnext + i0, Pn);
            df f[3][VEC], kk[3][VEC];
            ld2(F + a, f[0]);
            ld2(F + N + a, f[1]);
            if (DIM == 3) ld2(F + 2 * N + a, f[2]);
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const df pe = e + 1 < VEC ? P0[e + 1] : pnext;
                kk[0][e] = fma(P0[e] - pe, c.ihx, f[0][e]);
                kk[1][e] = ytop ? df(0.0f, 0.0f) : fma(P0[e] - Pn[e], ihy, f[1][e]);
                if (DIM == 3) kk[2][e] = fma(P0[e] - Pt[e], c.ihz, f[2][e]);
            }
#pragma unroll
            for (int cc = 0; cc < DIM; ++cc) {
                const long ea = cc * N + a;
                if (ra.stage < 0) {
                    st2(us + ea, kk[cc]);
                    continue;
                }
                double uv[VEC];
                df av[VEC], sv[VEC];
                ld2(u0 + ea, uv);
                if (LS) {
                    if (ra.stage > 0) ld2(acc + ea, av);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        const df inc = ra.stage > 0 ? fma(dtz, av[e], dta * kk[cc][e]) : dta * kk[cc][e];
                        uv[e] += df_to_double(inc);
                        if (ra.last) {
                            const unsigned long long q = abs_bits(uv[e]);
                            bad |= (q >> 52) == 0x7ffull;
                            if (cc == 0) mxx[e] = q > mxx[e] ? q : mxx[e];
                            else if (cc == 1) mxy = q > mxy ? q : mxy;
                            else qz = q > qz ? q : qz;
                        }
                    }
                    if (!ra.last) st2(acc + ea, kk[cc]);
                    st2((uto ? uto : u0) + ea, uv);
                } else if (ra.stage == 0) {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        av[e] = bb * kk[cc][e];
                        sv[e] = fma(dta, kk[cc][e], df_split(uv[e]));
                    }
                    if (acc) st2(acc + ea, av);
                    st2(us + ea, sv);
                } else if (ra.stage < 3) {
                    ld2(acc + ea, av);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        av[e] = fma(bb, kk[cc][e], av[e]);
                        sv[e] = fma(dta, kk[cc][e], df_split(uv[e]));
                    }
                    st2(acc + ea, av);
                    st2(us + ea, sv);
                } else {
                    ld2(acc + ea, av);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        uv[e] += df_to_double(dtt * fma(bb, kk[cc][e], av[e]));
                        const unsigned long long q = abs_bits(uv[e]);
                        bad |= (q >> 52) == 0x7ffull;
                        if (cc == 0) mxx[e] = q > mxx[e] ? q : mxx[e];
                        else if (cc == 1) mxy = q > mxy ? q : mxy;
                        else qz = q > qz ? q : qz;
                    }
                    st2(u0 + ea, uv);
                }
            }
        } else {
            Pt[0] = Pt[1] = df(0.0f, 0.0f);
        }
        if (fin && ra.mx && DIM == 3) {
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long t = __shfl_xor_sync(0xffffffffu, qz, o);
                qz = t > qz ? t : qz;
            }
            if (lane == 0 && qz > 0ull) atomicMax(&ra.mx[nx + ny + k], qz);
        }
        P0[0] = Pt[0];
        P0[1] = Pt[1];
    }
    if (fin) {
        if (ra.mx) {
            __shared__ unsigned long long sx[8][32 * VEC + 1];
#pragma unroll
            for (int e = 0; e < VEC; ++e) sx[row][lane * VEC + e] = mxx[e];
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long t = __shfl_xor_sync(0xffffffffu, mxy, o);
                mxy = t > mxy ? t : mxy;
            }
            if (lane == 0 && j < ny && mxy > 0ull) atomicMax(&ra.mx[nx + j], mxy);
            __syncthreads();
            if (row == 0 && iv < nvx) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    unsigned long long m = sx[0][lane * VEC + e];
                    for (int r = 1; r < 8; ++r) m = sx[r][lane * VEC + e] > m ? sx[r][lane * VEC + e] : m;
                    if (m > 0ull) atomicMax(&ra.mx[i0 + e], m);
                }
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(ra.err_flag, 1u);
    }
}

// r = D F (App. B divergence kernel) in double-float on a uniform periodic grid:
// r_I = sum_a (F^a_I - F^a_{I-e_a}) / d_a. One cell per thread (grid-stride); the neighbours below
// come through the caches.
template <int DIM>
__global__ void __launch_bounds__(256) k_div_df(int nx, int ny, int nz, df idx, df idy, df idz,
                                                const df* __restrict__ F, df* __restrict__ r) {
    const long N = (long)nx * ny * nz;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < N; t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nx);
        const long rest = t / nx;
        const int j = (int)(rest % ny);
        const int k = (int)(rest / ny);
        const long tx = i > 0 ? t - 1 : t + nx - 1;
        const long ty = j > 0 ? t - nx : t + (long)(ny - 1) * nx;
        df acc = (ldg_t(F + t) - ldg_t(F + tx)) * idx;
        acc = fma(ldg_t(F + N + t) - ldg_t(F + N + ty), idy, acc);
        if (DIM == 3) {
            const long tz = k > 0 ? t - (long)nx * ny : t + (long)(nz - 1) * nx * ny;
            acc = fma(ldg_t(F + 2 * N + t) - ldg_t(F + 2 * N + tz), idz, acc);
        }
        r[t] = acc;
    }
}

}  // namespace ins
