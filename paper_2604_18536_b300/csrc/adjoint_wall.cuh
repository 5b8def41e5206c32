// Pullback of F on wall-bounded grids (channel: x, z periodic and uniform, y a no-slip wall,
// possibly stretched) for the step VJP (paper Sec. 3.4 and App. B pullbacks).
//
// Scatter form: every face output F^a_I is the sum of the App. A / App. B terms
//   convection  -(V_+ T_+ - V_- T_-) / width   (products of two interpolations of u),
//   diffusion   nu (c+ u_{I+e_b} + c- u_{I-e_b} - (c+ + c-) u_I),
// and each thread transposes the terms of its own faces, adding w^a_I dF^a_I/du_J into
// ubar_J with atomics. Neighbour values follow the forward boundary rules: x and z wrap;
// across a wall in y, u^y is 0 (wall-normal velocity) and u^x, u^z take the odd ghost
// (minus the first or last stored value), so the ghost's derivative lands on that stored
// value with a minus sign. The stored top wall faces of u^y are not unknowns: their
// outputs are skipped (the caller masks the inputs and the result).
//
// Also: the projection pullback P^T = M Omega P Omega^-1 M (Omega the face volumes, whose
// x/z factors cancel: rows of u^x, u^z are scaled by d_y[j], rows of u^y by h_y[j]), and
// the stage finish ubar0 += q, kbar = dt (b ybar + a q) for the scatter result q.
#pragma once

#include "common.cuh"

namespace ins {

template <typename T>
struct WallAdj {
    Geo<T> g;
    T nu;
};

// u^c at (i, j, k) with the boundary rules; returns the storage index and the sign
// (0: the value is a wall-normal zero).
struct Ref {
    long idx;
    int sgn;
};

__device__ __forceinline__ Ref wref(int c, int i, int j, int k, int nx, int ny, int nz, long N) {
    i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
    k = k < 0 ? k + nz : (k >= nz ? k - nz : k);
    int s = 1;
    if (j < 0 || j >= ny) {
        if (c == 1) return Ref{0, 0};
        j = j < 0 ? 0 : ny - 1;
        s = -1;
    }
    return Ref{c * N + ((long)k * ny + j) * nx + i, s};
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_adj_rhs_wall(WallAdj<T> c, const T* __restrict__ u, const T* __restrict__ w,
                                                      T* __restrict__ q, double* __restrict__ nu_part) {
    const Geo<T>& G = c.g;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const long N = (long)nx * ny * nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    double nup = 0.0;
    if (i < nx && j < ny) {
        const int n3[3] = {nx, ny, nz};
        const int I3[3] = {i, j, k};
        auto R = [&](int comp, int di, int dj, int dk) { return wref(comp, i + di, j + dj, k + dk, nx, ny, nz, N); };
        auto val = [&](const Ref& r) { return r.sgn == 0 ? (T)0 : (r.sgn > 0 ? u[r.idx] : -u[r.idx]); };
        auto add = [&](const Ref& r, T v) {
            if (r.sgn != 0) atomicAdd(&q[r.idx], r.sgn > 0 ? v : -v);
        };
        // 1/h and 1/d of direction a at index m (m = -1: the spacing below the first cell;
        // m = n: the mirrored ghost cell above a wall, or the wrap)
        auto invh = [&](int a, int m) {
            if (m < 0) return a == 1 ? G.coef(1, C_INV_D, 0) : G.coef(a, C_INV_H, n3[a] - 1);
            return G.coef(a, C_INV_H, m);
        };
        auto invd = [&](int a, int m) {
            if (m >= n3[a]) return a == 1 ? G.coef(1, C_INV_D, n3[a] - 1) : G.coef(a, C_INV_D, m - n3[a]);
            return G.coef(a, C_INV_D, m);
        };
        for (int a = 0; a < DIM; ++a) {
            if (a == 1 && j == ny - 1) continue;   // stored top wall face: not an unknown
            const Ref ra = R(a, 0, 0, 0);
            const T W = w[ra.idx];
            if (W == (T)0) continue;
            const int ea[3] = {a == 0, a == 1, a == 2};
            const int ia = I3[a];
            // self term: -(vp^2 - vm^2) / h_a
            {
                const Ref rp = R(a, ea[0], ea[1], ea[2]), rm = R(a, -ea[0], -ea[1], -ea[2]);
                const T u0 = val(ra), vp = (T)0.5 * (u0 + val(rp)), vm = (T)0.5 * (val(rm) + u0);
                const T cc = W * invh(a, ia);
                add(ra, -cc * (vp - vm));
                add(rp, -cc * vp);
                add(rm, cc * vm);
            }
            for (int b = 0; b < DIM; ++b) {
                if (b == a) continue;
                const int eb[3] = {b == 0, b == 1, b == 2};
                const int ib = I3[b];
                const T wl = G.coef(a, C_WL, ia), wr = G.coef(a, C_WR, ia);
                const Ref r1 = R(b, 0, 0, 0), r2 = R(b, ea[0], ea[1], ea[2]);
                const Ref r3 = R(b, -eb[0], -eb[1], -eb[2]), r4 = R(b, ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2]);
                const Ref rtp = R(a, eb[0], eb[1], eb[2]), rtm = R(a, -eb[0], -eb[1], -eb[2]);
                const T Vp = wl * val(r1) + wr * val(r2);
                const T Vm = wl * val(r3) + wr * val(r4);
                const T u0 = val(ra);
                const T Tp = (T)0.5 * (u0 + val(rtp)), Tm = (T)0.5 * (val(rtm) + u0);
                const T cc = W * invd(b, ib);
                add(r1, -cc * Tp * wl);
                add(r2, -cc * Tp * wr);
                add(r3, cc * Tm * wl);
                add(r4, cc * Tm * wr);
                add(ra, (T)0.5 * cc * (Vm - Vp));
                add(rtp, -(T)0.5 * cc * Vp);
                add(rtm, (T)0.5 * cc * Vm);
            }
            // diffusion (nu lap) and the nu partial <w, lap>
            T lap = (T)0;
            for (int b = 0; b < DIM; ++b) {
                const int eb[3] = {b == 0, b == 1, b == 2};
                const int ib = I3[b];
                T cp, cm;
                if (b == a) {
                    cp = invd(a, ia + 1) * invh(a, ia);
                    cm = invd(a, ia) * invh(a, ia);
                } else {
                    cp = invh(b, ib) * invd(b, ib);
                    cm = invh(b, ib - 1) * invd(b, ib);
                }
                const Ref rp = R(a, eb[0], eb[1], eb[2]), rm = R(a, -eb[0], -eb[1], -eb[2]);
                const T u0 = val(ra);
                lap += cp * val(rp) + cm * val(rm) - (cp + cm) * u0;
                add(rp, c.nu * W * cp);
                add(rm, c.nu * W * cm);
                add(ra, -c.nu * W * (cp + cm));
            }
            nup += (double)W * (double)lap;
        }
    }
    for (int o = 16; o > 0; o >>= 1) nup += __shfl_xor_sync(0xffffffffu, nup, o);
    __shared__ double red[8];
    if (threadIdx.x == 0) red[threadIdx.y] = nup;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double s = 0.0;
        for (int r = 0; r < 8; ++r) s += red[r];
        nu_part[((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
}

// out^a[row j] = mask * in^a * f^a_j with f = 1/d_y, 1/h_y, 1/d_y (inverse) or d_y, h_y, d_y;
// the stored top wall faces of u^y become 0. out may equal in.
template <typename T>
__global__ void k_row_scale(const T* __restrict__ in, T* __restrict__ out, const double* __restrict__ hy,
                            const double* __restrict__ dy, int nx, int ny, long N, int dim, int inverse) {
    const long n = (long)dim * N;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const int a = (int)(t / N);
        const long r = t - a * N;
        const int j = (int)((r / nx) % ny);
        double f = a == 1 ? hy[j] : dy[j];
        if (inverse) f = 1.0 / f;
        const bool top = a == 1 && j == ny - 1;
        out[t] = top ? (T)0 : (T)((double)in[t] * f);
    }
}

// ubar0 += q; kbar = dt (bn y + an q), y = ybar or (null) the old ubar0; the stored top
// wall faces of u^y are skipped (q there is not a pullback of an unknown).
template <typename T>
__global__ void k_adj_finish(const T* __restrict__ q, const T* __restrict__ ybar, T* __restrict__ ubar0,
                             T* __restrict__ kbar, const double* dt_dev, double dt_host, double bn, double an, int nx,
                             int ny, long N, int dim) {
    const double dt = dt_dev ? *dt_dev : dt_host;
    const T dtb = (T)(dt * bn), dta = (T)(dt * an);
    const long n = (long)dim * N;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const int a = (int)(t / N);
        const long r = t - a * N;
        const int j = (int)((r / nx) % ny);
        const T qv = (a == 1 && j == ny - 1) ? (T)0 : q[t];
        const T old = ubar0[t];
        ubar0[t] = old + qv;
        if (kbar) kbar[t] = fma(dtb, ybar ? ybar[t] : old, dta * qv);
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
