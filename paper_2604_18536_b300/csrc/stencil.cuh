// Stencil kernels of the staggered finite-volume scheme (paper App. A momentum
// equation, App. B kernels) and the fused projection + RK update.
//
// k_divergence, k_sub_grad: D u and src - G p (projection, right-hand side).
// k_rk_update: k = F - G p and the stage update of the classic RK4 scheme or (LS) of
// the low-storage 3-stage Wray scheme; k_cfl_finalize: the
// CFL time step from per-index maxima; k_diag: energy, divergence, CFL maxima.
// (F and D F are computed by k_rhs_div in rhs.cuh.)
#pragma once

#include "common.cuh"

namespace ins {

// phi = D u (used by the projection).
template <typename T, int DIM, bool WALL>
__global__ void k_divergence(Geo<T> g, const T* __restrict__ u, T* __restrict__ phi) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long N = (long)nx * ny * nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long a = ((long)k * ny + j) * nx + i;
    const int im = i == 0 ? nx - 1 : i - 1;
    T d = (u[a] - u[a - i + im]) * g.coef(0, C_INV_D, i);
    T uym;
    if (j == 0) uym = WALL ? (T)0 : u[N + a + (long)(ny - 1) * nx];
    else uym = u[N + a - nx];
    d += (u[N + a] - uym) * g.coef(1, C_INV_D, j);
    if (DIM == 3) {
        const long az = k == 0 ? a + (long)(nz - 1) * nx * ny : a - (long)nx * ny;
        d += (u[2 * N + a] - u[2 * N + az]) * g.coef(2, C_INV_D, k);
    }
    phi[a] = d;
}

// out = src - G p (projection of u, or the projected right-hand side of F).
template <typename T, int DIM, bool WALL>
__global__ void k_sub_grad(Geo<T> g, const T* __restrict__ src, const T* __restrict__ p, T* __restrict__ out) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long N = (long)nx * ny * nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const long a = ((long)k * ny + j) * nx + i;
    const T p0 = p[a];
    const T pe = p[a - i + (i + 1 == nx ? 0 : i + 1)];
    out[a] = src[a] - (pe - p0) * g.coef(0, C_INV_H, i);
    if (WALL && j == ny - 1) {
        out[N + a] = (T)0;
    } else {
        const T pn = p[j + 1 == ny ? a - (long)(ny - 1) * nx : a + nx];
        out[N + a] = src[N + a] - (pn - p0) * g.coef(1, C_INV_H, j);
    }
    if (DIM == 3) {
        const long plane = (long)nx * ny;
        const T pt = p[k + 1 == nz ? a - (long)(nz - 1) * plane : a + plane];
        out[2 * N + a] = src[2 * N + a] - (pt - p0) * g.coef(2, C_INV_H, k);
    }
}

// Stage update of classic RK4 (Sec. 2.6.2), k = F - G p:
//  stage 0: acc = b0 k;          us = u0 + dt a1 k
//  stage 1,2: acc += b k;        us = u0 + dt a k
//  stage 3: u0 = u0 + dt (acc + b3 k) (in place), plus the CFL maxima and the finite check.
// CFL maxima: max_I |u^a_I| / h_a[i_a] = max_i (max over the other indices of |u^a|) / h_a[i]
// because a correctly rounded division by a fixed positive h is monotone. The stage-3
// update therefore only reduces max |u^a| per index of direction a (bit patterns of
// non-negative doubles order like the doubles) into mx[off_a + i]; the divisions happen
// once per index in k_cfl_finalize, giving the same bits as dividing every element.
struct RkArgs {
    const double* dt_dev;
    double dt_host;
    double a_next;   // RK4: a_{s+1,s}; low-storage: gamma_s
    double b;        // RK4: b_s; low-storage: zeta_s (weight of the previous stage's k)
    int stage;
    int last;        // low-storage: this is the last stage (CFL maxima, finite check)
    unsigned long long* mx;   // [nx + ny + nz] per-index maxima of |u^a|; null: skip
    unsigned int* err_flag;   // bit 0: non-finite value seen
};

// Block shape must be (32, 8): x rows of one warp each.
//
// RK4 (LS = false): stage 0 acc = b k, us = u0 + dt a k; stages 1, 2 acc += b k,
// us = u0 + dt a k; stage 3 u0 += dt (acc + b k).
// Low storage (LS = true, the two-register form u_{s+1} = u_s + dt (gamma_s k_s +
// zeta_s k_{s-1})): u0 holds u_s, acc holds k_{s-1} (read for stage > 0) and receives k_s
// (unless last); the result goes to us, or back into u0 when us is null.
template <typename T, int DIM, bool WALL, bool LS = false>
__global__ void __launch_bounds__(256) k_rk_update(Geo<T> g, const T* __restrict__ F, const T* __restrict__ p,
                                                   T* __restrict__ u0, T* __restrict__ acc, T* __restrict__ us,
                                                   RkArgs ra) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long N = (long)nx * ny * nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const bool in = i < nx && j < ny;
    const double dt = ra.dt_dev ? *ra.dt_dev : ra.dt_host;
    const T dta = (T)(dt * ra.a_next), bb = (T)ra.b, dtt = (T)dt;
    const T dtz = (T)(dt * ra.b);
    const bool fin = LS ? ra.last != 0 : ra.stage == 3;
    double q[3] = {0.0, 0.0, 0.0};
    bool bad = false;
    if (in) {
        const long a = ((long)k * ny + j) * nx + i;
        const T p0 = p[a];
        T kk[3];
        kk[0] = F[a] - (p[a - i + (i + 1 == nx ? 0 : i + 1)] - p0) * g.coef(0, C_INV_H, i);
        if (WALL && j == ny - 1) kk[1] = (T)0;
        else kk[1] = F[N + a] - (p[j + 1 == ny ? a - (long)(ny - 1) * nx : a + nx] - p0) * g.coef(1, C_INV_H, j);
        if (DIM == 3) {
            const long plane = (long)nx * ny;
            kk[2] = F[2 * N + a] - (p[k + 1 == nz ? a - (long)(nz - 1) * plane : a + plane] - p0) *
                                       g.coef(2, C_INV_H, k);
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            const long e = c * N + a;
            const T u0v = u0[e];
            if (LS) {
                T inc = dta * kk[c];
                if (ra.stage > 0) inc = fma(dtz, acc[e], inc);
                const T un = u0v + inc;
                if (!ra.last) acc[e] = kk[c];
                if (us) us[e] = un;
                else u0[e] = un;
                if (ra.last) {
                    q[c] = fabs((double)un);
                    bad |= !isfinite(un);
                }
            } else if (ra.stage == 0) {
                if (acc) acc[e] = bb * kk[c];   // null: stage state only (the step VJP's recompute)
                us[e] = u0v + dta * kk[c];
            } else if (ra.stage < 3) {
                acc[e] = acc[e] + bb * kk[c];
                us[e] = u0v + dta * kk[c];
            } else {
                const T un = u0v + dtt * (acc[e] + bb * kk[c]);
                u0[e] = un;
                q[c] = fabs((double)un);
                bad |= !isfinite(un);
            }
        }
    }
    if (fin) {
        if (ra.mx) {
            __shared__ double sx[8][33];
            const int lane = threadIdx.x, row = threadIdx.y;
            // x: max over the 8 rows of the block, per column i
            sx[row][lane] = q[0];
            // y: max over the warp (one row j)
            double qy = q[1];
            for (int o = 16; o > 0; o >>= 1) qy = fmax(qy, __shfl_xor_sync(0xffffffffu, qy, o));
            if (lane == 0 && j < ny && qy > 0.0)
                atomicMax(&ra.mx[nx + j], (unsigned long long)__double_as_longlong(qy));
            double qz = q[2];
            if (DIM == 3) {
                for (int o = 16; o > 0; o >>= 1) qz = fmax(qz, __shfl_xor_sync(0xffffffffu, qz, o));
            }
            __syncthreads();
            if (row == 0) {
                double m = sx[0][lane];
#pragma unroll
                for (int r = 1; r < 8; ++r) m = fmax(m, sx[r][lane]);
                if (i < nx && m > 0.0) atomicMax(&ra.mx[i], (unsigned long long)__double_as_longlong(m));
            }
            if (DIM == 3) {
                __syncthreads();
                if (lane == 0) sx[row][32] = qz;
                __syncthreads();
                if (row == 0 && lane == 0) {
                    double m = sx[0][32];
                    for (int r = 1; r < 8; ++r) m = fmax(m, sx[r][32]);
                    if (m > 0.0) atomicMax(&ra.mx[nx + ny + k], (unsigned long long)__double_as_longlong(m));
                }
            }
        }
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(ra.err_flag, 1u);
    }
}

// dt = cfl * min(1 / max_{a,i} mx[off_a + i] / h_a[i], dmin^2 / nu); resets mx to 0.
// h64 holds h_x, h_y, h_z back to back (the same layout as mx). One block of 256 threads.
static __global__ void k_cfl_finalize(unsigned long long* mx, const double* __restrict__ h64, int ntot, double dmin2_nu,
                               double cfl, double* dt_out) {
    __shared__ double red[256];
    double m = 0.0;
    for (int t = threadIdx.x; t < ntot; t += blockDim.x) {
        const double v = __longlong_as_double((long long)mx[t]);
        m = fmax(m, v / h64[t]);
        mx[t] = 0ull;
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mm = red[0];
        const double conv = mm == 0.0 ? INFINITY : 1.0 / mm;
        *dt_out = cfl * fmin(conv, dmin2_nu);
    }
}

// Per-block partial sums/maxima for ins_diag: ke (weighted), max |div|, max |u|/h, nonfinite count.
template <typename T, int DIM, bool WALL>
__global__ void k_diag(Geo<T> g, const T* __restrict__ u, const double* __restrict__ vol_face, double* __restrict__ out,
                       unsigned long long* __restrict__ maxes) {
    // vol_face: per-direction face-volume factors, [a][n_a] products handled on the fly:
    // |Omega^a_I| = h_a[i_a] * prod_{b != a} d_b[i_b], given as three per-direction arrays
    // w_h[a] at vol_face + a*(nx+ny+nz) (h_a) and w_d at vol_face + 3*(nx+ny+nz) (d).
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long N = (long)nx * ny * nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const int off[3] = {0, nx, nx + ny};
    const int S = nx + ny + nz;
    const double* hh = vol_face;            // h_a at hh[off[a] + idx]
    const double* dd = vol_face + S;        // d_a at dd[off[a] + idx]
    double ke = 0.0, dv = 0.0, cf = 0.0, nf = 0.0;
    if (i < nx && j < ny) {
        const long a = ((long)k * ny + j) * nx + i;
        const int id[3] = {i, j, k};
        for (int c = 0; c < DIM; ++c) {
            const double v = (double)u[c * N + a];
            double w = hh[off[c] + id[c]];
            for (int b = 0; b < DIM; ++b)
                if (b != c) w *= dd[off[b] + id[b]];
            if (WALL && c == 1 && j == ny - 1) w = 0.0;
            ke += 0.5 * w * v * v;
            cf = fmax(cf, fabs(v) / hh[off[c] + id[c]]);
            if (!isfinite(v)) nf += 1.0;
        }
        // divergence
        const int im = i == 0 ? nx - 1 : i - 1;
        double d = ((double)u[a] - (double)u[a - i + im]) / dd[off[0] + i];
        double uym = (j == 0) ? (WALL ? 0.0 : (double)u[N + a + (long)(ny - 1) * nx]) : (double)u[N + a - nx];
        d += ((double)u[N + a] - uym) / dd[off[1] + j];
        if (DIM == 3) {
            const long az = k == 0 ? a + (long)(nz - 1) * nx * ny : a - (long)nx * ny;
            d += ((double)u[2 * N + a] - (double)u[2 * N + az]) / dd[off[2] + k];
        }
        dv = fabs(d);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ke += __shfl_xor_sync(0xffffffffu, ke, o);
        nf += __shfl_xor_sync(0xffffffffu, nf, o);
        dv = fmax(dv, __shfl_xor_sync(0xffffffffu, dv, o));
        cf = fmax(cf, __shfl_xor_sync(0xffffffffu, cf, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], ke);
        atomicAdd(&out[3], nf);
        if (dv > 0.0 || dv != dv) atomicMax(&maxes[0], (unsigned long long)__double_as_longlong(dv));
        if (cf > 0.0 || cf != cf) atomicMax(&maxes[1], (unsigned long long)__double_as_longlong(cf));
    }
}

}  // namespace ins
