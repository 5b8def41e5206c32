// Pullback of the stage right-hand side F(u) = C(u) + nu diffusion(u) + f
// (paper Sec. 3.4, pullback equation; App. B pullbacks) on uniform periodic grids.
//
// With w the incoming cotangent of F at a stage state u:
//   ubar = J_C(u)^T w + nu diffusion(w)   (the diffusion is symmetric on a uniform
//                                          periodic grid), and
//   dF/dnu contributes <w, diffusion(u)> = <u, diffusion(w)> to nubar.
// J_C^T w is the transpose of the convection bilinear form in both arguments,
// written in gather form (no atomics) after summation by parts. For component
// a at cell J, with S_ab(J) = u_b(J) + u_b(J + e_a) (u_b summed along a):
//   self:  1/(2 D_a) [ (u_a + u_a^{+a}) (w_a^{+a} - w_a) + (u_a^{-a} + u_a) (w_a - w_a^{-a}) ]
//   b != a, u_a transported by u_b through the b-faces of the a-volume:
//          1/(4 D_b) [ S_ab(J) (w_a^{+b} - w_a) + S_ab(J - e_b) (w_a - w_a^{-b}) ]
//   b != a, u_a advecting u_b through the a-faces of the b-volume:
//          1/(4 D_a) [ S_ab(J) (w_b^{+a} - w_b) + S_ab(J - e_b) (w_b^{+a-b} - w_b^{-b}) ]
// The footprint is one cell in every direction, including the diagonal
// neighbours J + e_a - e_b.
//
// The same kernel finishes the reverse stage of the RK4 step pullback:
// ubar0 += ubar_s, and (when kb is given) the next stage cotangent
// kbar_{s-1} = dt b_{s-1} ybar + dt a_{s,s-1} ubar_s.
#pragma once

#include "common.cuh"

namespace ins {

template <typename T>
struct AdjCoef {
    int nx, ny, nz;
    T c1[3];     // 1/(2 D_a)
    T c2[3];     // 1/(4 D_a)
    T l2[3];     // 1/D_a^2
    T nu;
    const double* dt_dev;   // dt on the device, or null: dt_host
    double dt_host;
    double bn, an;          // b_{s-1}, a_{s,s-1} for the next stage cotangent
};

// Block (32, 8), grid (ceil(nx/32), ceil(ny/8), nz). nu_part[block] receives the block's
// partial sum of <u, diffusion(w)> (FP64, fixed order within the block).
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_adj_rhs(AdjCoef<T> c, const T* __restrict__ u, const T* __restrict__ w,
                                                 const T* __restrict__ ybar, T* __restrict__ ubar0,
                                                 T* __restrict__ kb, double* __restrict__ nu_part,
                                                 const T* __restrict__ extra) {
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    const long N = (long)nx * ny * nz;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    const bool ok = i < nx && j < ny;
    const double dt = c.dt_dev ? *c.dt_dev : c.dt_host;
    const T dtb = (T)(dt * c.bn), dta = (T)(dt * c.an);
    double nup = 0.0;
    if (ok) {
        const int n3[3] = {nx, ny, nz};
        const int id[3] = {i, j, k};
        // neighbour index along a with offset s in {-1, 0, +1}
        auto nb = [&](int a, int s) {
            int v = id[a] + s;
            return v < 0 ? v + n3[a] : (v >= n3[a] ? v - n3[a] : v);
        };
        // address of J + s_a e_a + s_b e_b
        auto at = [&](int a, int sa, int b, int sb) {
            int ix[3] = {i, j, k};
            ix[a] = nb(a, sa);
            if (b != a) ix[b] = nb(b, sb);
            return ((long)ix[2] * ny + ix[1]) * nx + ix[0];
        };
        const long J = ((long)k * ny + j) * nx + i;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const T* ua = u + a * N;
            const T* wa = w + a * N;
            const T ua0 = ua[J], uap = ua[at(a, 1, a, 0)], uam = ua[at(a, -1, a, 0)];
            const T wa0 = wa[J], wap = wa[at(a, 1, a, 0)], wam = wa[at(a, -1, a, 0)];
            T acc = c.c1[a] * fma(ua0 + uap, wap - wa0, (uam + ua0) * (wa0 - wam));
            T lap = c.l2[a] * (wap + wam - (T)2 * wa0);
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                if (b == a) continue;
                const T* ub = u + b * N;
                const T* wb = w + b * N;
                const long Jmb = at(b, -1, b, 0);
                const long Jpa = at(a, 1, a, 0);
                const long Jpamb = at(a, 1, b, -1);
                const T S0 = ub[J] + ub[Jpa];
                const T S1 = ub[Jmb] + ub[Jpamb];
                const T wabp = wa[at(b, 1, b, 0)], wabm = wa[Jmb];
                acc = fma(c.c2[b], fma(S0, wabp - wa0, S1 * (wa0 - wabm)), acc);
                acc = fma(c.c2[a], fma(S0, wb[Jpa] - wb[J], S1 * (wb[Jpamb] - wb[Jmb])), acc);
                lap = fma(c.l2[b], wabp + wabm - (T)2 * wa0, lap);
            }
            T ubs = fma(c.nu, lap, acc);
            if (extra) ubs += extra[a * N + J];   // closure pullback J_m^T w
            nup += (double)ua0 * (double)lap;
            const long e = a * N + J;
            ubar0[e] = ubar0[e] + ubs;
            if (kb) kb[e] = fma(dtb, ybar[e], dta * ubs);
        }
    }
    // block partial of <u, diffusion(w)>
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

// out = (dt * beta) * x (the last stage's cotangent dt b_4 ybar); dt from the device or dt_host.
template <typename T>
__global__ void k_scale_dt(const T* __restrict__ x, T* __restrict__ out, const double* dt_dev, double dt_host,
                           double beta, long n) {
    const T alpha = (T)((dt_dev ? *dt_dev : dt_host) * beta);
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        out[t] = alpha * x[t];
}

// *acc += sum of the partials, in a fixed order (one block of 256 threads).
__global__ void k_sum_partials(const double* __restrict__ part, long n, double* __restrict__ acc) {
    __shared__ double red[256];
    double s = 0.0;
    for (long t = threadIdx.x; t < n; t += blockDim.x) s += part[t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *acc += red[0];
}

}  // namespace ins
