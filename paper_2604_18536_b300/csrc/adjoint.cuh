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
// kbar_{s-1} = dt b_{s-1} ybar + dt a_{s,s-1} ubar_s; with ybar null the value of ubar0
// before the update takes ybar's place (the chained state cotangent of a low-storage scheme).
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

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
            const T old = ubar0[e];
            ubar0[e] = old + ubs;
            if (kb) kb[e] = fma(dtb, ybar ? ybar[e] : old, dta * ubs);
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
template <typename T, typename S = T>
__global__ void k_scale_dt(const S* __restrict__ x, T* __restrict__ out, const double* dt_dev, double dt_host,
                           double beta, long n) {
    const T alpha = (T)((dt_dev ? *dt_dev : dt_host) * beta);
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        out[t] = alpha * cvt_in<T>(x[t]);
}

// *acc += sum of the partials, in a fixed order (one block of 256 threads).
static __global__ void k_sum_partials(const double* __restrict__ part, long n, double* __restrict__ acc) {
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

namespace ins {

// The same pullback as k_adj_rhs for 3-D periodic grids, with the z march of k_rhs_div:
// a CTA of 32 x 8 threads owns a 32 x 8 column and a chunk of planes; the planes k-1, k,
// k+1 of u and w (all three components, one-cell halo in x and y, which covers every
// diagonal neighbour J + e_a - e_b the gather form reads) sit in dynamic shared memory as a
// four-slot ring; plane k+2 is loaded into registers while plane k is computed and stored into
// the slot of plane k-2 before the iteration's single barrier.
constexpr int AJX = 32, AJY = 8;
constexpr int AJSX = AJX + 2, AJSY = AJY + 2, AJSP = AJSX * AJSY;
constexpr int AJNT = AJX * AJY;
constexpr int AJPF = (AJSP + AJNT - 1) / AJNT;

// ubar0 <- old + ubs for a cotangent stored in the arithmetic type, or in FP64 for the double-float
// kernel (the FP64 accumulator keeps its precision: the double-float increment is added in FP64)
__device__ __forceinline__ float adj_accum(float old, float x) { return old + x; }
__device__ __forceinline__ double adj_accum(double old, double x) { return old + x; }
__device__ __forceinline__ double adj_accum(double old, df x) { return old + df_to_double(x); }
__device__ __forceinline__ double to_f64(float x) { return (double)x; }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(df x) { return df_to_double(x); }

// UI: storage type of the stage state u; Y: storage type of the cotangents ybar, uin and ubar0
// (T, or double for the double-float kernel of an FP64 grid).
template <typename T, typename UI = T, typename Y = T>
__global__ void __launch_bounds__(AJNT) k_adj_rhs_z(AdjCoef<T> c, const UI* __restrict__ u, const T* __restrict__ w,
                                                   const Y* __restrict__ ybar, Y* __restrict__ ubar0,
                                                   T* __restrict__ kb, double* __restrict__ nu_part,
                                                   const T* __restrict__ extra, int kchunk,
                                                   const Y* __restrict__ uin) {
    extern __shared__ __align__(16) unsigned char ajsm[];
    T(*s)[6][AJSP] = reinterpret_cast<T(*)[6][AJSP]>(ajsm);   // s[slot][comp: u 0-2, w 3-5][cell]
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    const long N = (long)nx * ny * nz;
    const long plane = (long)nx * ny;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * AJX;
    const int i0 = blockIdx.x * AJX, j0 = blockIdx.y * AJY;
    const int i = i0 + tx, j = j0 + ty;
    const bool ok = i < nx && j < ny;
    const int kb0 = blockIdx.z * kchunk, ke = min(kb0 + kchunk, nz);
    const double dt = c.dt_dev ? *c.dt_dev : c.dt_host;
    const T dtb = (T)(dt * c.bn), dta = (T)(dt * c.an);
    // in-plane source offsets of this thread's share of a plane
    int off[AJPF];
#pragma unroll
    for (int q = 0; q < AJPF; ++q) {
        const int e = tid + q * AJNT;
        off[q] = -1;
        if (e < AJSP) {
            const int li = e % AJSX, lj = e / AJSX;
            int gi = (i0 - 1 + li) % nx, gj = (j0 - 1 + lj) % ny;
            gi += gi < 0 ? nx : 0;
            gj += gj < 0 ? ny : 0;
            off[q] = gj * nx + gi;
        }
    }
    T v[6][AJPF];
    auto fetch = [&](int kk) {
        const long base = (long)kk * plane;
#pragma unroll
        for (int q = 0; q < AJPF; ++q)
            if (off[q] >= 0) {
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    v[cc][q] = cvt_in<T>(u[cc * N + base + off[q]]);
                    v[3 + cc][q] = w[cc * N + base + off[q]];
                }
            }
    };
    auto commit = [&](int slot) {
#pragma unroll
        for (int q = 0; q < AJPF; ++q)
            if (off[q] >= 0) {
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) s[slot][cc][tid + q * AJNT] = v[cc][q];
            }
    };
    auto wz = [nz](int k) { return k < 0 ? k + nz : (k >= nz ? k - nz : k); };
    auto slot = [kb0](int q) { return (q - kb0 + 1) & 3; };   // plane q >= kb0 - 1
    fetch(wz(kb0 - 1));
    commit(slot(kb0 - 1));
    fetch(wz(kb0));
    commit(slot(kb0));
    fetch(wz(kb0 + 1));
    commit(slot(kb0 + 1));
    __syncthreads();
    const int c0 = (ty + 1) * AJSX + (tx + 1);
    // offsets within a plane: +x = 1, +y = AJSX
    double nup = 0.0;
    T nupt = (T)0;   // this thread's part of <u, diffusion(w)> in the arithmetic type
    for (int k = kb0; k < ke; ++k) {
        const bool more = k + 1 < ke;
        if (more) fetch(wz(k + 2));
        if (ok) {
            const T* P[3] = {s[slot(k - 1)][0], s[slot(k)][0], s[slot(k + 1)][0]};   // planes k-1, k, k+1
            T lpart = (T)0;   // sum over the three faces of u . diffusion(w) / nu
            // the finish's own-cell values first, so their loads overlap the stencil arithmetic
            const long Jc = (long)k * plane + (long)j * nx + i;
            Y oldv[3];
            T yv[3], xv[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                oldv[a] = uin[a * N + Jc];   // the accumulator's previous value (ubar0, or ybar first)
                yv[a] = cvt_in<T>(ybar ? ybar[a * N + Jc] : oldv[a]);
                xv[a] = extra ? extra[a * N + Jc] : (T)0;
            }
            // value of field f (0-2 u, 3-5 w) at J + (dx, dy, dz)
            auto at = [&](int f, int dx, int dy, int dz) { return P[dz + 1][f * AJSP + c0 + dx + dy * AJSX]; };
            const long J = (long)k * plane + (long)j * nx + i;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int ea[3] = {0, 0, 0};
                ea[a] = 1;
                const T ua0 = at(a, 0, 0, 0), uap = at(a, ea[0], ea[1], ea[2]), uam = at(a, -ea[0], -ea[1], -ea[2]);
                const T wa0 = at(3 + a, 0, 0, 0), wap = at(3 + a, ea[0], ea[1], ea[2]),
                        wam = at(3 + a, -ea[0], -ea[1], -ea[2]);
                T acc = c.c1[a] * fma(ua0 + uap, wap - wa0, (uam + ua0) * (wa0 - wam));
                T lap = c.l2[a] * (wap + wam - (T)2 * wa0);
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if (b == a) continue;
                    int eb[3] = {0, 0, 0};
                    eb[b] = 1;
                    const T S0 = at(b, 0, 0, 0) + at(b, ea[0], ea[1], ea[2]);
                    const T S1 = at(b, -eb[0], -eb[1], -eb[2]) + at(b, ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2]);
                    const T wabp = at(3 + a, eb[0], eb[1], eb[2]), wabm = at(3 + a, -eb[0], -eb[1], -eb[2]);
                    const T wb0 = at(3 + b, 0, 0, 0), wbpa = at(3 + b, ea[0], ea[1], ea[2]);
                    const T wbm = at(3 + b, -eb[0], -eb[1], -eb[2]);
                    const T wbpam = at(3 + b, ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2]);
                    acc = fma(c.c2[b], fma(S0, wabp - wa0, S1 * (wa0 - wabm)), acc);
                    acc = fma(c.c2[a], fma(S0, wbpa - wb0, S1 * (wbpam - wbm)), acc);
                    lap = fma(c.l2[b], wabp + wabm - (T)2 * wa0, lap);
                }
                T ubs = fma(c.nu, lap, acc);
                if (extra) ubs += xv[a];
                lpart = fma(ua0, lap, lpart);
                const long e = a * N + J;
                ubar0[e] = adj_accum(oldv[a], ubs);
                if (kb) kb[e] = fma(dtb, yv[a], dta * ubs);
            }
            if constexpr (std::is_same<T, df>::value) nupt += lpart;
            else nup += (double)lpart;
        }
        // plane k + 2 into the slot of plane k - 2, which no thread reads after the previous barrier
        if (more) commit(slot(k + 2));
        __syncthreads();
    }
    if constexpr (std::is_same<T, df>::value) nup = to_f64(nupt);
    for (int o = 16; o > 0; o >>= 1) nup += __shfl_xor_sync(0xffffffffu, nup, o);
    __shared__ double red[AJY];
    if (tx == 0) red[ty] = nup;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int r = 0; r < AJY; ++r) t += red[r];
        nu_part[((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
}

}  // namespace ins
