// Face-averaging filter and shell energy spectrum (filtered DNS as closure
// training data, paper Sec. 4; energy spectra as the closure's error measure).
//
// Filter: a coarse grid m times coarser in every direction; the coarse u^a on
// the face to the right of coarse cell I is the mean of the m^(d-1) fine u^a
// on the fine faces that tile it (fine face index (I_a + 1) m - 1 along a,
// fine cells I_b m .. I_b m + m - 1 along the other directions). Face means
// keep a divergence-free field divergence free on the coarse grid.
//
// Spectrum: E(k) = sum over wavevectors with floor(|kvec| + 1/2) = k of
// 1/2 sum_a |uhat_a(kvec)|^2 / N^(2d), uhat the unnormalised DFT. The half
// spectrum kx in [0, nx/2] is stored, so every kx except 0 and nx/2 stands for
// two wavevectors. Shell indices are computed in FP64 from integer wavenumbers.
#pragma once

#include "common.cuh"

namespace ins {

template <typename T, int DIM>
__global__ void k_filter_face(const T* __restrict__ fine, T* __restrict__ coarse, int cx, int cy, int cz, int m) {
    const long Nc = (long)cx * cy * cz;
    const long fx = (long)cx * m, fy = (long)cy * m, fz = DIM == 3 ? (long)cz * m : 1;
    const long Nf = fx * fy * fz;
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= DIM * Nc) return;
    const int a = (int)(t / Nc);
    const long r = t - a * Nc;
    const int I = (int)(r % cx);
    const int J = (int)((r / cx) % cy);
    const int K = (int)(r / ((long)cx * cy));
    const T* f = fine + a * Nf;
    // fine index ranges: along a the single face (I_a + 1) m - 1, along the others m cells
    int lo[3] = {I * m, J * m, K * m};
    int cnt[3] = {m, m, DIM == 3 ? m : 1};
    const int ci[3] = {I, J, K};
    lo[a] = (ci[a] + 1) * m - 1;
    cnt[a] = 1;
    double s = 0.0;
    for (int kk = 0; kk < cnt[2]; ++kk)
        for (int jj = 0; jj < cnt[1]; ++jj)
            for (int ii = 0; ii < cnt[0]; ++ii)
                s += (double)f[((long)(lo[2] + kk) * fy + (lo[1] + jj)) * fx + (lo[0] + ii)];
    const int nsum = cnt[0] * cnt[1] * cnt[2];
    coarse[t] = (T)(s / nsum);
}

// Accumulate 1/2 |S|^2 (times the half-spectrum weight) into shells. S is the forward
// x, y (, z) transform of one component in the layout of the Poisson half spectrum.
// Block-local histogram in shared memory, then one atomicAdd per shell per block.
template <typename T>
__global__ void k_shell_bin(const cplx<T>* __restrict__ S, int nx, int ny, int nz, int nxh, int kmax,
                            double* __restrict__ E, double norm) {
    extern __shared__ double hist[];
    for (int t = threadIdx.x; t <= kmax; t += blockDim.x) hist[t] = 0.0;
    __syncthreads();
    const long n = (long)nxh * ny * nz;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const int kx = (int)(t % nxh);
        const long rr = t / nxh;
        const int jy = (int)(rr % ny);
        const int jz = (int)(rr / ny);
        const int ky = jy <= ny / 2 ? jy : jy - ny;   // numpy.fft.fftfreq ordering
        const int kz = jz <= nz / 2 ? jz : jz - nz;
        const double kk = sqrt((double)kx * kx + (double)ky * ky + (double)kz * kz);
        const int shell = (int)floor(kk + 0.5);
        if (shell > kmax) continue;
        const cplx<T> v = S[t];
        const double w = (kx == 0 || 2 * kx == nx) ? 1.0 : 2.0;
        const double e = 0.5 * w * ((double)v.re * v.re + (double)v.im * v.im) * norm;
        atomicAdd(&hist[shell], e);
    }
    __syncthreads();
    for (int t = threadIdx.x; t <= kmax; t += blockDim.x)
        if (hist[t] != 0.0) atomicAdd(&E[t], hist[t]);
}

}  // namespace ins

namespace ins {

// Plane statistics along the wall-normal y of a channel (paper Sec. 6.2: mean velocity and
// Reynolds stresses from velocities interpolated to the volume centres). One block per row j;
// FP64 sums over (i, k) of uc_a and uc_a uc_b, uc_a = (u^a_I + u^a_{I-e_a}) / 2 with the wall
// value 0 below the first cell for u^y. out[q * ny + j]: q = 0..2 means, 3..8 covariances
// (xx, xy, xz, yy, yz, zz).
template <typename T>
__global__ void k_wall_profiles(const T* __restrict__ u, int nx, int ny, int nz, double* __restrict__ out) {
    const int j = blockIdx.x;
    const long N = (long)nx * ny * nz;
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (long t = threadIdx.x; t < (long)nx * nz; t += blockDim.x) {
        const int i = (int)(t % nx), k = (int)(t / nx);
        const long a = ((long)k * ny + j) * nx + i;
        const int im = i == 0 ? nx - 1 : i - 1;
        const int km = k == 0 ? nz - 1 : k - 1;
        const double cx = 0.5 * ((double)u[a] + (double)u[a - i + im]);
        const double cy = 0.5 * ((double)u[N + a] + (j == 0 ? 0.0 : (double)u[N + a - nx]));
        const double cz = 0.5 * ((double)u[2 * N + a] + (double)u[2 * N + ((long)km * ny + j) * nx + i]);
        s[0] += cx; s[1] += cy; s[2] += cz;
        s[3] += cx * cx; s[4] += cx * cy; s[5] += cx * cz;
        s[6] += cy * cy; s[7] += cy * cz; s[8] += cz * cz;
    }
    __shared__ double red[9][256];
    for (int q = 0; q < 9; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 9; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double inv = 1.0 / ((double)nx * nz);
        double m[3];
        for (int q = 0; q < 3; ++q) {
            m[q] = red[q][0] * inv;
            out[q * ny + j] = m[q];
        }
        const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
        for (int q = 0; q < 6; ++q) out[(3 + q) * ny + j] = red[3 + q][0] * inv - m[pa[q]] * m[pb[q]];
    }
}

}  // namespace ins
