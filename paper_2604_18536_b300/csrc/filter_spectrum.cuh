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
