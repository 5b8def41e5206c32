// Impl::spectrum, cfl, diag: shell spectrum, CFL time step and field diagnostics. Included by
// ins_grid.cu.
#pragma once

#include "ins_internal.cuh"

namespace {

// Shell energy spectrum of a periodic field (see ins.h, ins_spectrum).
template <typename T, int DIM, bool WALL>
ins_status Impl<T, DIM, WALL>::spectrum(ins_grid* g, const T* u, double* E, int kmax) {
    if (ins_status s0 = set_smem_attrs<T>(); s0 != INS_OK) return s0;
    cudaStream_t st = g->stream;
    const int nx = g->nx, ny = g->ny, nz = g->nz, nxh = g->nxh;
    const long lines = (long)ny * nz;
    cplx<T>* S = reinterpret_cast<cplx<T>*>(g->S);
    INS_CUDA(cudaMemsetAsync(E, 0, sizeof(double) * (kmax + 1), st));
    const double ntot = (double)g->N;
    for (int a = 0; a < g->dim; ++a) {
        const T* comp = u + (size_t)a * g->N;
        FftLine<T> lx = make_line<T>(g, 0);
        if (reg_fft_len(nx, sizeof(T) == 8)) {
            KLAUNCH(g, "fft_x_r2c", x_reg<T>(nx, true, st, lx.tw, comp, S, nullptr, (int)lines, nxh));
        } else {
            const int lg = g->lg_tw_x;
            const long pairs = (lines + 1) / 2;
            const unsigned blocks = (unsigned)((pairs + (1 << lg) - 1) >> lg);
            KLAUNCH(g, "fft_x_r2c", k_fft_x_r2c<T><<<blocks, FFT_THREADS, fft_smem<T>(nx, lg), st>>>(
                                        lx, comp, S, (int)lines, nxh, lg));
        }
        for (int d = 1; d < g->dim; ++d) {
            FftLine<T> pl = make_line<T>(g, d);
            long ncol, cdiv, outer, lstride;
            if (d == 1) {
                ncol = (long)nz * nxh;
                cdiv = nxh;
                outer = (long)ny * nxh;
                lstride = nxh;
            } else {
                ncol = (long)ny * nxh;
                cdiv = ncol;
                outer = 0;
                lstride = (long)ny * nxh;
            }
            if (reg_fft_len(pl.L)) {
                KLAUNCH(g, "fft_strided", strided_reg<T>(pl.L, st, pl.tw, S, ncol, cdiv, outer, lstride, 0,
                                                         (const T*)nullptr));
            } else {
                const int lg = d == 1 ? g->lg_tw_y : g->lg_tw_z;
                const unsigned blocks = (unsigned)((ncol + (1 << lg) - 1) >> lg);
                KLAUNCH(g, "fft_strided", k_fft_strided<T><<<blocks, FFT_THREADS, fft_smem<T>(pl.L, lg), st>>>(
                                              pl, S, ncol, cdiv, outer, lstride, 0, (const T*)nullptr, lg));
            }
        }
        KLAUNCH(g, "shell_bin", k_shell_bin<T><<<592, 256, (kmax + 1) * sizeof(double), st>>>(
                                    S, nx, ny, nz, nxh, kmax, E, 1.0 / (ntot * ntot)));
    }
    return INS_OK;
}

template <typename T, int DIM, bool WALL>
ins_status Impl<T, DIM, WALL>::cfl(ins_grid* g, const T* u, double cfl, double* dt_dev) {
    // reuse the stage-4 path's reduction: a read-only pass
    INS_CUDA(cudaMemsetAsync(g->diag, 0, 4 * sizeof(double), g->stream));
    INS_CUDA(cudaMemsetAsync(g->diag_max, 0, 2 * sizeof(unsigned long long), g->stream));
    KLAUNCH(g, "diag", k_diag<T, DIM, WALL><<<cell_grid(g), dim3(32, 8), 0, g->stream>>>(
                           make_geo<T>(g), u, g->geo64, g->diag, g->diag_max));
    // max |u^a|/h_a was reduced into diag_max[1]; finish on the device
    KLAUNCH(g, "cfl_finalize", k_cfl_finalize<<<1, 256, 0, g->stream>>>(g->diag_max + 1, g->one, 1, g->dmin2_nu, cfl, dt_dev));
    return INS_OK;
}

template <typename T, int DIM, bool WALL>
ins_status Impl<T, DIM, WALL>::diag(ins_grid* g, const T* u, double out[4]) {
    INS_CUDA(cudaMemsetAsync(g->diag, 0, 4 * sizeof(double), g->stream));
    INS_CUDA(cudaMemsetAsync(g->diag_max, 0, 2 * sizeof(unsigned long long), g->stream));
    KLAUNCH(g, "diag", k_diag<T, DIM, WALL><<<cell_grid(g), dim3(32, 8), 0, g->stream>>>(
                           make_geo<T>(g), u, g->geo64, g->diag, g->diag_max));
    double h[4];
    unsigned long long mx[2];
    INS_CUDA(cudaMemcpyAsync(h, g->diag, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    INS_CUDA(cudaMemcpyAsync(mx, g->diag_max, sizeof(mx), cudaMemcpyDeviceToHost, g->stream));
    INS_CUDA(cudaStreamSynchronize(g->stream));
    double vol = 1.0;
    for (int a = 0; a < g->dim; ++a) {
        double L = 0.0;
        for (double x : g->d[a]) L += x;
        vol *= L;
    }
    double dv, cf;
    std::memcpy(&dv, &mx[0], 8);
    std::memcpy(&cf, &mx[1], 8);
    out[0] = h[0] / vol;
    out[1] = dv;
    out[2] = cf;
    out[3] = h[3];
    if (h[3] > 0.0 || !std::isfinite(h[0])) return fail(INS_ERR_NONFINITE, "non-finite values in the field");
    return INS_OK;
}

}  // namespace
