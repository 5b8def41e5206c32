// libins: grid handles, settings, diagnostics, spectrum and wall statistics, the face-average
// filter, launch accounting and profiling, and the FMA-rate probe (C ABI in include/ins.h).
//
// The grid handle owns: per-direction stencil coefficients (field dtype), FP64
// geometry for the exact CFL rule and diagnostics, FFT twiddle tables, the
// spectral inverse-Laplacian table (all-periodic grids) or the FP64 Thomas
// factors (wall-normal y), and the step workspace (F, RK accumulator, stage
// state, r/p and the half spectrum). Nothing is allocated after creation.
#include "ins_internal.cuh"
#include "impl_diag.cuh"

extern "C" {

const char* ins_last_error(void) { return g_err.c_str(); }

const char* ins_version(void) { return "libins 0.1 (sm_103a)"; }

ins_status ins_grid_create(const ins_grid_desc* desc, void* stream, ins_grid** out) {
    g_err.clear();
    if (!desc || !out) return fail(INS_ERR_ARG, "ins_grid_create: null desc or out");
    *out = nullptr;
    const ins_grid_desc& D = *desc;
    if (D.dim != 2 && D.dim != 3) return fail(INS_ERR_ARG, "dim must be 2 or 3");
    if (D.dtype != INS_F32 && D.dtype != INS_F64) return fail(INS_ERR_ARG, "dtype must be INS_F32 or INS_F64");
    if (!(D.nu >= 0.0) || !std::isfinite(D.nu)) return fail(INS_ERR_ARG, "nu must be finite and >= 0");
    if (D.scheme != INS_RK4 && D.scheme != INS_WRAY3) return fail(INS_ERR_ARG, "scheme must be INS_RK4 or INS_WRAY3");
    for (int a = 0; a < D.dim; ++a) {
        if (D.n[a] < 2 || D.n[a] > 4096) return fail(INS_ERR_ARG, "n[a] must be in [2, 4096]");
        if (D.bc[a] != INS_PERIODIC && D.bc[a] != INS_WALL) return fail(INS_ERR_ARG, "bc must be PERIODIC or WALL");
        if (!D.face_coords[a]) return fail(INS_ERR_ARG, "face_coords[a] is null");
        if (!std::isfinite(D.force[a])) return fail(INS_ERR_ARG, "force must be finite");
    }
    for (int a = 0; a < D.dim; ++a) {
        const bool wall = D.bc[a] == INS_WALL;
        if (wall && a != 1) return fail(INS_ERR_UNSUPPORTED, "only y may be a wall direction");
    }
    const bool wall_y = D.bc[1] == INS_WALL;
    const long N = (long)D.n[0] * D.n[1] * (D.dim == 3 ? D.n[2] : 1);
    if (N > (1L << 31) - 1) return fail(INS_ERR_UNSUPPORTED, "more than 2^31 - 1 cells");

    ins_grid* g = new ins_grid();
    g->dim = D.dim;
    g->nx = D.n[0];
    g->ny = D.n[1];
    g->nz = D.dim == 3 ? D.n[2] : 1;
    g->wall_y = wall_y ? 1 : 0;
    g->dtype = D.dtype;
    g->scheme = D.scheme;
    g->nu = D.nu;
    for (int a = 0; a < 3; ++a) g->force[a] = a < D.dim ? D.force[a] : 0.0;
    g->stream = reinterpret_cast<cudaStream_t>(stream);
    g->N = N;
    g->nxh = g->nx / 2 + 1;
    g->hlo.assign(3, 1.0);
    const int n3[3] = {g->nx, g->ny, g->nz};
    auto bail = [&](ins_status s, const std::string& m) {
        if (g->base) cudaFree(g->base);
        delete g;
        return fail(s, m);
    };
    // geometry (host, FP64)
    double dmin = INFINITY;
    for (int a = 0; a < 3; ++a) {
        const int n = n3[a];
        if (a >= D.dim) {
            g->d[a].assign(n, 1.0);
            g->h[a].assign(n, 1.0);
            continue;
        }
        const double* f = D.face_coords[a];
        g->d[a].resize(n);
        for (int i = 0; i < n; ++i) {
            const double w = f[i + 1] - f[i];
            if (!(w > 0.0) || !std::isfinite(w)) return bail(INS_ERR_ARG, "face coordinates must increase strictly");
            g->d[a][i] = w;
            dmin = std::fmin(dmin, w);
        }
        const bool wall = D.bc[a] == INS_WALL;
        g->h[a].resize(n);
        for (int i = 0; i < n; ++i) {
            const double dn = (i + 1 < n) ? g->d[a][i + 1] : (wall ? g->d[a][n - 1] : g->d[a][0]);
            g->h[a][i] = 0.5 * (g->d[a][i] + dn);
        }
        g->hlo[a] = wall ? g->d[a][0] : 0.5 * (g->d[a][n - 1] + g->d[a][0]);
        if (wall) {
            // uniform wall-normal spacing with an FFT-friendly n: the DCT-II solve is available
            double mean = 0.0;
            for (double w : g->d[a]) mean += w;
            mean /= n;
            bool uni = n <= 2048;
            for (double w : g->d[a]) uni = uni && std::fabs(w - mean) <= 1e-10 * mean;
            std::vector<int> rad;
            if (uni && factor_radices(n, rad)) {
                g->wall_dct = 1;   // available; the Thomas solve stays the default (faster here)
                g->nst[a] = (int)rad.size();
                for (size_t s = 0; s < rad.size(); ++s) g->radix[a][s] = rad[s];
            }
        }
        if (!wall) {
            double mean = 0.0;
            for (double w : g->d[a]) mean += w;
            mean /= n;
            for (double w : g->d[a])
                if (std::fabs(w - mean) > 1e-10 * mean)
                    return bail(INS_ERR_UNSUPPORTED, "periodic directions must be uniformly spaced");
            std::vector<int> rad;
            if (n > 2048) return bail(INS_ERR_UNSUPPORTED, "periodic n must be <= 2048");
            if (!factor_radices(n, rad)) return bail(INS_ERR_UNSUPPORTED, "periodic n must be 2^p 3^q 5^r 7^s");
            g->nst[a] = (int)rad.size();
            for (size_t s = 0; s < rad.size(); ++s) g->radix[a][s] = rad[s];
        }
    }
    g->dmin2_nu = g->nu > 0.0 ? dmin * dmin / g->nu : INFINITY;

    const size_t ts = D.dtype == INS_F64 ? 8 : 4;
    const int dim = g->dim;
    const long nxh = g->nxh;
    const long spec = nxh * g->ny * g->nz;
    const long ncol = (long)g->nz * nxh;
    // layout of the single allocation
    std::vector<size_t> sizes;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t off = 0;
    size_t o_coef, o_geo, o_one, o_tw[3], o_scale = 0, o_lam, o_thlo = 0, o_thinv = 0, o_thcp = 0, o_thd = 0, o_F, o_acc,
                                             o_us, o_rp, o_S, o_cfl, o_err, o_diag, o_dmax;
    const size_t nsum = (size_t)g->nx + g->ny + g->nz;
    o_coef = off; off += al((size_t)C_COUNT * nsum * ts);
    const size_t o_ycoef = off; off += al((size_t)CY_COUNT * g->ny * ts);
    // double-float copy of the coefficients: the double-float pullback of an FP64 channel
    const bool coef_df = D.dtype == INS_F64 && wall_y && dim == 3;
    const size_t o_coefdf = off; off += coef_df ? al((size_t)C_COUNT * nsum * 8) : 0;
    o_geo = off; off += al(2 * nsum * 8);
    o_one = off; off += al(8);
    for (int a = 0; a < 3; ++a) {
        o_tw[a] = off;
        off += al((size_t)n3[a] * 2 * ts);
    }
    o_lam = off; off += al(nsum * 8);
    const size_t o_qw = off; off += g->wall_dct ? al((size_t)g->ny * 2 * ts) : 0;
    // FP32 periodic: [columns of the fused pass | its line | 1/N] (3-D: ny nxh | nz; 2-D: nxh | ny)
    const size_t neig = (!wall_y && D.dtype == INS_F32) ? (size_t)(dim == 3 ? g->ny * nxh + g->nz : nxh + g->ny) + 1 : 0;
    const size_t o_eig = off; off += al(neig * 4);
    // double-float FP64 step: FP64 periodic grids and 3-D channels (walls in y: the wall-normal
    // direction is solved by the Thomas sweep), x even for the two-cell update; the periodic FFT
    // lengths run the register kernels where they have them, else the Stockham kernels
    const bool df_ok = D.dtype == INS_F64 && (!wall_y || dim == 3) && g->nx % 2 == 0;
    size_t o_twdf[3] = {0, 0, 0}, o_scdf = 0;
    if (df_ok) {
        for (int a = 0; a < 3; ++a) {
            o_twdf[a] = off;
            off += al((size_t)n3[a] * 16);
        }
        if (!wall_y) {
            o_scdf = off;
            off += al((size_t)spec * 8);
        }
    }
    if (!wall_y) {
        o_scale = off; off += al((size_t)spec * ts);
    } else {
        o_thlo = off; off += al((size_t)g->ny * 2 * 8);
        o_thinv = off; off += al((size_t)g->ny * ncol * 8);
        o_thcp = off; off += al((size_t)g->ny * ncol * 8);
        o_thd = off; off += al((size_t)g->ny * ncol * 16);
    }
    o_F = off; off += al((size_t)dim * N * ts);
    o_acc = off; off += al((size_t)dim * N * ts);
    o_us = off; off += D.scheme == INS_RK4 ? al((size_t)dim * N * ts) : 0;   // the low-storage scheme needs no stage state
    o_rp = off; off += al((size_t)N * ts);
    const bool fused_rk = D.dtype == INS_F32 && dim == 3 && D.scheme == INS_RK4;
    const size_t o_pbuf = off; off += fused_rk ? al((size_t)N * ts) : 0;
    o_S = off; off += al((size_t)spec * 2 * ts);
    o_cfl = off; off += al(nsum * 8);
    o_err = off; off += al(4);
    o_diag = off; off += al(4 * 8);
    o_dmax = off; off += al(2 * 8);
    g->bytes = off;
    cudaError_t e = cudaMalloc(&g->base, off);
    if (e != cudaSuccess) {
        g->base = nullptr;
        cudaGetLastError();
        return bail(INS_ERR_OOM, std::string("workspace allocation failed: ") + cudaGetErrorString(e));
    }
    char* b = reinterpret_cast<char*>(g->base);
    g->coef = b + o_coef;
    g->ycoef = b + o_ycoef;
    g->coef_df = coef_df ? b + o_coefdf : nullptr;
    g->geo64 = reinterpret_cast<double*>(b + o_geo);
    g->one = reinterpret_cast<double*>(b + o_one);
    for (int a = 0; a < 3; ++a) g->tw[a] = b + o_tw[a];
    g->lam = reinterpret_cast<double*>(b + o_lam);
    g->dct_qw = g->wall_dct ? b + o_qw : nullptr;
    g->eig = neig ? reinterpret_cast<float*>(b + o_eig) : nullptr;
    g->df_ok = g->use_df = df_ok ? 1 : 0;
    if (df_ok) {
        for (int a = 0; a < 3; ++a) g->tw_df[a] = b + o_twdf[a];
        g->scale_df = wall_y ? nullptr : b + o_scdf;
    }
    if (!wall_y) {
        g->scale = b + o_scale;
    } else {
        g->th_lo = reinterpret_cast<double*>(b + o_thlo);
        g->th_up = g->th_lo + g->ny;
        g->th_invm = reinterpret_cast<double*>(b + o_thinv);
        g->th_cp = reinterpret_cast<double*>(b + o_thcp);
        g->th_d = b + o_thd;
    }
    g->F = b + o_F;
    g->acc = b + o_acc;
    g->us = D.scheme == INS_RK4 ? b + o_us : nullptr;
    g->pbuf = fused_rk ? b + o_pbuf : nullptr;
    g->rp = b + o_rp;
    g->S = b + o_S;
    g->cfl_max = reinterpret_cast<unsigned long long*>(b + o_cfl);
    g->err_flag = reinterpret_cast<unsigned int*>(b + o_err);
    g->diag = reinterpret_cast<double*>(b + o_diag);
    g->diag_max = reinterpret_cast<unsigned long long*>(b + o_dmax);

    auto up = [&](void* dst, const void* src, size_t n) -> bool {
        return cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    // coefficients
    bool ok = true;
    if (D.dtype == INS_F64) {
        std::vector<double> c;
        fill_coefs<double>(g, c);
        ok &= up(g->coef, c.data(), c.size() * 8);
        if (g->coef_df) {
            std::vector<float> cd(2 * c.size());
            for (size_t q = 0; q < c.size(); ++q) {
                cd[2 * q] = (float)c[q];
                cd[2 * q + 1] = (float)(c[q] - (double)cd[2 * q]);
            }
            ok &= up(g->coef_df, cd.data(), cd.size() * 4);
        }
    } else {
        std::vector<float> c;
        fill_coefs<float>(g, c);
        ok &= up(g->coef, c.data(), c.size() * 4);
    }
    {
        // per-row coefficients of y (used by k_rhs_div when y is a wall direction)
        const int ny = g->ny;
        const auto& d = g->d[1];
        const auto& h = g->h[1];
        std::vector<double> yc((size_t)CY_COUNT * ny);
        for (int j = 0; j < ny; ++j) {
            const double dn = (j + 1 < ny) ? d[j + 1] : (wall_y ? d[ny - 1] : d[0]);
            const double hp = (j > 0) ? h[j - 1] : g->hlo[1];
            yc[CY_F * ny + j] = 0.25 / d[j];
            yc[CY_S * ny + j] = 0.25 / h[j];
            yc[CY_WL * ny + j] = d[j] / (d[j] + dn);
            yc[CY_WR * ny + j] = dn / (d[j] + dn);
            yc[CY_AP * ny + j] = g->nu / (dn * h[j]);
            yc[CY_AM * ny + j] = g->nu / (d[j] * h[j]);
            yc[CY_BP * ny + j] = g->nu / (h[j] * d[j]);
            yc[CY_BM * ny + j] = g->nu / (hp * d[j]);
            yc[CY_I * ny + j] = 1.0 / d[j];
        }
        if (D.dtype == INS_F64) {
            ok &= up(g->ycoef, yc.data(), yc.size() * 8);
        } else {
            std::vector<float> yf(yc.begin(), yc.end());
            ok &= up(g->ycoef, yf.data(), yf.size() * 4);
        }
    }
    {
        std::vector<double> geo(2 * nsum);
        size_t o = 0;
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < n3[a]; ++i) geo[o++] = g->h[a][i];
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < n3[a]; ++i) geo[o++] = g->d[a][i];
        ok &= up(g->geo64, geo.data(), geo.size() * 8);
        const double one = 1.0;
        ok &= up(g->one, &one, 8);
    }
    if (!ok) return bail(INS_ERR_CUDA, "geometry upload failed");
    for (int a = 0; a < dim; ++a) {
        if (a == 1 && wall_y && !g->wall_dct) continue;
        ins_status s = D.dtype == INS_F64 ? upload_twiddles<double>(g, a, g->tw[a], n3[a])
                                          : upload_twiddles<float>(g, a, g->tw[a], n3[a]);
        if (s == INS_OK && df_ok) {
            // exp(-2 pi i m / L) as double-float pairs (re.hi, re.lo, im.hi, im.lo)
            std::vector<float> tw(4 * (size_t)n3[a]);
            for (int m = 0; m < n3[a]; ++m) {
                const double ang = 2.0 * M_PI * (double)m / (double)n3[a];
                const df re(std::cos(ang)), im(-std::sin(ang));
                tw[4 * m] = re.hi;
                tw[4 * m + 1] = re.lo;
                tw[4 * m + 2] = im.hi;
                tw[4 * m + 3] = im.lo;
            }
            if (!up(g->tw_df[a], tw.data(), tw.size() * 4)) s = fail(INS_ERR_CUDA, "twiddle upload failed");
        }
        if (s != INS_OK) {
            std::string m = g_err;
            return bail(s, m);
        }
    }
    // eigenvalues of D G along periodic directions: -4 sin^2(pi k/n) / (d h)
    {
        std::vector<double> lam(nsum, 0.0);
        size_t o = 0;
        for (int a = 0; a < 3; ++a) {
            const int n = n3[a];
            const bool per = a < dim && !(a == 1 && wall_y);
            const bool dct = a == 1 && g->wall_dct;
            for (int k = 0; k < n; ++k) {
                double v = 0.0;
                if (per) {
                    const double s = std::sin(M_PI * (double)k / (double)n);
                    v = -4.0 * s * s / (g->d[a][0] * g->h[a][0]);
                } else if (dct) {   // Neumann rows, uniform spacing: DCT-II eigenvalues
                    const double s = std::sin(M_PI * (double)k / (2.0 * n));
                    v = -4.0 * s * s / (g->d[a][0] * g->d[a][0]);
                }
                lam[o++] = v;
            }
        }
        ok &= up(g->lam, lam.data(), lam.size() * 8);
        if (g->eig) {
            // the fused forward/scale/inverse pass runs along z (3-D) or y (2-D); its column c is
            // (kx, ky) = (c % nxh, c / nxh) in 3-D and kx = c in 2-D
            const double ntot = (double)N;
            const double* lx = lam.data();
            const double* ly = lam.data() + g->nx;
            const double* lz = lam.data() + g->nx + g->ny;
            std::vector<float> ev;
            if (dim == 3) {
                for (int j = 0; j < g->ny; ++j)
                    for (long i = 0; i < nxh; ++i) ev.push_back((float)(ntot * (lx[i] + ly[j])));
                for (int k = 0; k < g->nz; ++k) ev.push_back((float)(ntot * lz[k]));
            } else {
                for (long i = 0; i < nxh; ++i) ev.push_back((float)(ntot * lx[i]));
                for (int j = 0; j < g->ny; ++j) ev.push_back((float)(ntot * ly[j]));
            }
            ev.push_back((float)(1.0 / ntot));   // the mean mode's factor (as in the table)
            ok &= up(g->eig, ev.data(), ev.size() * 4);
        }
        if (!wall_y) {
            const double ntot = (double)N;
            if (D.dtype == INS_F64)
                k_make_scale<double><<<1024, 256>>>(reinterpret_cast<double*>(g->scale), g->lam, g->lam + g->nx,
                                                    g->lam + g->nx + g->ny, (int)nxh, g->ny, g->nz, ntot);
            else
                k_make_scale<float><<<1024, 256>>>(reinterpret_cast<float*>(g->scale), g->lam, g->lam + g->nx,
                                                   g->lam + g->nx + g->ny, (int)nxh, g->ny, g->nz, ntot);
            if (df_ok)
                k_make_scale<df><<<1024, 256>>>(reinterpret_cast<df*>(g->scale_df), g->lam, g->lam + g->nx,
                                                g->lam + g->nx + g->ny, (int)nxh, g->ny, g->nz, ntot);
            if (cudaGetLastError() != cudaSuccess) return bail(INS_ERR_CUDA, "scale table kernel failed");
        } else {
            // Thomas factors per (kx, kz) mode, FP64, constant in time
            const int ny = g->ny;
            const auto& d = g->d[1];
            const auto& h = g->h[1];
            std::vector<double> lo(ny, 0.0), upc(ny, 0.0);
            for (int j = 1; j < ny; ++j) lo[j] = 1.0 / (d[j] * h[j - 1]);
            for (int j = 0; j + 1 < ny; ++j) upc[j] = 1.0 / (d[j] * h[j]);
            // twisted factorisation meeting at row mid = ny / 2 (see k_thomas2): top rows eliminated
            // downwards, bottom rows upwards, the middle row's pivot from both; the inverse FFTs'
            // normalisation sn folded in (f * sn, lo / sn, up / sn)
            std::vector<double> invm((size_t)ny * ncol), cp((size_t)ny * ncol);
            const int mid = ny / 2;
            const double sn = 1.0 / ((double)g->nx * (dim == 3 ? g->nz : 1));
            for (long col = 0; col < ncol; ++col) {
                const int kx = (int)(col % nxh), kz = (int)(col / nxh);
                const double lamxz = lam[kx] + (dim == 3 ? lam[g->nx + g->ny + kz] : 0.0);
                auto diag = [&](int j) { return (col == 0 && j == 0) ? 1.0 : -lo[j] - upc[j] + lamxz; };
                auto upr = [&](int j) { return (col == 0 && j == 0) ? 0.0 : upc[j]; };
                double gtop = 0.0;   // g_{j-1} of the downward sweep
                for (int j = 0; j < mid; ++j) {
                    const double piv = diag(j) - lo[j] * gtop;
                    gtop = upr(j) / piv;
                    invm[(size_t)j * ncol + col] = sn / piv;
                    cp[(size_t)j * ncol + col] = gtop;
                }
                double gbot = 0.0;   // g_{j+1} of the upward sweep
                for (int j = ny - 1; j > mid; --j) {
                    const double piv = diag(j) - upr(j) * gbot;
                    gbot = lo[j] / piv;
                    invm[(size_t)j * ncol + col] = sn / piv;
                    cp[(size_t)j * ncol + col] = gbot;
                }
                invm[(size_t)mid * ncol + col] = sn / (diag(mid) - lo[mid] * gtop - upr(mid) * gbot);
                cp[(size_t)mid * ncol + col] = 0.0;
            }
            if (g->wall_dct) {
                std::vector<double> qw(2 * (size_t)ny);
                for (int k = 0; k < ny; ++k) {
                    qw[2 * k] = std::cos(M_PI * k / (2.0 * ny));
                    qw[2 * k + 1] = -std::sin(M_PI * k / (2.0 * ny));
                }
                if (D.dtype == INS_F64) {
                    ok &= up(g->dct_qw, qw.data(), qw.size() * 8);
                } else {
                    std::vector<float> qf(qw.begin(), qw.end());
                    ok &= up(g->dct_qw, qf.data(), qf.size() * 4);
                }
            }
            std::vector<double> los(ny), ups(ny);
            for (int j = 0; j < ny; ++j) {
                los[j] = lo[j] / sn;
                ups[j] = upc[j] / sn;
            }
            if (D.dtype == INS_F32) {
                // FP32 spectra are solved in double-float arithmetic: the tables go to the device as
                // (hi, lo) float pairs in the same 8 bytes, so the sweeps need no FP64 -> double-float split
                auto to_df = [](std::vector<double>& v) {
                    for (double& x : v) {
                        const float hi = (float)x, lo = (float)(x - (double)hi);
                        float pr[2] = {hi, lo};
                        std::memcpy(&x, pr, 8);
                    }
                };
                to_df(los);
                to_df(ups);
                to_df(invm);
                to_df(cp);
            }
            ok &= up(g->th_lo, los.data(), (size_t)ny * 8);
            ok &= up(g->th_up, ups.data(), (size_t)ny * 8);
            ok &= up(g->th_invm, invm.data(), invm.size() * 8);
            ok &= up(g->th_cp, cp.data(), cp.size() * 8);
        }
    }
    if (!ok) return bail(INS_ERR_CUDA, "table upload failed");
    if (cudaMemset(g->cfl_max, 0, nsum * 8) != cudaSuccess || cudaMemset(g->err_flag, 0, 4) != cudaSuccess)
        return bail(INS_ERR_CUDA, "memset failed");
    ins_status s = D.dtype == INS_F64 ? set_smem_attrs<double>() : set_smem_attrs<float>();
    if (s != INS_OK) {
        std::string m = g_err;
        return bail(s, m);
    }
    if (D.dtype == INS_F64) {
        g->lg_tw_x = choose_lgtw<double>(g->nx);
        g->lg_tw_y = choose_lgtw<double>(g->ny);
        g->lg_tw_z = choose_lgtw<double>(g->nz);
    } else {
        g->lg_tw_x = choose_lgtw<float>(g->nx);
        g->lg_tw_y = choose_lgtw<float>(g->ny);
        g->lg_tw_z = choose_lgtw<float>(g->nz);
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bail(INS_ERR_CUDA, std::string("grid setup failed: ") + cudaGetErrorString(e));
    *out = g;
    return INS_OK;
}

ins_status ins_grid_destroy(ins_grid* g) {
    if (!g) return INS_OK;
    cudaStreamSynchronize(g->stream);
    if (g->step_exec) cudaGraphExecDestroy(g->step_exec);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->vjp) cudaFree(g->vjp);
    if (g->mbuf) cudaFree(g->mbuf);
    if (g->eddy_buf) cudaFree(g->eddy_buf);
    if (g->eddy_rows) cudaFree(g->eddy_rows);
    cudaError_t e = cudaFree(g->base);
    delete g;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree");
    return INS_OK;
}

ins_status ins_set_stream(ins_grid* g, void* stream) {
    if (!g) return fail(INS_ERR_ARG, "null grid");
    g->stream = reinterpret_cast<cudaStream_t>(stream);
    return INS_OK;
}

ins_status ins_set_f64_arithmetic(ins_grid* g, int mode) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    if (mode != INS_ARITH_NATIVE && mode != INS_ARITH_DOUBLE_FLOAT) return fail(INS_ERR_ARG, "unknown arithmetic mode");
    if (mode == INS_ARITH_DOUBLE_FLOAT && !g->df_ok)
        return fail(INS_ERR_UNSUPPORTED,
                    "double-float arithmetic needs an FP64 grid, periodic or a 3-D channel with walls in y, with "
                    "even nx");
    g->use_df = mode == INS_ARITH_DOUBLE_FLOAT ? 1 : 0;
    return INS_OK;
}

ins_status ins_get_f64_arithmetic(const ins_grid* g, int* mode) {
    if (!g || !mode) return fail(INS_ERR_ARG, "null argument");
    *mode = g->use_df ? INS_ARITH_DOUBLE_FLOAT : INS_ARITH_NATIVE;
    return INS_OK;
}

ins_status ins_workspace_bytes(const ins_grid* g, size_t* bytes) {
    if (!g || !bytes) return fail(INS_ERR_ARG, "null argument");
    *bytes = g->bytes;
    return INS_OK;
}

ins_status ins_spectrum(ins_grid* g, const void* u, double* E_dev, int kmax) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    CHECK(check_ptr(g, u, "u"));
    if (!E_dev) return fail(INS_ERR_ARG, "E_dev is null");
    if (kmax < 0 || kmax > 4096) return fail(INS_ERR_ARG, "kmax must be in [0, 4096]");
    if (g->wall_y) return fail(INS_ERR_UNSUPPORTED, "ins_spectrum: periodic grids only");
    return dispatch_dtype(g, [&](auto z) {
        using T = decltype(z);
        return dispatch<T>(g, [&](auto impl) { return decltype(impl)::spectrum(g, (const T*)u, E_dev, kmax); });
    });
}

ins_status ins_wall_profiles(ins_grid* g, const void* u, double* out_dev) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    CHECK(check_ptr(g, u, "u"));
    if (!out_dev) return fail(INS_ERR_ARG, "out_dev is null");
    if (!g->wall_y || g->dim != 3) return fail(INS_ERR_UNSUPPORTED, "ins_wall_profiles: 3-D grids with a wall in y");
    if (g->dtype == INS_F64)
        KLAUNCH(g, "wall_profiles", k_wall_profiles<double><<<g->ny, 256, 0, g->stream>>>((const double*)u, g->nx, g->ny, g->nz, out_dev));
    else
        KLAUNCH(g, "wall_profiles", k_wall_profiles<float><<<g->ny, 256, 0, g->stream>>>((const float*)u, g->nx, g->ny, g->nz, out_dev));
    return INS_OK;
}

ins_status ins_filter_face_average(int dim, const int n_coarse[3], int ratio, int dtype, const void* u_fine,
                                   void* u_coarse, void* stream) {
    g_err.clear();
    if (!n_coarse || !u_fine || !u_coarse) return fail(INS_ERR_ARG, "null argument");
    if (dim != 2 && dim != 3) return fail(INS_ERR_ARG, "dim must be 2 or 3");
    if (ratio < 1 || ratio > 64) return fail(INS_ERR_ARG, "ratio must be in [1, 64]");
    if (dtype != INS_F32 && dtype != INS_F64) return fail(INS_ERR_ARG, "bad dtype");
    const int cx = n_coarse[0], cy = n_coarse[1], cz = dim == 3 ? n_coarse[2] : 1;
    if (cx < 1 || cy < 1 || cz < 1) return fail(INS_ERR_ARG, "coarse sizes must be >= 1");
    const long total = (long)dim * cx * cy * cz;
    if ((long)cx * ratio * cy * ratio * (dim == 3 ? (long)cz * ratio : 1) > (1L << 31))
        return fail(INS_ERR_UNSUPPORTED, "fine grid above 2^31 cells");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (dtype == INS_F64) {
        if (dim == 3) k_filter_face<double, 3><<<blocks, 256, 0, st>>>((const double*)u_fine, (double*)u_coarse, cx, cy, cz, ratio);
        else k_filter_face<double, 2><<<blocks, 256, 0, st>>>((const double*)u_fine, (double*)u_coarse, cx, cy, cz, ratio);
    } else {
        if (dim == 3) k_filter_face<float, 3><<<blocks, 256, 0, st>>>((const float*)u_fine, (float*)u_coarse, cx, cy, cz, ratio);
        else k_filter_face<float, 2><<<blocks, 256, 0, st>>>((const float*)u_fine, (float*)u_coarse, cx, cy, cz, ratio);
    }
    INS_LAUNCHED("filter_face");
    return INS_OK;
}

ins_status ins_cfl_dt(ins_grid* g, const void* u, double cfl, double* dt_dev) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    CHECK(check_ptr(g, u, "u"));
    if (!dt_dev) return fail(INS_ERR_ARG, "dt_dev is null");
    if (!(std::isfinite(cfl) && cfl > 0.0)) return fail(INS_ERR_ARG, "cfl must be finite and > 0");
    return dispatch_dtype(g, [&](auto z) {
        using T = decltype(z);
        return dispatch<T>(g, [&](auto impl) { return decltype(impl)::cfl(g, (const T*)u, cfl, dt_dev); });
    });
}

ins_status ins_diag(ins_grid* g, const void* u, double out[4]) {
    g_err.clear();
    if (!g || !out) return fail(INS_ERR_ARG, "null argument");
    CHECK(check_ptr(g, u, "u"));
    return dispatch_dtype(g, [&](auto z) {
        using T = decltype(z);
        return dispatch<T>(g, [&](auto impl) { return decltype(impl)::diag(g, (const T*)u, out); });
    });
}

ins_status ins_check_finite(ins_grid* g) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    unsigned int f = 0;
    INS_CUDA(cudaMemcpyAsync(&f, g->err_flag, 4, cudaMemcpyDeviceToHost, g->stream));
    INS_CUDA(cudaStreamSynchronize(g->stream));
    if (f) {
        INS_CUDA(cudaMemsetAsync(g->err_flag, 0, 4, g->stream));
        INS_CUDA(cudaStreamSynchronize(g->stream));
        return fail(INS_ERR_NONFINITE, "a step produced a non-finite value");
    }
    return INS_OK;
}

ins_status ins_launch_count(const ins_grid* g, unsigned long long* n) {
    if (!g || !n) return fail(INS_ERR_ARG, "null argument");
    *n = g->launches;
    return INS_OK;
}

ins_status ins_profile_enable(ins_grid* g, int on) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    if (on && g->ev.empty()) {
        g->ev.resize(16384);
        for (auto& e : g->ev) INS_CUDA(cudaEventCreate(&e));
    }
    g->prof = on != 0;
    g->ev_used = 0;
    g->rec_name.clear();
    g->prof_dropped = 0;
    return INS_OK;
}

ins_status ins_profile_read(ins_grid* g, ins_kernel_stat* out, int cap, int* n_out) {
    g_err.clear();
    if (!g || !n_out || (cap > 0 && !out)) return fail(INS_ERR_ARG, "null argument");
    INS_CUDA(cudaStreamSynchronize(g->stream));
    std::vector<double> tot(g->names.size(), 0.0);
    std::vector<long long> cnt(g->names.size(), 0);
    for (size_t r = 0; r < g->rec_name.size(); ++r) {
        float ms = 0.f;
        INS_CUDA(cudaEventElapsedTime(&ms, g->ev[2 * r], g->ev[2 * r + 1]));
        tot[g->rec_name[r]] += ms;
        cnt[g->rec_name[r]] += 1;
    }
    int n = 0;
    for (size_t i = 0; i < g->names.size() && n < cap; ++i) {
        if (!cnt[i]) continue;
        std::memset(out[n].name, 0, sizeof(out[n].name));
        std::strncpy(out[n].name, g->names[i].c_str(), sizeof(out[n].name) - 1);
        out[n].launches = cnt[i];
        out[n].total_ms = tot[i];
        ++n;
    }
    *n_out = n;
    g->ev_used = 0;
    g->rec_name.clear();
    if (g->prof_dropped) {
        g->prof_dropped = 0;
        return fail(INS_ERR_ARG, "event pool exhausted: read the profile more often");
    }
    return INS_OK;
}

}  // extern "C"

namespace {
template <typename T, int CH>
__global__ void k_fma_rate(T* out, int iters, T a, T b) {
    T acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CH; ++c) acc[c] = fma(acc[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
ins_status fma_rate(void* stream, double* flops) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    INS_CUDA(cudaGetDevice(&dev));
    INS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    const int iters = sizeof(T) == 8 ? 4000 : 100000;
    T* out = nullptr;
    INS_CUDA(cudaMalloc(&out, (size_t)blocks * threads * sizeof(T)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_rate<T, 8><<<blocks, threads, 0, st>>>(out, 64, (T)1.0000001, (T)1e-9);
    cudaEventRecord(e0, st);
    k_fma_rate<T, 8><<<blocks, threads, 0, st>>>(out, iters, (T)1.0000001, (T)1e-9);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "fma rate");
    *flops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3);
    return INS_OK;
}
}  // namespace

extern "C" ins_status ins_measure_fma_rate(int dtype, void* stream, double* flops_per_s) {
    g_err.clear();
    if (!flops_per_s || (dtype != INS_F32 && dtype != INS_F64)) return fail(INS_ERR_ARG, "bad argument");
    return dtype == INS_F64 ? fma_rate<double>(stream, flops_per_s) : fma_rate<float>(stream, flops_per_s);
}

