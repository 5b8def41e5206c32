// Impl::step_vjp, step_vjp_wall: the pullback of one step (stage recompute from the step input,
// then the stages in reverse). Included by ins_vjp.cu.
#pragma once

#include "ins_internal.cuh"

namespace {

// Pullback of one RK4 step (uniform periodic grids): recompute the stage states from the
// checkpoint u_n, then run the stages in reverse (see ins.h, ins_step_vjp).
// Pullback of one step on a wall-bounded grid: stage recompute as below, P^T = M Omega P
// Omega^-1 M, J_F^T in gather form (k_adj_rhs_wall_g); the stored top wall faces of u^y are not
// unknowns (cotangents there are ignored and returned as 0).
template <typename T, int DIM, bool WALL>
ins_status Impl<T, DIM, WALL>::step_vjp_wall(ins_grid* g, const T* un, const double* dt_dev, double dt_host, const T* ybar, T* ubar, double* nubar) {
    if (3 * g->N >= (1L << 31)) return fail(INS_ERR_UNSUPPORTED, "ins_step_vjp: wall grids need 3 x cells < 2^31");
    static const double A[3] = {0.5, 0.5, 1.0};
    static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const long N = g->N;
    const size_t fld = (size_t)g->dim * N * sizeof(T);
    const size_t fa = (fld + 255) & ~size_t(255);
    const dim3 cg = cell_grid(g);
    const long nblk = (long)cg.x * cg.y * cg.z;
    const size_t need = 4 * fa + (size_t)nblk * 8;
    if (g->vjp_bytes < need) {
        if (g->vjp) cudaFree(g->vjp);
        g->vjp = nullptr;
        g->vjp_bytes = 0;
        cudaError_t e = cudaMalloc(&g->vjp, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(INS_ERR_OOM, std::string("step-VJP workspace: ") + cudaGetErrorString(e));
        }
        g->vjp_bytes = need;
    }
    char* vb = reinterpret_cast<char*>(g->vjp);
    T* U[4] = {const_cast<T*>(un), reinterpret_cast<T*>(vb), reinterpret_cast<T*>(vb + fa),
               reinterpret_cast<T*>(vb + 2 * fa)};
    T* W = reinterpret_cast<T*>(vb + 3 * fa);
    double* part = reinterpret_cast<double*>(vb + 4 * fa);
    T* F = reinterpret_cast<T*>(g->F);
    T* rp = reinterpret_cast<T*>(g->rp);
    T* scratch = reinterpret_cast<T*>(g->acc);
    const bool lowst = g->scheme == INS_WRAY3;
    const int nst = lowst ? 3 : 4;
    ins_status s;
    for (int st = 0; st < nst - 1; ++st) {
        if ((s = launch_rhs_div<T, DIM, WALL>(g, U[st], F, rp)) != INS_OK) return s;
        if ((s = poisson<T>(g, rp, rp)) != INS_OK) return s;
        RkArgs ra;
        ra.dt_dev = dt_dev;
        ra.dt_host = dt_host;
        ra.mx = nullptr;
        ra.err_flag = g->err_flag;
        ra.last = 0;
        if (lowst) {
            ra.a_next = WRAY3_GAMMA[st];
            ra.b = WRAY3_ZETA[st];
            ra.stage = st;
            if ((s = rk_update<true>(g, F, rp, U[st], scratch, U[st + 1], ra)) != INS_OK) return s;
        } else {
            ra.a_next = A[st];
            ra.b = 0.0;
            ra.stage = 0;   // us = u0 + dt a k only (no acc)
            if ((s = rk_update<false>(g, F, rp, U[0], nullptr, U[st + 1], ra)) != INS_OK) return s;
        }
    }
    const long n = (long)g->dim * N;
    const double* hy = g->geo64 + g->nx;
    const double* dy = g->geo64 + (g->nx + g->ny + g->nz) + g->nx;
    constexpr bool ZMARCH = DIM == 3 && std::is_same<T, float>::value;
    // FP32 3-D with vector rows: the last stage's cotangent dt b ybar is formed inside its P^T passes
    // and the first z march reads ybar as the accumulator's previous value (no copy, no scaled field)
    const double blast = lowst ? WRAY3_GAMMA[2] : B[3];
    const bool fold = ZMARCH && rk_vec_ok<T>(g, ybar) && reinterpret_cast<uintptr_t>(rp) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(W) % 16 == 0;
    if (!fold) {
        INS_CUDA(cudaMemcpyAsync(ubar, ybar, fld, cudaMemcpyDeviceToDevice, g->stream));
        KLAUNCH(g, "scale", k_scale_dt<T><<<1184, 256, 0, g->stream>>>(ybar, F, dt_dev, dt_host, blast, n));
    }
    // z chunks of the 3-D adjoint march: about two waves of two CTAs per SM
    const long cols = (long)cg.x * cg.y;
    const long nch = std::max(1L, std::min((long)g->nz, (4L * device_sm_count() + cols / 2) / cols));
    const int zkc = ZMARCH ? (int)((g->nz + nch - 1) / nch) : 1;
    const dim3 zg(cg.x, cg.y, ZMARCH ? (g->nz + zkc - 1) / zkc : 1);
    const long znblk = ZMARCH ? (long)zg.x * zg.y * zg.z : nblk;
    if constexpr (ZMARCH) {
        static bool attr = false;
        if (!attr) {
            INS_CUDA(cudaFuncSetAttribute(k_adj_rhs_wall_z<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          wall_adj_smem<T>()));
            INS_CUDA(cudaFuncSetAttribute(k_adj_rhs_wall_z<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          wall_adj_smem<T>()));
            attr = true;
        }
    }
    WallAdjG<T> wa;
    wa.g = make_geo<T>(g);
    wa.nu = (T)g->nu;
    wa.dt_dev = dt_dev;
    wa.dt_host = dt_host;
    for (int st = nst - 1; st >= 0; --st) {
        // w = P^T kbar = M Omega P (Omega^-1 M kbar)
        const bool first = fold && st == nst - 1;
        const T* uin = first ? ybar : ubar;   // the accumulator's previous value
        if (first) {
            constexpr int V = VecT<T>::N;
            if ((s = vec_width(g) == V ? div_scaled_vec<V, true>(g, ybar, rp, dt_dev, dt_host, blast)
                                       : div_scaled_vec<V / 2, true>(g, ybar, rp, dt_dev, dt_host, blast)) != INS_OK)
                return s;
            if ((s = poisson<T>(g, rp, rp)) != INS_OK) return s;
            if ((s = vec_width(g) == V ? sub_scaled_vec<V, true>(g, ybar, rp, W, hy, dy, dt_dev, dt_host, blast)
                                       : sub_scaled_vec<V / 2, true>(g, ybar, rp, W, hy, dy, dt_dev, dt_host, blast)) !=
                INS_OK)
                return s;
        } else {
            if ((s = div_scaled_fast(g, F, rp)) != INS_OK) return s;
            if ((s = poisson<T>(g, rp, rp)) != INS_OK) return s;
            if ((s = sub_scaled_fast(g, F, rp, W, hy, dy)) != INS_OK) return s;
        }
        if (lowst) {
            wa.bn = st > 0 ? WRAY3_GAMMA[st - 1] + WRAY3_ZETA[st] : 0.0;
            wa.an = st > 0 ? WRAY3_GAMMA[st - 1] : 0.0;
        } else {
            wa.bn = st > 0 ? B[st - 1] : 0.0;
            wa.an = st > 0 ? A[st - 1] : 0.0;
        }
        // ubar0 += J_F^T w; the next stage cotangent into F
        // FP32 3-D: the z march (shared-memory ring); FP64 and 2-D: neighbours from global memory
        // (in FP64 the march's register count leaves one CTA per SM, and the global form is faster)
        if constexpr (ZMARCH) {
            if (first) {
                KLAUNCH(g, "adj_rhs", (k_adj_rhs_wall_z<T, true><<<zg, dim3(32, 8), wall_adj_smem<T>(), g->stream>>>(
                                          wa, U[st], W, lowst ? nullptr : ybar, ubar, st > 0 ? F : nullptr, part, zkc, uin)));
            } else {
                KLAUNCH(g, "adj_rhs", (k_adj_rhs_wall_z<T><<<zg, dim3(32, 8), wall_adj_smem<T>(), g->stream>>>(
                                          wa, U[st], W, lowst ? nullptr : ybar, ubar, st > 0 ? F : nullptr, part, zkc, uin)));
            }
        } else
            KLAUNCH(g, "adj_rhs", (k_adj_rhs_wall_g<T, DIM><<<cg, dim3(32, 8), 0, g->stream>>>(
                                      wa, U[st], W, lowst ? nullptr : ybar, ubar, st > 0 ? F : nullptr, part)));
        if (nubar) KLAUNCH(g, "sum_partials", k_sum_partials<<<1, 256, 0, g->stream>>>(part, znblk, nubar));
    }
    KLAUNCH(g, "mask_top", k_mask_top<T><<<592, 256, 0, g->stream>>>(ubar, g->nx, g->ny, g->nz, N));
    return INS_OK;
}

// Pullback of one classic RK4 step of an FP64 3-D channel in double-float arithmetic (the
// counterpart of the double-float channel step): the stage states are recomputed by the
// double-float step kernels, P^T = M Omega P Omega^-1 M runs the row-scaled passes and the Poisson
// solve in double-float, and J_F^T (k_adj_rhs_wall_g<df, ...>) in double-float, while the state
// cotangent ubar accumulates in FP64 and the nu partials are reduced in FP64. The stored top wall
// faces of u^y are not unknowns (cotangents there are ignored and returned as 0).
inline ins_status step_vjp_wall_df(ins_grid* g, const double* un, const double* dt_dev, double dt_host,
                                   const double* ybar, double* ubar, double* nubar) {
    if (3 * g->N >= (1L << 31)) return fail(INS_ERR_UNSUPPORTED, "ins_step_vjp: wall grids need 3 x cells < 2^31");
    static const double A[3] = {0.5, 0.5, 1.0};
    static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const long N = g->N;
    const size_t fld = (size_t)3 * N * sizeof(double);
    const size_t fa = (fld + 255) & ~size_t(255);
    const dim3 cg = cell_grid(g);
    const long nblk = (long)cg.x * cg.y * cg.z;
    const size_t need = 4 * fa + (size_t)nblk * 8;
    if (g->vjp_bytes < need) {
        if (g->vjp) cudaFree(g->vjp);
        g->vjp = nullptr;
        g->vjp_bytes = 0;
        cudaError_t e = cudaMalloc(&g->vjp, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(INS_ERR_OOM, std::string("step-VJP workspace: ") + cudaGetErrorString(e));
        }
        g->vjp_bytes = need;
    }
    char* vb = reinterpret_cast<char*>(g->vjp);
    df* U[4] = {nullptr, reinterpret_cast<df*>(vb), reinterpret_cast<df*>(vb + fa), reinterpret_cast<df*>(vb + 2 * fa)};
    df* W = reinterpret_cast<df*>(vb + 3 * fa);
    double* part = reinterpret_cast<double*>(vb + 4 * fa);
    df* F = reinterpret_cast<df*>(g->F);
    df* rp = reinterpret_cast<df*>(g->rp);
    ins_status s;
    // stage states u_1 .. u_3 (u_{s+1} = u_n + dt a_s k_s, no accumulator)
    for (int st = 0; st < 3; ++st) {
        s = st == 0 ? launch_rhs_div_df<3, double, true>(g, un, F, rp) : launch_rhs_div_df<3, df, true>(g, U[st], F, rp);
        if (s != INS_OK) return s;
        if ((s = poisson<df>(g, rp, rp)) != INS_OK) return s;
        RkArgs ra;
        ra.dt_dev = dt_dev;
        ra.dt_host = dt_host;
        ra.mx = nullptr;
        ra.err_flag = g->err_flag;
        ra.last = 0;
        ra.a_next = A[st];
        ra.b = 0.0;
        ra.stage = 0;
        if ((s = rk_update_df<3, false, true>(g, F, rp, const_cast<double*>(un), nullptr, U[st + 1], ra)) != INS_OK)
            return s;
    }
    const long n = 3 * N;
    const double* hy = g->geo64 + g->nx;
    const double* dy = g->geo64 + (g->nx + g->ny + g->nz) + g->nx;
    INS_CUDA(cudaMemcpyAsync(ubar, ybar, fld, cudaMemcpyDeviceToDevice, g->stream));
    KLAUNCH(g, "scale", (k_scale_dt<df, double><<<1184, 256, 0, g->stream>>>(ybar, F, dt_dev, dt_host, B[3], n)));
    const Geo<df> geo = make_geo<df>(g);
    // the adjoint stencil as a z march (shared-memory ring of u and w), about two waves of two CTAs
    // per SM; the chunk from the wave count
    const long cols = (long)cg.x * cg.y;
    const long nch = std::max(1L, std::min((long)g->nz, (4L * device_sm_count() + cols / 2) / cols));
    const int zkc = (int)((g->nz + nch - 1) / nch);
    const dim3 zg(cg.x, cg.y, (g->nz + zkc - 1) / zkc);
    const long znblk = (long)zg.x * zg.y * zg.z;
    {
        static bool attr[64] = {};
        int dev = 0;
        INS_CUDA(cudaGetDevice(&dev));
        if (dev >= 0 && dev < 64 && !attr[dev]) {
            INS_CUDA(cudaFuncSetAttribute(k_adj_rhs_wall_z<df, false, double, double>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, wall_adj_smem<df>()));
            INS_CUDA(cudaFuncSetAttribute(k_adj_rhs_wall_z<df, false, df, double>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, wall_adj_smem<df>()));
            attr[dev] = true;
        }
    }
    WallAdjG<df> wa;
    wa.g = geo;
    wa.nu = df(g->nu);
    wa.dt_dev = dt_dev;
    wa.dt_host = dt_host;
    for (int st = 3; st >= 0; --st) {
        // w = P^T kbar = M Omega P (Omega^-1 M kbar)
        KLAUNCH(g, "divergence", (k_wall_div_scaled<df, 3><<<cg, dim3(32, 8), 0, g->stream>>>(geo, F, rp)));
        if ((s = poisson<df>(g, rp, rp)) != INS_OK) return s;
        KLAUNCH(g, "sub_grad", (k_wall_sub_scaled<df, 3><<<cg, dim3(32, 8), 0, g->stream>>>(geo, F, rp, W, hy, dy)));
        wa.bn = st > 0 ? B[st - 1] : 0.0;
        wa.an = st > 0 ? A[st - 1] : 0.0;
        // ubar += J_F^T w (FP64 accumulation); the next stage cotangent into F
        if (st == 0)
            KLAUNCH(g, "adj_rhs", (k_adj_rhs_wall_z<df, false, double, double><<<zg, dim3(32, 8), wall_adj_smem<df>(),
                                                                              g->stream>>>(
                                      wa, un, W, ybar, ubar, nullptr, part, zkc, nullptr)));
        else
            KLAUNCH(g, "adj_rhs", (k_adj_rhs_wall_z<df, false, df, double><<<zg, dim3(32, 8), wall_adj_smem<df>(),
                                                                          g->stream>>>(
                                      wa, U[st], W, ybar, ubar, F, part, zkc, nullptr)));
        if (nubar) KLAUNCH(g, "sum_partials", k_sum_partials<<<1, 256, 0, g->stream>>>(part, znblk, nubar));
    }
    KLAUNCH(g, "mask_top", k_mask_top<double><<<592, 256, 0, g->stream>>>(ubar, g->nx, g->ny, g->nz, N));
    return INS_OK;
}

// Pullback of one step (classic RK4 or Wray's low-storage RK3) of an FP64 periodic 3-D grid in
// double-float arithmetic (the counterpart of the double-float step, ins_set_f64_arithmetic): the
// stage states are recomputed by the double-float step kernels, P^T = P runs the double-float Poisson
// passes, and the adjoint stencil evaluates J_F^T in double-float while the state cotangent ubar
// accumulates in FP64 (each stage's increment added in FP64) and the nu partials are reduced in FP64.
inline ins_status step_vjp_df(ins_grid* g, const double* un, const double* dt_dev, double dt_host,
                              const double* ybar, double* ubar, double* nubar) {
    static const double A[3] = {0.5, 0.5, 1.0};
    static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const bool lowst = g->scheme == INS_WRAY3;
    const int nst = lowst ? 3 : 4;
    const long N = g->N;
    const size_t fld = (size_t)3 * N * sizeof(double);
    const int abx = (g->nx + AJX - 1) / AJX, aby = (g->ny + AJY - 1) / AJY;
    const size_t adj_smem = 4 * 6 * AJSP * sizeof(df);
    static int per_sm = 0;
    INS_CUDA(cudaFuncSetAttribute(k_adj_rhs_z<df, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)adj_smem));
    INS_CUDA(cudaFuncSetAttribute(k_adj_rhs_z<df, df, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)adj_smem));
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_rhs_z<df, df, double>, AJX * AJY, adj_smem);
        if (per_sm < 1) per_sm = 1;
    }
    const int akc = wave_chunk((long)abx * aby, g->nz, (long)per_sm * device_sm_count(), 2);
    const dim3 ag(abx, aby, (g->nz + akc - 1) / akc);
    const long nblk = (long)ag.x * ag.y * ag.z;
    const size_t fa = (fld + 255) & ~size_t(255);
    const size_t need = 5 * fa + (size_t)nblk * 8;
    if (g->vjp_bytes < need) {
        if (g->vjp) cudaFree(g->vjp);
        g->vjp = nullptr;
        g->vjp_bytes = 0;
        cudaError_t e = cudaMalloc(&g->vjp, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(INS_ERR_OOM, std::string("step-VJP workspace: ") + cudaGetErrorString(e));
        }
        g->vjp_bytes = need;
    }
    // stage states: RK4 keeps u_2 .. u_4 as double-float pairs (u_s = u_n + dt a k_{s-1}); Wray's
    // low-storage states chain (u_{s+1} = u_s + dt (gamma k_s + zeta k_{s-1})) and stay FP64
    char* vb = reinterpret_cast<char*>(g->vjp);
    df* U[4] = {nullptr, reinterpret_cast<df*>(vb), reinterpret_cast<df*>(vb + fa), reinterpret_cast<df*>(vb + 2 * fa)};
    double* U64[3] = {const_cast<double*>(un), reinterpret_cast<double*>(vb), reinterpret_cast<double*>(vb + fa)};
    df* W = reinterpret_cast<df*>(vb + 3 * fa);
    double* part = reinterpret_cast<double*>(vb + 5 * fa);
    df* F = reinterpret_cast<df*>(g->F);
    df* rp = reinterpret_cast<df*>(g->rp);
    df* kprev = reinterpret_cast<df*>(g->acc);
    ins_status s;
    auto args = [&](double a_next, double b, int stage) {
        RkArgs ra;
        ra.dt_dev = dt_dev;
        ra.dt_host = dt_host;
        ra.a_next = a_next;
        ra.b = b;
        ra.stage = stage;
        ra.last = 0;
        ra.mx = nullptr;
        ra.err_flag = g->err_flag;
        return ra;
    };
    if (lowst) {
        for (int st = 0; st < 2; ++st) {
            if ((s = launch_rhs_div_df<3, double>(g, U64[st], F, rp)) != INS_OK) return s;
            if ((s = poisson<df>(g, rp, rp)) != INS_OK) return s;
            if ((s = rk_update_df<3, true>(g, F, rp, U64[st], kprev, nullptr, args(WRAY3_GAMMA[st], WRAY3_ZETA[st], st),
                                           U64[st + 1])) != INS_OK)
                return s;
        }
    } else {
        // the stage states u_{s+1} = u_n + dt a_{s+1,s} k_s (stage 0 of the update without an
        // accumulator writes only the stage state)
        for (int st = 0; st < 3; ++st) {
            s = st == 0 ? launch_rhs_div_df<3, double>(g, un, F, rp) : launch_rhs_div_df<3, df>(g, U[st], F, rp);
            if (s != INS_OK) return s;
            if ((s = poisson<df>(g, rp, rp)) != INS_OK) return s;
            if ((s = rk_update_df<3>(g, F, rp, const_cast<double*>(un), nullptr, U[st + 1], args(A[st], 0.0, 0))) !=
                INS_OK)
                return s;
        }
    }
    // reverse: ubar starts as ybar; the last stage's cotangent dt b_last ybar
    const double blast = lowst ? WRAY3_GAMMA[2] : B[3];
    INS_CUDA(cudaMemcpyAsync(ubar, ybar, fld, cudaMemcpyDeviceToDevice, g->stream));
    KLAUNCH(g, "scale", (k_scale_dt<df, double><<<1184, 256, 0, g->stream>>>(ybar, F, dt_dev, dt_host, blast, 3 * N)));
    AdjCoef<df> ac;
    ac.nx = g->nx;
    ac.ny = g->ny;
    ac.nz = g->nz;
    for (int a = 0; a < 3; ++a) {
        const double D = g->d[a][0];
        ac.c1[a] = df(0.5 / D);
        ac.c2[a] = df(0.25 / D);
        ac.l2[a] = df(1.0 / (D * D));
    }
    ac.nu = df(g->nu);
    ac.dt_dev = dt_dev;
    ac.dt_host = dt_host;
    const df idx(1.0 / g->d[0][0]), idy(1.0 / g->d[1][0]), idz(1.0 / g->d[2][0]);
    for (int st = nst - 1; st >= 0; --st) {
        // w = P kbar_s (P is symmetric on a uniform periodic grid)
        KLAUNCH(g, "divergence", (k_div_df<3><<<4 * device_sm_count(), 256, 0, g->stream>>>(g->nx, g->ny, g->nz, idx, idy,
                                                                                          idz, F, rp)));
        if ((s = poisson<df>(g, rp, rp)) != INS_OK) return s;
        if ((s = rk_update_df<3>(g, F, rp, nullptr, nullptr, W, args(0.0, 0.0, -1))) != INS_OK) return s;
        if (lowst) {
            // kbar_{s-1} = dt gamma_{s-1} (Ubar_{s+1} + ubar_s) + dt zeta_s Ubar_{s+1}
            ac.bn = st > 0 ? WRAY3_GAMMA[st - 1] + WRAY3_ZETA[st] : 0.0;
            ac.an = st > 0 ? WRAY3_GAMMA[st - 1] : 0.0;
        } else {
            ac.bn = st > 0 ? B[st - 1] : 0.0;
            ac.an = st > 0 ? A[st - 1] : 0.0;
        }
        const double* ysrc = lowst ? nullptr : ybar;   // null: the kernel chains ubar itself
        df* kb = st > 0 ? F : nullptr;
        if (lowst || st == 0)
            KLAUNCH(g, "adj_rhs", (k_adj_rhs_z<df, double, double><<<ag, dim3(AJX, AJY), adj_smem, g->stream>>>(
                                      ac, lowst ? U64[st] : un, W, ysrc, ubar, kb, part, nullptr, akc, ubar)));
        else
            KLAUNCH(g, "adj_rhs", (k_adj_rhs_z<df, df, double><<<ag, dim3(AJX, AJY), adj_smem, g->stream>>>(
                                      ac, U[st], W, ysrc, ubar, kb, part, nullptr, akc, ubar)));
        if (nubar) KLAUNCH(g, "sum_partials", k_sum_partials<<<1, 256, 0, g->stream>>>(part, nblk, nubar));
    }
    return INS_OK;
}

template <typename T, int DIM, bool WALL>
ins_status Impl<T, DIM, WALL>::step_vjp(ins_grid* g, const T* un, const double* dt_dev, double dt_host, const T* ybar, T* ubar, double* nubar) {
    if constexpr (WALL && DIM == 3 && std::is_same<T, double>::value) {
        if (g->use_df && !g->closure && !g->eddy && !g->use_dct && g->scheme == INS_RK4 &&
            reinterpret_cast<uintptr_t>(un) % 16 == 0)
            return step_vjp_wall_df(g, un, dt_dev, dt_host, ybar, ubar, nubar);
    }
    if constexpr (WALL) return step_vjp_wall(g, un, dt_dev, dt_host, ybar, ubar, nubar);
    if constexpr (std::is_same<T, double>::value && DIM == 3 && !WALL) {
        if (g->use_df && !g->closure && !g->eddy && reinterpret_cast<uintptr_t>(un) % 16 == 0)
            return step_vjp_df(g, un, dt_dev, dt_host, ybar, ubar, nubar);
    }
    static const double A[3] = {0.5, 0.5, 1.0};
    static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const long N = g->N;
    const size_t fld = (size_t)g->dim * N * sizeof(T);
    const dim3 cg = cell_grid(g);
    // z-marching adjoint stencil (3-D): chunks of planes per CTA, the chunk from the wave count
    // of the resident CTAs (each CTA stages its chunk plus two halo planes)
    // FP32 (step fusion level 2): the two-cells-per-thread march k_adj_rhs_z2 on 64 x 8 columns
    bool pair_adj = false;
    if constexpr (DIM == 3 && std::is_same<T, float>::value) {
        auto al8 = [](const void* q) { return q == nullptr || reinterpret_cast<uintptr_t>(q) % 8 == 0; };
        pair_adj = g->fusion == 2 && g->nx % 2 == 0 && 3 * g->N < (1L << 31) && al8(un) && al8(ubar) && al8(ybar);
    }
    const int abx = pair_adj ? (g->nx + 63) / 64 : (g->nx + AJX - 1) / AJX, aby = (g->ny + AJY - 1) / AJY;
    const size_t adj_smem = pair_adj ? (size_t)ax2_smem() : 4 * 6 * AJSP * sizeof(T);
    static int adj_per_sm = 0, adj2_per_sm = 0;
    if (DIM == 3) {
        if (pair_adj) {
            if constexpr (std::is_same<T, float>::value) {
                INS_CUDA(cudaFuncSetAttribute(k_adj_rhs_z2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_smem));
                if (!adj2_per_sm) {
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&adj2_per_sm, k_adj_rhs_z2, 256, adj_smem);
                    if (adj2_per_sm < 1) adj2_per_sm = 1;
                }
            }
        } else {
            INS_CUDA(cudaFuncSetAttribute(k_adj_rhs_z<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_smem));
            if (!adj_per_sm) {
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&adj_per_sm, k_adj_rhs_z<T>, AJX * AJY, adj_smem);
                if (adj_per_sm < 1) adj_per_sm = 1;
            }
        }
    }
    const long adj_resident = (long)(pair_adj ? adj2_per_sm : adj_per_sm) * device_sm_count();
    const int akc = DIM == 3 ? wave_chunk((long)abx * aby, g->nz, adj_resident, 2) : 1;
    const dim3 ag(abx, aby, (g->nz + akc - 1) / akc);
    const long nblk = DIM == 3 ? (long)ag.x * ag.y * ag.z : (long)cg.x * cg.y * cg.z;
    const size_t need = 5 * ((fld + 255) & ~size_t(255)) + (size_t)nblk * 8;
    if (g->vjp_bytes < need) {
        if (g->vjp) cudaFree(g->vjp);
        g->vjp = nullptr;
        g->vjp_bytes = 0;
        cudaError_t e = cudaMalloc(&g->vjp, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(INS_ERR_OOM, std::string("step-VJP workspace: ") + cudaGetErrorString(e));
        }
        g->vjp_bytes = need;
    }
    char* vb = reinterpret_cast<char*>(g->vjp);
    const size_t fa = (fld + 255) & ~size_t(255);
    T* U[4] = {const_cast<T*>(un), reinterpret_cast<T*>(vb), reinterpret_cast<T*>(vb + fa),
               reinterpret_cast<T*>(vb + 2 * fa)};
    T* W = reinterpret_cast<T*>(vb + 3 * fa);
    T* Cb = reinterpret_cast<T*>(vb + 4 * fa);       // closure pullback of the stage
    double* part = reinterpret_cast<double*>(vb + 5 * fa);
    T* F = reinterpret_cast<T*>(g->F);
    T* rp = reinterpret_cast<T*>(g->rp);
    T* scratch = reinterpret_cast<T*>(g->acc);
    ins_status s;
    const bool lowst = g->scheme == INS_WRAY3;
    const int nst = lowst ? 3 : 4;
    // forward: RK4 u_{s+1} = u_n + dt a_{s+1,s} k_s, s = 0, 1, 2; Wray
    // u_{s+1} = u_s + dt (gamma_s k_s + zeta_s k_{s-1}), s = 0, 1 (k_{s-1} kept in scratch)
    for (int st = 0; lowst && st < 2; ++st) {
        T* m = nullptr;
        if ((s = closure_term<T>(g, U[st], &m, false)) != INS_OK) return s;
        if ((s = launch_rhs_div<T, DIM, WALL>(g, U[st], F, rp, m)) != INS_OK) return s;
        if ((s = poisson<T>(g, rp, rp)) != INS_OK) return s;
        RkArgs ra;
        ra.dt_dev = dt_dev;
        ra.dt_host = dt_host;
        ra.a_next = WRAY3_GAMMA[st];
        ra.b = WRAY3_ZETA[st];
        ra.stage = st;
        ra.last = 0;
        ra.mx = nullptr;
        ra.err_flag = g->err_flag;
        if ((s = rk_update<true>(g, F, rp, U[st], scratch, U[st + 1], ra)) != INS_OK) return s;
    }
    // FP32 3-D RK4 without a closure: stages 2 and 3 recomputed by the fused boundary kernel, which
    // stores the staged u_{s+1} of its own cells (no accumulator; p and r in separate buffers)
    bool fused_rc = false;
    if constexpr (DIM == 3 && std::is_same<T, float>::value) {
        fused_rc = !lowst && !g->closure && !g->eddy && g->pbuf && g->us && pair_ok(g, un) &&
                   reinterpret_cast<uintptr_t>(un) % 16 == 0;
        if (fused_rc) {
            T* Fb[2] = {F, reinterpret_cast<T*>(g->us)};
            T* pp = reinterpret_cast<T*>(g->pbuf);
            if ((s = launch_rhs_div<T, DIM, WALL>(g, U[0], Fb[0], rp)) != INS_OK) return s;
            if ((s = poisson<T>(g, rp, pp)) != INS_OK) return s;
            for (int st = 0; st < 2; ++st) {
                FusedArgs fa;
                fa.dt_dev = dt_dev;
                fa.dt_host = dt_host;
                fa.a_next = A[st];
                fa.b = 0.0;
                fa.stage = st;
                fa.ust = U[st + 1];
                if ((s = launch_pair<WALL, true, true>(g, "update_rhs_div", Fb[st & 1], pp, U[0], nullptr,
                                                       Fb[(st + 1) & 1], rp, fa)) != INS_OK)
                    return s;
                if ((s = poisson<T>(g, rp, pp)) != INS_OK) return s;
            }
            RkArgs ra;
            ra.dt_dev = dt_dev;
            ra.dt_host = dt_host;
            ra.a_next = A[2];
            ra.b = 0.0;
            ra.stage = 0;
            ra.last = 0;
            ra.mx = nullptr;
            ra.err_flag = g->err_flag;
            if ((s = rk_update<false>(g, Fb[0], pp, U[0], nullptr, U[3], ra)) != INS_OK) return s;
        }
    }
    for (int st = 0; !lowst && !fused_rc && st < 3; ++st) {
        T* m = nullptr;
        if ((s = closure_term<T>(g, U[st], &m, false)) != INS_OK) return s;
        if ((s = launch_rhs_div<T, DIM, WALL>(g, U[st], F, rp, m)) != INS_OK) return s;
        if ((s = poisson<T>(g, rp, rp)) != INS_OK) return s;
        RkArgs ra;
        ra.dt_dev = dt_dev;
        ra.dt_host = dt_host;
        ra.a_next = A[st];
        ra.b = 0.0;
        ra.stage = 0;     // writes us = u0 + dt a k only (no acc), leaves u0 untouched
        ra.last = 0;
        ra.mx = nullptr;
        ra.err_flag = g->err_flag;
        if ((s = rk_update<false>(g, F, rp, U[0], nullptr, U[st + 1], ra)) != INS_OK) return s;
    }
    // reverse. 3-D with vector rows: the last stage's cotangent dt b ybar is formed inside its P^T
    // passes and the first adjoint march reads ybar as the accumulator's previous value, so neither
    // the copy ubar <- ybar nor the scaled field is materialised.
    const double blast = lowst ? WRAY3_GAMMA[2] : B[3];
    // (FP32 only: in FP64 the folded multiplies load the FP64 pipe as much as the passes they save)
    const bool fold = DIM == 3 && sizeof(T) == 4 && rk_vec_ok<T>(g, ybar) &&
                      reinterpret_cast<uintptr_t>(rp) % 16 == 0 && reinterpret_cast<uintptr_t>(W) % 16 == 0;
    if (!fold) {
        INS_CUDA(cudaMemcpyAsync(ubar, ybar, fld, cudaMemcpyDeviceToDevice, g->stream));
        const long n = (long)g->dim * N;
        KLAUNCH(g, "scale", k_scale_dt<T><<<1184, 256, 0, g->stream>>>(ybar, F, dt_dev, dt_host, blast, n));
    }
    AdjCoef<T> ac;
    ac.nx = g->nx;
    ac.ny = g->ny;
    ac.nz = g->nz;
    for (int a = 0; a < 3; ++a) {
        const double D = g->d[a][0];
        ac.c1[a] = (T)(0.5 / D);
        ac.c2[a] = (T)(0.25 / D);
        ac.l2[a] = (T)(1.0 / (D * D));
    }
    ac.nu = (T)g->nu;
    ac.dt_dev = dt_dev;
    ac.dt_host = dt_host;
    for (int st = nst - 1; st >= 0; --st) {
        // w = P kbar_s (P is symmetric on a uniform periodic grid)
        const bool first = fold && st == nst - 1;
        const T* uin = first ? ybar : ubar;   // the accumulator's previous value
        if (first) {
            constexpr int V = VecT<T>::N;
            if ((s = vec_width(g) == V ? div_fold_vec<V>(g, ybar, rp, dt_dev, dt_host, blast)
                                       : div_fold_vec<V / 2>(g, ybar, rp, dt_dev, dt_host, blast)) != INS_OK)
                return s;
            if ((s = poisson<T>(g, rp, rp)) != INS_OK) return s;
            if ((s = vec_width(g) == V ? sub_fold_vec<V>(g, ybar, rp, W, dt_dev, dt_host, blast)
                                       : sub_fold_vec<V / 2>(g, ybar, rp, W, dt_dev, dt_host, blast)) != INS_OK)
                return s;
        } else {
            if ((s = div_fast(g, F, rp)) != INS_OK) return s;
            if ((s = poisson<T>(g, rp, rp)) != INS_OK) return s;
            if ((s = sub_grad_fast(g, F, rp, W)) != INS_OK) return s;
        }
        if (lowst) {
            // kbar_{s-1} = dt gamma_{s-1} (Ubar_{s+1} + ubar_s) + dt zeta_s Ubar_{s+1}
            ac.bn = st > 0 ? WRAY3_GAMMA[st - 1] + WRAY3_ZETA[st] : 0.0;
            ac.an = st > 0 ? WRAY3_GAMMA[st - 1] : 0.0;
        } else {
            ac.bn = st > 0 ? B[st - 1] : 0.0;
            ac.an = st > 0 ? A[st - 1] : 0.0;
        }
        const T* ysrc = lowst ? nullptr : ybar;   // null: the kernel chains ubar itself
        const T* extra = nullptr;
        if (g->closure) {
            T* m = nullptr;
            if ((s = closure_term<T>(g, U[st], &m, true)) != INS_OK) return s;
            INS_CUDA(cudaMemsetAsync(Cb, 0, fld, g->stream));
            if ((s = closure_pullback<T>(g, W, Cb)) != INS_OK) return s;
            extra = Cb;
        }
        if (DIM == 3) {
            bool done = false;
            if constexpr (std::is_same<T, float>::value) {
                if (pair_adj) {
                    KLAUNCH(g, "adj_rhs", k_adj_rhs_z2<<<ag, dim3(32, 8), adj_smem, g->stream>>>(
                                              ac, U[st], W, ysrc, ubar, st > 0 ? F : nullptr, part, extra, akc, uin));
                    done = true;
                }
            }
            if (!done)
                KLAUNCH(g, "adj_rhs", k_adj_rhs_z<T><<<ag, dim3(AJX, AJY), adj_smem, g->stream>>>(
                                          ac, U[st], W, ysrc, ubar, st > 0 ? F : nullptr, part, extra, akc, uin));
        } else {
            KLAUNCH(g, "adj_rhs", k_adj_rhs<T, DIM><<<cg, dim3(32, 8), 0, g->stream>>>(
                                      ac, U[st], W, ysrc, ubar, st > 0 ? F : nullptr, part, extra));
        }
        if (nubar) KLAUNCH(g, "sum_partials", k_sum_partials<<<1, 256, 0, g->stream>>>(part, nblk, nubar));
    }
    return INS_OK;
}

}  // namespace
