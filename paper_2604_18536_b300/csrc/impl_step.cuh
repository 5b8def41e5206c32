// Impl::step_wray3, step_fused, step: the RK step of every grid configuration (classic RK4 with
// per-stage projection, Wray's low-storage RK3, the FP32 fused stage boundaries). Included by ins_step.cu.
#pragma once

#include "ins_internal.cuh"

namespace {

// Wray's low-storage 3-stage RK (two registers: F and k_{s-1}); u is updated in place.
template <typename T, int DIM, bool WALL>
ins_status Impl<T, DIM, WALL>::step_wray3(ins_grid* g, T* u, const double* dt_dev, double dt_host, double* next_dt, double cfl) {
    T* F = reinterpret_cast<T*>(g->F);
    T* rp = reinterpret_cast<T*>(g->rp);
    T* kprev = reinterpret_cast<T*>(g->acc);
    ins_status s;
    for (int st = 0; st < 3; ++st) {
        T* m = nullptr;
        if ((s = closure_term<T>(g, u, &m, false)) != INS_OK) return s;
        if ((s = launch_rhs_div<T, DIM, WALL>(g, u, F, rp, m)) != INS_OK) return s;
        if ((s = poisson<T>(g, rp, rp)) != INS_OK) return s;
        RkArgs ra;
        ra.dt_dev = dt_dev;
        ra.dt_host = dt_host;
        ra.a_next = WRAY3_GAMMA[st];
        ra.b = WRAY3_ZETA[st];
        ra.stage = st;
        ra.last = st == 2;
        ra.mx = (st == 2 && next_dt) ? g->cfl_max : nullptr;
        ra.err_flag = g->err_flag;
        if ((s = rk_update<true>(g, F, rp, u, kprev, nullptr, ra)) != INS_OK) return s;
    }
    if (next_dt) {
        KLAUNCH(g, "cfl_finalize", k_cfl_finalize<<<1, 256, 0, g->stream>>>(g->cfl_max, g->geo64, g->nx + g->ny + g->nz, g->dmin2_nu, cfl,
                                                next_dt));
    }
    return INS_OK;
}

// FP32 3-D RK4 without a closure: the update of stage s and the evaluation of stage s + 1
// run as one kernel (k_update_rhs_div); F alternates between two buffers, p_s and r_{s+1}
// live in separate buffers, no stage state is stored.
template <typename T, int DIM, bool WALL>
ins_status Impl<T, DIM, WALL>::step_fused(ins_grid* g, T* u, const double* dt_dev, double dt_host, double* next_dt, double cfl) {
    static const double A[3] = {0.5, 0.5, 1.0};
    static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    T* Fb[2] = {reinterpret_cast<T*>(g->F), reinterpret_cast<T*>(g->us)};
    T* rr = reinterpret_cast<T*>(g->rp);
    T* pp = reinterpret_cast<T*>(g->pbuf);
    T* acc = reinterpret_cast<T*>(g->acc);
    ins_status s;
    const RhsCoef<T> rc = make_rhs_coef<T>(g);
    const T* ihy = make_geo<T>(g).c[1] + (size_t)C_INV_H * g->ny;
    const T ihx = (T)(1.0 / g->h[0][0]), ihz = (T)(1.0 / g->h[2][0]);
    const dim3 blk(RBX, RBY, 1);
    const dim3 grd((g->nx + RBX - 1) / RBX, (g->ny + RBY - 1) / RBY, (g->nz + g->kchunk - 1) / g->kchunk);
    static_assert(std::is_same<T, float>::value && DIM == 3, "FP32 3-D only");
    const bool pair = pair_ok(g, u);   // the caller's field is 16-byte aligned, nx % 4 == 0 (rk_vec_ok)
    FusedArgs fa;
    fa.dt_dev = dt_dev;
    fa.dt_host = dt_host;
    fa.a_next = 0.0;
    fa.b = 0.0;
    fa.stage = 0;
    if ((s = launch_rhs_div<T, DIM, WALL>(g, u, Fb[0], rr)) != INS_OK) return s;
    if ((s = poisson<T>(g, rr, pp)) != INS_OK) return s;
    for (int st = 0; st < 3; ++st) {
        fa.a_next = A[st];
        fa.b = B[st];
        fa.stage = st;
        if (pair) {
            if ((s = launch_pair<WALL, true>(g, "update_rhs_div", Fb[st & 1], pp, u, acc, Fb[(st + 1) & 1], rr, fa)) !=
                INS_OK)
                return s;
        } else
            KLAUNCH(g, "update_rhs_div", k_update_rhs_div<T, WALL><<<grd, blk, 0, g->stream>>>(
                                             rc, ihx, ihz, ihy, Fb[st & 1], pp, u, acc, Fb[(st + 1) & 1], rr, fa,
                                             g->kchunk));
        if ((s = poisson<T>(g, rr, pp)) != INS_OK) return s;
    }
    RkArgs ra;
    ra.dt_dev = dt_dev;
    ra.dt_host = dt_host;
    ra.a_next = 0.0;
    ra.b = B[3];
    ra.stage = 3;
    ra.last = 1;
    ra.mx = next_dt ? g->cfl_max : nullptr;
    ra.err_flag = g->err_flag;
    if ((s = rk_update<false>(g, Fb[1], pp, u, acc, nullptr, ra)) != INS_OK) return s;
    if (next_dt) {
        KLAUNCH(g, "cfl_finalize", k_cfl_finalize<<<1, 256, 0, g->stream>>>(g->cfl_max, g->geo64, g->nx + g->ny + g->nz, g->dmin2_nu, cfl,
                                                next_dt));
    }
    return INS_OK;
}

// ------------------------------------------------------------ double-float FP64 step
// Wray's low-storage RK3 on an FP64 grid in double-float arithmetic: u (FP64) is updated in place each
// stage (the stage's increment added in FP64), k_{s-1} kept as double-float pairs. WALL: 3-D channels.
template <int DIM, bool WALL = false>
ins_status step_wray3_df(ins_grid* g, double* u, const double* dt_dev, double dt_host, double* next_dt, double cfl) {
    df* F = reinterpret_cast<df*>(g->F);
    df* rp = reinterpret_cast<df*>(g->rp);
    df* kprev = reinterpret_cast<df*>(g->acc);
    ins_status s;
    for (int st = 0; st < 3; ++st) {
        if ((s = launch_rhs_div_df<DIM, double, WALL>(g, u, F, rp)) != INS_OK) return s;
        if ((s = poisson<df>(g, rp, rp)) != INS_OK) return s;
        RkArgs ra;
        ra.dt_dev = dt_dev;
        ra.dt_host = dt_host;
        ra.a_next = WRAY3_GAMMA[st];
        ra.b = WRAY3_ZETA[st];
        ra.stage = st;
        ra.last = st == 2;
        ra.mx = (st == 2 && next_dt) ? g->cfl_max : nullptr;
        ra.err_flag = g->err_flag;
        if ((s = rk_update_df<DIM, true, WALL>(g, F, rp, u, kprev, nullptr, ra)) != INS_OK) return s;
    }
    if (next_dt) {
        KLAUNCH(g, "cfl_finalize", k_cfl_finalize<<<1, 256, 0, g->stream>>>(g->cfl_max, g->geo64, g->nx + g->ny + g->nz,
                                                                            g->dmin2_nu, cfl, next_dt));
    }
    return INS_OK;
}

// The classic RK4 step of an FP64 grid in double-float arithmetic (ins_set_f64_arithmetic): F, r/p,
// the spectrum, acc and the stage state hold double-float pairs; u stays FP64. WALL: 3-D channel
// grids (walls in y, stretched rows; the wall-normal solve is the double-float Thomas sweep).
template <int DIM, bool WALL = false>
ins_status step_df(ins_grid* g, double* u, const double* dt_dev, double dt_host, double* next_dt, double cfl) {
    static const double A[4] = {0.5, 0.5, 1.0, 0.0};
    static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    df* F = reinterpret_cast<df*>(g->F);
    df* rp = reinterpret_cast<df*>(g->rp);
    df* acc = reinterpret_cast<df*>(g->acc);
    df* us = reinterpret_cast<df*>(g->us);
    ins_status s;
    for (int st = 0; st < 4; ++st) {
        s = st == 0 ? launch_rhs_div_df<DIM, double, WALL>(g, u, F, rp) : launch_rhs_div_df<DIM, df, WALL>(g, us, F, rp);
        if (s != INS_OK) return s;
        if ((s = poisson<df>(g, rp, rp)) != INS_OK) return s;
        RkArgs ra;
        ra.dt_dev = dt_dev;
        ra.dt_host = dt_host;
        ra.a_next = A[st];
        ra.b = B[st];
        ra.stage = st;
        ra.last = st == 3;
        ra.mx = (st == 3 && next_dt) ? g->cfl_max : nullptr;
        ra.err_flag = g->err_flag;
        if ((s = rk_update_df<DIM, false, WALL>(g, F, rp, u, acc, us, ra)) != INS_OK) return s;
    }
    if (next_dt) {
        KLAUNCH(g, "cfl_finalize", k_cfl_finalize<<<1, 256, 0, g->stream>>>(g->cfl_max, g->geo64, g->nx + g->ny + g->nz,
                                                                            g->dmin2_nu, cfl, next_dt));
    }
    return INS_OK;
}

template <typename T, int DIM, bool WALL>
ins_status Impl<T, DIM, WALL>::step(ins_grid* g, T* u, const double* dt_dev, double dt_host, double* next_dt, double cfl) {
    if constexpr (std::is_same<T, double>::value && (!WALL || DIM == 3)) {
        if (g->scheme == INS_WRAY3 && g->use_df && !g->closure && !g->eddy && !(WALL && g->use_dct) &&
            reinterpret_cast<uintptr_t>(u) % 16 == 0)
            return step_wray3_df<DIM, WALL>(g, u, dt_dev, dt_host, next_dt, cfl);
    }
    if (g->scheme == INS_WRAY3) return step_wray3(g, u, dt_dev, dt_host, next_dt, cfl);
    if constexpr (std::is_same<T, double>::value && (!WALL || DIM == 3)) {
        if (g->use_df && !g->closure && !g->eddy && !(WALL && g->use_dct) && reinterpret_cast<uintptr_t>(u) % 16 == 0)
            return step_df<DIM, WALL>(g, u, dt_dev, dt_host, next_dt, cfl);
    }
    if constexpr (DIM == 3 && std::is_same<T, float>::value) {
        if (g->pbuf && !g->closure && !g->eddy && g->fusion > 0 && rk_vec_ok<T>(g, u))
            return step_fused(g, u, dt_dev, dt_host, next_dt, cfl);
    }
    static const double A[4] = {0.5, 0.5, 1.0, 0.0};
    static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    T* F = reinterpret_cast<T*>(g->F);
    T* rp = reinterpret_cast<T*>(g->rp);
    T* acc = reinterpret_cast<T*>(g->acc);
    T* us = reinterpret_cast<T*>(g->us);
    ins_status s;
    for (int st = 0; st < 4; ++st) {
        const T* src = st == 0 ? u : us;
        T* m = nullptr;
        if ((s = closure_term<T>(g, src, &m, false)) != INS_OK) return s;
        if ((s = launch_rhs_div<T, DIM, WALL>(g, src, F, rp, m)) != INS_OK) return s;
        if ((s = poisson<T>(g, rp, rp)) != INS_OK) return s;
        RkArgs ra;
        ra.dt_dev = dt_dev;
        ra.dt_host = dt_host;
        ra.a_next = A[st];
        ra.b = B[st];
        ra.stage = st;
        ra.last = st == 3;
        ra.mx = (st == 3 && next_dt) ? g->cfl_max : nullptr;
        ra.err_flag = g->err_flag;
        if ((s = rk_update<false>(g, F, rp, u, acc, us, ra)) != INS_OK) return s;
    }
    if (next_dt) {
        KLAUNCH(g, "cfl_finalize", k_cfl_finalize<<<1, 256, 0, g->stream>>>(g->cfl_max, g->geo64, g->nx + g->ny + g->nz, g->dmin2_nu, cfl,
                                                next_dt));
    }
    return INS_OK;
}

}  // namespace
