// libins: the pullback of one step, ins_step_vjp (C ABI in include/ins.h; the per-config
// implementations are in impl_vjp.cuh).
#include "ins_internal.cuh"
#include "impl_vjp.cuh"

extern "C" {

ins_status ins_step_vjp(ins_grid* g, const void* u_n, const double* dt_dev, double dt_host, const void* ubar_np1,
                        void* ubar_n, double* nubar_dev) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    CHECK(check_ptr(g, u_n, "u_n"));
    CHECK(check_ptr(g, ubar_np1, "ubar_np1"));
    CHECK(check_ptr(g, ubar_n, "ubar_n"));
    if (ubar_n == ubar_np1 || ubar_n == u_n) return fail(INS_ERR_ARG, "ubar_n must not alias u_n or ubar_np1");
    if (!dt_dev && !(std::isfinite(dt_host) && dt_host >= 0.0)) return fail(INS_ERR_ARG, "dt_host must be finite, >= 0");
    if (g->eddy) return fail(INS_ERR_UNSUPPORTED, "ins_step_vjp: eddy-viscosity models have no pullback here");
    return dispatch_dtype(g, [&](auto z) {
        using T = decltype(z);
        return dispatch<T>(g, [&](auto impl) {
            return decltype(impl)::step_vjp(g, (const T*)u_n, dt_dev, dt_host, (const T*)ubar_np1, (T*)ubar_n,
                                            nubar_dev);
        });
    });
}

}  // extern "C"
