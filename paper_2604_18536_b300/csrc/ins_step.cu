// libins: the stencil operators, the projection and the RK step with its CUDA-graph replay (C ABI
// in include/ins.h; the per-config implementations are Impl in ins_internal.cuh and impl_step.cuh).
#include "ins_internal.cuh"
#include "impl_step.cuh"

extern "C" {

ins_status ins_rhs(ins_grid* g, const void* u, void* dudt, void* p) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    CHECK(check_ptr(g, u, "u"));
    CHECK(check_ptr(g, dudt, "dudt"));
    if (p) CHECK(check_ptr(g, p, "p"));
    return dispatch_dtype(g, [&](auto z) {
        using T = decltype(z);
        return dispatch<T>(g, [&](auto impl) {
            return decltype(impl)::rhs(g, (const T*)u, (T*)dudt, (T*)p);
        });
    });
}

ins_status ins_project(ins_grid* g, const void* u_in, void* u_out, void* p) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    CHECK(check_ptr(g, u_in, "u_in"));
    CHECK(check_ptr(g, u_out, "u_out"));
    if (p) CHECK(check_ptr(g, p, "p"));
    return dispatch_dtype(g, [&](auto z) {
        using T = decltype(z);
        return dispatch<T>(g, [&](auto impl) {
            return decltype(impl)::project(g, (const T*)u_in, (T*)u_out, (T*)p);
        });
    });
}

ins_status ins_divergence(ins_grid* g, const void* u, void* phi) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    CHECK(check_ptr(g, u, "u"));
    CHECK(check_ptr(g, phi, "phi"));
    return dispatch_dtype(g, [&](auto z) {
        using T = decltype(z);
        return dispatch<T>(g, [&](auto impl) { return decltype(impl)::divergence(g, (const T*)u, (T*)phi); });
    });
}

ins_status ins_set_wall_solver(ins_grid* g, int solver) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "ins_set_wall_solver: null grid");
    if (solver != INS_WALL_THOMAS && solver != INS_WALL_DCT) return fail(INS_ERR_ARG, "unknown wall solver");
    if (!g->wall_y) return fail(INS_ERR_UNSUPPORTED, "ins_set_wall_solver: no wall direction");
    if (solver == INS_WALL_DCT && !g->wall_dct)
        return fail(INS_ERR_UNSUPPORTED, "DCT solve needs a uniform wall-normal grid with n = 2^p 3^q 5^r 7^s <= 2048");
    g->use_dct = solver == INS_WALL_DCT;
    return INS_OK;
}

ins_status ins_set_step_fusion(ins_grid* g, int enable) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "ins_set_step_fusion: null grid");
    if (enable < 0 || enable > 2) return fail(INS_ERR_ARG, "ins_set_step_fusion: level must be 0, 1 or 2");
    g->fusion = enable;
    return INS_OK;
}

ins_status ins_set_march_chunk(ins_grid* g, int planes) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "ins_set_march_chunk: null grid");
    if (planes < 0) return fail(INS_ERR_ARG, "ins_set_march_chunk: planes must be >= 0");
    g->march_chunk = planes;
    return INS_OK;
}

static ins_status step_launch(ins_grid* g, void* u, const double* dt_dev, double dt_host, double* next_dt_dev,
                              double cfl) {
    return dispatch_dtype(g, [&](auto z) {
        using T = decltype(z);
        return dispatch<T>(g, [&](auto impl) {
            return decltype(impl)::step(g, (T*)u, dt_dev, dt_host, next_dt_dev, cfl);
        });
    });
}

ins_status ins_step(ins_grid* g, void* u, const double* dt_dev, double dt_host, double* next_dt_dev, double cfl) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    CHECK(check_ptr(g, u, "u"));
    if (!dt_dev && !(std::isfinite(dt_host) && dt_host >= 0.0)) return fail(INS_ERR_ARG, "dt_host must be finite, >= 0");
    if (next_dt_dev && !(std::isfinite(cfl) && cfl > 0.0)) return fail(INS_ERR_ARG, "cfl must be finite and > 0");
    return step_launch(g, u, dt_dev, dt_host, next_dt_dev, cfl);
}

ins_status ins_step_n(ins_grid* g, void* u, int nsteps, const double* dt_dev, double dt_host, double* next_dt_dev,
                      double cfl) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    if (nsteps < 0) return fail(INS_ERR_ARG, "ins_step_n: nsteps must be >= 0");
    if (nsteps == 0) return INS_OK;
    // the first step runs as plain launches (lazy workspace, kernel attributes)
    ins_status s = ins_step(g, u, dt_dev, dt_host, next_dt_dev, cfl);
    if (s != INS_OK || nsteps == 1) return s;
    const std::vector<double> key = {(double)reinterpret_cast<uintptr_t>(u), (double)reinterpret_cast<uintptr_t>(dt_dev),
                                     dt_host, (double)reinterpret_cast<uintptr_t>(next_dt_dev), cfl,
                                     (double)g->scheme, (double)g->fusion, (double)g->march_chunk, (double)g->use_dct,
                                     (double)g->eddy, g->eddy_C, (double)reinterpret_cast<uintptr_t>(g->closure), (double)g->use_df,
                                     (double)reinterpret_cast<uintptr_t>(g->stream)};
    if (!g->step_exec || key != g->graph_key) {
        if (g->step_exec) {
            cudaGraphExecDestroy(g->step_exec);
            g->step_exec = nullptr;
        }
        if (!g->cap_stream) INS_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
        const cudaStream_t saved = g->stream;
        const bool prof = g->prof;
        const unsigned long long l0 = g->launches;
        g->stream = g->cap_stream;
        g->prof = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
        ins_status cs = e == cudaSuccess ? step_launch(g, u, dt_dev, dt_host, next_dt_dev, cfl) : INS_ERR_CUDA;
        if (e == cudaSuccess) e = cudaStreamEndCapture(g->cap_stream, &graph);
        g->stream = saved;
        g->prof = prof;
        g->step_kernels = g->launches - l0;
        g->launches = l0;   // captured, not run
        if (cs == INS_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&g->step_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (cs != INS_OK || e != cudaSuccess || !g->step_exec) {
            // the step cannot be captured here: plain launches
            cudaGetLastError();
            g->step_exec = nullptr;
            g_err.clear();
            for (int i = 1; i < nsteps; ++i)
                if ((s = ins_step(g, u, dt_dev, dt_host, next_dt_dev, cfl)) != INS_OK) return s;
            return INS_OK;
        }
        g->graph_key = key;
    }
    for (int i = 1; i < nsteps; ++i) {
        INS_CUDA(cudaGraphLaunch(g->step_exec, g->stream));
        g->launches += g->step_kernels;
    }
    return INS_OK;
}

}  // extern "C"
