// libins: the CNN closure (ins_closure_* in include/ins.h): parameter blobs, the tcgen05
// convolution launches of the forward pass, the data gradient and the weight gradient, and the
// closure term and pullback that the step and the step VJP call.
#include "ins_internal.cuh"

namespace {
constexpr int CL_CIN[4] = {3, 32, 32, 32};
constexpr int CL_COUT[4] = {32, 32, 32, 3};
// blob geometry (N rows, KG channel groups) of the forward and transposed weights
constexpr int CL_FN[4] = {32, 32, 32, 16}, CL_FKG[4] = {2, 4, 4, 4};
constexpr int CL_TN[4] = {16, 32, 32, 32}, CL_TKG[4] = {4, 4, 4, 2};

template <int CG, int N, int EPI>
size_t conv_smem() {
    constexpr int KG = CG == 1 ? 2 : CG;
    return (size_t)CV_SLOTS * CG * CV_CGB + 27 * (size_t)N * KG * 16;
}

template <int CG, int N, int EPI>
ins_status conv_attr() {
    INS_CUDA(cudaFuncSetAttribute(k_conv3d_tc<CG, N, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)conv_smem<CG, N, EPI>()));
    return INS_OK;
}

template <int CG, int N, int EPI>
ins_status conv_launch(ins_grid* g, ConvArgs a) {
    a.nx = g->nx;
    a.ny = g->ny;
    a.nz = g->nz;
    // z chunks of whole 4-plane groups, one CTA per SM: the chunk with the shortest estimated
    // makespan (waves x groups per CTA), the longest among equals (fewer weight and halo loads)
    const long cols = (long)(g->nx / CV_TX) * (g->ny / CV_TY);
    const long sms = device_sm_count();
    int zc = CV_G;
    long best = -1;
    for (int c = CV_G; c < g->nz + CV_G; c += CV_G) {
        const long ctas = cols * ((g->nz + c - 1) / c);
        const long cost = (ctas + sms - 1) / sms * (c / CV_G);
        if (best < 0 || cost <= best) {
            best = cost;
            zc = c;
        }
    }
    a.zchunk = zc;
    const dim3 grd(g->nx / CV_TX, g->ny / CV_TY, (g->nz + zc - 1) / zc);
    // profile names by shape: 8 -> 32 channels (first layer, last data gradient), 32 -> 32 forward
    // and data gradient, 32 -> 16 (3 used; last layer, first data gradient)
    constexpr const char* name = CG == 1 ? "conv3d_tc_8to32"
                                 : N == 16 ? "conv3d_tc_32to16"
                                 : EPI == EPI_GELU ? "conv3d_tc_32to32" : "conv3d_tc_32to32_dgrad";
    // programmatic dependent launch: the kernel's set-up may overlap the previous kernel's tail
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grd;
    cfg.blockDim = dim3(CV_THREADS);
    cfg.dynamicSmemBytes = conv_smem<CG, N, EPI>();
    cfg.stream = g->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    KLAUNCH(g, name, INS_CUDA(cudaLaunchKernelEx(&cfg, k_conv3d_tc<CG, N, EPI>, a)));
    return INS_OK;
}

// Grid of k_wgrad_plane: 16 x 8 columns, z chunks.
// One CTA per SM at a time: the z chunk with the shortest estimated time in units of one plane's
// MMAs (measured: about 2.4 us per plane, 7 us of set-up and accumulator read-out per CTA, and the
// reduction of one 110 KB partial block per CTA): waves x (planes + 3) + CTAs / 40. A second
// partial wave of CTAs doubles the time.
dim3 wgrad_plane_grid(const ins_grid* g, int* zchunk) {
    const long cols = (long)(g->nx / WP_TX) * (g->ny / WP_TY);
    const long sms = device_sm_count();
    int zc = g->nz;
    long best = -1;
    for (int c = 1; c <= g->nz; ++c) {
        const long ctas = cols * ((g->nz + c - 1) / c);
        const long cost = 40 * ((ctas + sms - 1) / sms) * (c + 3) + ctas;
        if (best < 0 || cost <= best) {
            best = cost;
            zc = c;
        }
    }
    *zchunk = zc;
    return dim3(g->nx / WP_TX, g->ny / WP_TY, (g->nz + zc - 1) / zc);
}

template <int CX, int CY>
ins_status wgrad_launch(ins_grid* g, const __nv_bfloat16* X, const __nv_bfloat16* dY, int cin, int cout, float* dW,
                        float* db, unsigned int* err, float* part = nullptr) {
    if (!dW) return INS_OK;
    if constexpr (CX == 32) {
        // 32 input channels: staged planes, the tap shifts in the MMA descriptors (no gathers);
        // about one CTA per SM (each holds all 27 tap accumulators in TMEM)
        if (part && g->nx % WP_TX == 0 && g->ny % WP_TY == 0) {
            constexpr int N = CY < 16 ? 16 : CY;
            static bool pattr = false;
            if (!pattr) {
                INS_CUDA(cudaFuncSetAttribute(k_wgrad_plane<CY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              WpShape<N>::SMEM));
                pattr = true;
            }
            int zc;
            const dim3 grd = wgrad_plane_grid(g, &zc);
            KLAUNCH(g, "wgrad_plane", (k_wgrad_plane<CY><<<grd, 256, WpShape<N>::SMEM, g->stream>>>(
                                    X, dY, g->nx, g->ny, g->nz, cout, zc, part, db, err)));
            const int ncta = (int)(grd.x * grd.y * grd.z);
            KLAUNCH(g, "wgrad_reduce", k_wgrad_reduce<<<(27 * 32 * cout + 31) / 32, 256, 0, g->stream>>>(
                                           part, ncta, N, cout, dW));
            return INS_OK;
        }
    }
    const long nvox = g->N;
    // tensor cores: 128 / CX taps per CTA, the voxels split over about two CTAs per SM in all
    constexpr int N = CY < 16 ? 16 : CY;
    constexpr int ngroups = (27 + 128 / CX - 1) / (128 / CX);
    static bool attr = false;
    if (!attr) {
        INS_CUDA(cudaFuncSetAttribute(k_wgrad_tc<CX, CY>, cudaFuncAttributeMaxDynamicSharedMemorySize, WgShape<N>::SMEM));
        attr = true;
    }
    long nchunk = (2L * device_sm_count()) / ngroups;     // one wave of two CTAs per SM
    const long stages = (nvox + WG_S - 1) / WG_S;
    nchunk = nchunk > stages ? stages : (nchunk < 1 ? 1 : nchunk);
    const long vchunk = ((stages + nchunk - 1) / nchunk) * WG_S;
    nchunk = (nvox + vchunk - 1) / vchunk;
    KLAUNCH(g, "wgrad_gather", k_wgrad_tc<CX, CY><<<dim3(ngroups, (unsigned)nchunk), WG_THREADS, WgShape<N>::SMEM, g->stream>>>(
                            X, dY, g->nx, g->ny, g->nz, cin, cout, vchunk, dW, db, err));
    return INS_OK;
}

// Forward through the four layers; keeps x0..x3 and (when save) z1..z3. m: dim fields of T.
template <typename T>
ins_status closure_forward(ins_grid* g, ins_closure* c, const T* u, T* m, bool save) {
    const long nvox = g->N;
    KLAUNCH(g, "pack_input", k_pack_input<T><<<592, 256, 0, g->stream>>>(u, nvox, c->x[0]));
    ConvArgs a{};
    a.err = c->err;
    ins_status s;
    for (int l = 0; l < 3; ++l) {
        a.x = c->x[l];
        a.wblob = c->wf[l];
        a.bias = c->bias[l];
        a.y = c->x[l + 1];
        a.zout = save ? c->z[l] : nullptr;
        s = l == 0 ? conv_launch<1, 32, EPI_GELU>(g, a) : conv_launch<4, 32, EPI_GELU>(g, a);
        if (s != INS_OK) return s;
    }
    a.x = c->x[3];
    a.wblob = c->wf[3];
    a.bias = c->bias[3];
    a.y = nullptr;
    a.zout = nullptr;
    a.out = m;
    a.out_f64 = sizeof(T) == 8;
    a.nreal = 3;
    return conv_launch<4, 16, EPI_OUT>(g, a);
}

// Backward from mbar (dim fields of T) using the activations of the last saving forward:
// ubar += J_m^T mbar, dW[l], db[l] += weight and bias gradients (when non-null).
template <typename T>
ins_status closure_backward(ins_grid* g, ins_closure* c, const T* mbar, T* ubar, float* const* dW, float* const* db) {
    const long nvox = g->N;
    KLAUNCH(g, "pack_input", k_pack_input<T><<<592, 256, 0, g->stream>>>(mbar, nvox, c->g4));
    ins_status s;
    if ((s = wgrad_launch<32, 8>(g, c->x[3], c->g4, 32, 3, dW[3], db[3], c->err, c->wpart)) != INS_OK) return s;
    ConvArgs a{};
    a.err = c->err;
    // layer 4 data gradient through GELU of layer 3
    a.x = c->g4;
    a.wblob = c->wt[3];
    a.y = c->ga;
    a.zin = c->z[2];
    if ((s = conv_launch<1, 32, EPI_DGELU>(g, a)) != INS_OK) return s;
    __nv_bfloat16* gin = c->ga;
    __nv_bfloat16* gout = c->gb;
    for (int l = 2; l >= 1; --l) {
        if ((s = wgrad_launch<32, 32>(g, c->x[l], gin, 32, 32, dW[l], db[l], c->err, c->wpart)) != INS_OK) return s;
        a.x = gin;
        a.wblob = c->wt[l];
        a.y = gout;
        a.zin = c->z[l - 1];
        if ((s = conv_launch<4, 32, EPI_DGELU>(g, a)) != INS_OK) return s;
        __nv_bfloat16* t = gin;
        gin = gout;
        gout = t;
    }
    if ((s = wgrad_launch<8, 32>(g, c->x[0], gin, 3, 32, dW[0], db[0], c->err)) != INS_OK) return s;
    a.x = gin;
    a.wblob = c->wt[0];
    a.y = nullptr;
    a.zin = nullptr;
    a.out = ubar;
    a.out_f64 = sizeof(T) == 8;
    a.nreal = 3;
    return conv_launch<4, 16, EPI_ACCUM>(g, a);
}
}  // namespace

// m(u) of the attached closure or eddy-viscosity model (*m = null when none is attached).
template <typename T>
ins_status closure_term(ins_grid* g, const T* u, T** m, bool save) {
    *m = nullptr;
    if (g->eddy) {
        T* term = reinterpret_cast<T*>(g->eddy_buf) + g->N;
        const ins_status s = eddy_term<T>(g, u, term);
        if (s == INS_OK) *m = term;
        return s;
    }
    if (!g->closure) return INS_OK;
    T* out = reinterpret_cast<T*>(g->mbuf);
    ins_status s = closure_forward<T>(g, g->closure, u, out, save);
    if (s == INS_OK) *m = out;
    return s;
}

// ubar += J_m^T w with the attached closure's saved activations; weight gradients accumulate
// into the buffers given to ins_closure_set_grads.
template <typename T>
ins_status closure_pullback(ins_grid* g, const T* w, T* ubar) {
    ins_closure* c = g->closure;
    return closure_backward<T>(g, c, w, ubar, c->gW, c->gB);
}

template ins_status closure_term<float>(ins_grid*, const float*, float**, bool);
template ins_status closure_term<double>(ins_grid*, const double*, double**, bool);
template ins_status closure_pullback<float>(ins_grid*, const float*, float*);
template ins_status closure_pullback<double>(ins_grid*, const double*, double*);

extern "C" {

ins_status ins_closure_create(ins_grid* g, ins_closure** out) {
    g_err.clear();
    if (!g || !out) return fail(INS_ERR_ARG, "null argument");
    *out = nullptr;
    if (g->dim != 3 || g->wall_y) return fail(INS_ERR_UNSUPPORTED, "the closure needs a 3-D periodic grid");
    if (g->nx % CV_TX || g->ny % CV_TY || g->nz < 2)
        return fail(INS_ERR_UNSUPPORTED, "the closure needs nx % 8 == 0, ny % 16 == 0 and nz >= 2");
    ins_closure* c = new ins_closure();
    c->g = g;
    c->nvox = g->N;
    const long nv = g->N;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t off = 0, o_wf[4], o_wt[4], o_x[4], o_z[3], o_ga, o_gb, o_g4, o_err;
    for (int l = 0; l < 4; ++l) {
        o_wf[l] = off;
        off += al((size_t)27 * CL_FN[l] * CL_FKG[l] * 16);
        o_wt[l] = off;
        off += al((size_t)27 * CL_TN[l] * CL_TKG[l] * 16);
    }
    for (int l = 0; l < 4; ++l) {
        o_x[l] = off;
        off += al((size_t)nv * (l == 0 ? 8 : 32) * 2);
    }
    for (int l = 0; l < 3; ++l) {
        o_z[l] = off;
        off += al((size_t)nv * 32 * 4);
    }
    o_ga = off; off += al((size_t)nv * 32 * 2);
    o_gb = off; off += al((size_t)nv * 32 * 2);
    o_g4 = off; off += al((size_t)nv * 8 * 2);
    o_err = off; off += al(4);
    size_t o_wp = 0;
    const bool plane_wgrad = g->nx % WP_TX == 0 && g->ny % WP_TY == 0;
    if (plane_wgrad) {
        int zc;
        const dim3 wg = wgrad_plane_grid(g, &zc);
        o_wp = off;
        off += al((size_t)wg.x * wg.y * wg.z * 27 * 32 * 32 * sizeof(float));
    }
    cudaError_t e = cudaMalloc(&c->buf, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(INS_ERR_OOM, std::string("closure workspace: ") + cudaGetErrorString(e));
    }
    c->bytes = off;
    char* b = reinterpret_cast<char*>(c->buf);
    for (int l = 0; l < 4; ++l) {
        c->wf[l] = reinterpret_cast<__nv_bfloat16*>(b + o_wf[l]);
        c->wt[l] = reinterpret_cast<__nv_bfloat16*>(b + o_wt[l]);
        c->x[l] = reinterpret_cast<__nv_bfloat16*>(b + o_x[l]);
    }
    for (int l = 0; l < 3; ++l) c->z[l] = reinterpret_cast<float*>(b + o_z[l]);
    c->ga = reinterpret_cast<__nv_bfloat16*>(b + o_ga);
    c->gb = reinterpret_cast<__nv_bfloat16*>(b + o_gb);
    c->g4 = reinterpret_cast<__nv_bfloat16*>(b + o_g4);
    c->err = reinterpret_cast<unsigned int*>(b + o_err);
    c->wpart = plane_wgrad ? reinterpret_cast<float*>(b + o_wp) : nullptr;
    bool ok = cudaMemset(c->buf, 0, off) == cudaSuccess;
    ins_status st = INS_OK;
    if (ok) st = conv_attr<1, 32, EPI_GELU>();
    if (st == INS_OK) st = conv_attr<4, 32, EPI_GELU>();
    if (st == INS_OK) st = conv_attr<4, 16, EPI_OUT>();
    if (st == INS_OK) st = conv_attr<1, 32, EPI_DGELU>();
    if (st == INS_OK) st = conv_attr<4, 32, EPI_DGELU>();
    if (st == INS_OK) st = conv_attr<4, 16, EPI_ACCUM>();
    if (!ok || st != INS_OK || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(c->buf);
        delete c;
        return st != INS_OK ? st : fail(INS_ERR_CUDA, "closure set-up failed");
    }
    *out = c;
    return INS_OK;
}

ins_status ins_closure_destroy(ins_closure* c) {
    if (!c) return INS_OK;
    if (c->g && c->g->closure == c) c->g->closure = nullptr;
    cudaStreamSynchronize(c->g ? c->g->stream : nullptr);
    cudaFree(c->buf);
    delete c;
    return INS_OK;
}

ins_status ins_closure_set_params(ins_closure* c, const float* const W[4], const float* const bias[4]) {
    g_err.clear();
    if (!c || !W || !bias) return fail(INS_ERR_ARG, "null argument");
    ins_grid* g = c->g;
    for (int l = 0; l < 4; ++l) {
        if (!W[l] || !bias[l]) return fail(INS_ERR_ARG, "null weight or bias pointer");
        KLAUNCH(g, "pack_weights", k_pack_weights<<<216, 256, 0, g->stream>>>(W[l], CL_CIN[l], CL_COUT[l], CL_FN[l],
                                                                             CL_FKG[l], 0, c->wf[l]));
        KLAUNCH(g, "pack_weights", k_pack_weights<<<216, 256, 0, g->stream>>>(W[l], CL_CIN[l], CL_COUT[l], CL_TN[l],
                                                                             CL_TKG[l], 1, c->wt[l]));
        c->bias[l] = bias[l];
    }
    c->params_set = 1;
    return INS_OK;
}

ins_status ins_closure_set_grads(ins_closure* c, float* const dW[4], float* const db[4]) {
    g_err.clear();
    if (!c) return fail(INS_ERR_ARG, "null closure");
    for (int l = 0; l < 4; ++l) {
        c->gW[l] = dW ? dW[l] : nullptr;
        c->gB[l] = db ? db[l] : nullptr;
    }
    return INS_OK;
}

ins_status ins_closure_fwd(ins_grid* g, ins_closure* c, const void* u, void* m, int save) {
    g_err.clear();
    if (!g || !c || c->g != g) return fail(INS_ERR_ARG, "closure and grid do not match");
    if (!c->params_set) return fail(INS_ERR_ARG, "ins_closure_set_params was not called");
    CHECK(check_ptr(g, u, "u"));
    CHECK(check_ptr(g, m, "m"));
    if (g->dtype == INS_F64) return closure_forward<double>(g, c, (const double*)u, (double*)m, save != 0);
    return closure_forward<float>(g, c, (const float*)u, (float*)m, save != 0);
}

ins_status ins_closure_bwd(ins_grid* g, ins_closure* c, const void* mbar, void* ubar_accum, float* const dW[4],
                           float* const db[4]) {
    g_err.clear();
    if (!g || !c || c->g != g) return fail(INS_ERR_ARG, "closure and grid do not match");
    CHECK(check_ptr(g, mbar, "mbar"));
    CHECK(check_ptr(g, ubar_accum, "ubar_accum"));
    float* const nw[4] = {nullptr, nullptr, nullptr, nullptr};
    float* const* w = dW ? dW : nw;
    float* const* bb = db ? db : nw;
    if (g->dtype == INS_F64) return closure_backward<double>(g, c, (const double*)mbar, (double*)ubar_accum, w, bb);
    return closure_backward<float>(g, c, (const float*)mbar, (float*)ubar_accum, w, bb);
}

ins_status ins_closure_saved(ins_closure* c, int layer, void* x_bf16, float* z) {
    g_err.clear();
    if (!c || layer < 0 || layer > 3) return fail(INS_ERR_ARG, "bad argument");
    const size_t nv = (size_t)c->nvox;
    cudaStream_t st = c->g->stream;
    if (x_bf16)
        INS_CUDA(cudaMemcpyAsync(x_bf16, c->x[layer], nv * (layer == 0 ? 8 : 32) * 2, cudaMemcpyDeviceToDevice, st));
    if (z && layer < 3) INS_CUDA(cudaMemcpyAsync(z, c->z[layer], nv * 32 * 4, cudaMemcpyDeviceToDevice, st));
    INS_CUDA(cudaStreamSynchronize(st));
    return INS_OK;
}

ins_status ins_closure_check(ins_closure* c) {
    g_err.clear();
    if (!c) return fail(INS_ERR_ARG, "null closure");
    unsigned int f = 0;
    INS_CUDA(cudaMemcpyAsync(&f, c->err, 4, cudaMemcpyDeviceToHost, c->g->stream));
    INS_CUDA(cudaStreamSynchronize(c->g->stream));
    if (f) {
        INS_CUDA(cudaMemsetAsync(c->err, 0, 4, c->g->stream));
        return fail(INS_ERR_TIMEOUT, "a tensor-core wait in the closure gave up");
    }
    return INS_OK;
}

ins_status ins_set_closure(ins_grid* g, ins_closure* c) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    if (c && c->g != g) return fail(INS_ERR_ARG, "closure belongs to another grid");
    if (c && !g->mbuf) {
        const size_t bytes = (size_t)g->dim * g->N * (g->dtype == INS_F64 ? 8 : 4);
        cudaError_t e = cudaMalloc(&g->mbuf, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g->mbuf = nullptr;
            return fail(INS_ERR_OOM, "closure output buffer");
        }
    }
    if (c && g->eddy) return fail(INS_ERR_UNSUPPORTED, "an eddy-viscosity model is attached (one closure at a time)");
    g->closure = c;
    return INS_OK;
}

}  // extern "C"
