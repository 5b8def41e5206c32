// Internal declarations shared by the translation units of libins: the grid and closure handles,
// error reporting, launch accounting, the Poisson-solve and stencil launchers, and the per-config
// implementation of every solver operation (Impl). The C ABI itself is declared in include/ins.h
// and defined by ins_grid.cu (handles, settings, diagnostics, measurement), ins_step.cu (operators,
// step, step VJP), ins_closure.cu (CNN closure), ins_eddy.cu (eddy viscosity) and ins_noalloc.cu.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ins.h"
#include "common.cuh"
#include "fft.cuh"
#include "fft_reg.cuh"
#include "rhs.cuh"
#include "stencil.cuh"
#include "rk.cuh"
#include "adjoint.cuh"
#include "adjoint_wall.cuh"
#include "adjoint_x2.cuh"
#include "filter_spectrum.cuh"
#include "conv_tc.cuh"
#include "eddy.cuh"
#include "rhs_x2.cuh"
#include "dfloat.cuh"
#include "rk_df.cuh"

using namespace ins;

// last error message of the calling thread (ins_last_error)
inline thread_local std::string g_err;

namespace {

ins_status fail(ins_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

ins_status cuda_fail(cudaError_t e, const char* where) {
    return fail(INS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define INS_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

#define INS_LAUNCHED(where)                                \
    do {                                                   \
        cudaError_t e_ = cudaGetLastError();               \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

bool factor_radices(int L, std::vector<int>& out) {
    out.clear();
    int e2 = 0;
    while (L % 2 == 0) {
        L /= 2;
        ++e2;
    }
    while (e2 >= 3) {
        out.push_back(8);
        e2 -= 3;
    }
    if (e2 == 2) out.push_back(4);
    if (e2 == 1) out.push_back(2);
    for (int p : {3, 5, 7}) {
        while (L % p == 0) {
            out.push_back(p);
            L /= p;
        }
    }
    return L == 1 && (int)out.size() <= FFT_MAX_STAGES;
}

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct ins_grid {
    int dim = 0, nx = 1, ny = 1, nz = 1, wall_y = 0, dtype = 0, scheme = INS_RK4;
    int march_chunk = 0;      // planes per CTA of the pair kernels (0: chosen from the wave count)
    int fusion = 2;           // FP32 3-D RK4 stage boundaries (ins_set_step_fusion): 0 separate
                              // kernels, 1 fused, 2 fused with two cells per thread
    double nu = 0.0, force[3] = {0, 0, 0};
    cudaStream_t stream = nullptr;
    long N = 0;             // cells
    int nxh = 0;            // nx/2 + 1
    std::vector<double> d[3], h[3], hlo;  // host geometry
    double dmin2_nu = INFINITY;

    // one device allocation, carved into pieces
    void* base = nullptr;
    size_t bytes = 0;
    void* coef = nullptr;          // T[3][C_COUNT][n_a] (per direction contiguous)
    void* coef_df = nullptr;       // the same as double-float pairs (FP64 channels with double-float arithmetic)
    void* ycoef = nullptr;         // T[CY_COUNT][ny]: per-row coefficients of a stretched wall direction
    double* geo64 = nullptr;       // h_x h_y h_z | d_x d_y d_z  (nx+ny+nz each)
    double* one = nullptr;         // a device 1.0 (divisor of an already divided maximum)
    void* tw[3] = {nullptr, nullptr, nullptr};
    int radix[3][FFT_MAX_STAGES];
    int nst[3] = {0, 0, 0};
    void* scale = nullptr;         // T, [nz][ny][nxh] (periodic)
    // double-float arithmetic of the FP64 step (periodic grids with register-FFT lengths): FFT
    // twiddles and the spectral table as (hi, lo) float pairs
    int df_ok = 0;                 // the grid supports it
    int use_df = 0;                // selected (ins_set_f64_arithmetic; default on where supported)
    void* tw_df[3] = {nullptr, nullptr, nullptr};
    void* scale_df = nullptr;
    float* eig = nullptr;          // FP32 periodic: N-scaled eigenvalue sums of the fused pass (see k_fft_strided_pipe)
    double* lam = nullptr;         // FP64 eigenvalues: x (nxh) | y (ny) | z (nz)
    double* th_lo = nullptr;       // Thomas: lo[ny], up[ny]
    double* th_up = nullptr;
    double* th_invm = nullptr;     // [ny][ncol] (FP32 grids: double-float pairs in the same bytes)
    double* th_cp = nullptr;       // [ny][ncol]
    void* th_d = nullptr;          // [ny][ncol] complex FP64 or double-float (16 bytes)
    // DCT-II solve along a uniform wall-normal y (available when y is uniform and ny factorises)
    int wall_dct = 0;              // available
    int use_dct = 0;               // selected (ins_set_wall_solver; default Thomas)
    void* dct_qw = nullptr;        // T complex [ny]: exp(-i pi k / (2 ny))
    void* F = nullptr;
    void* acc = nullptr;
    void* us = nullptr;
    void* rp = nullptr;
    void* pbuf = nullptr;          // FP32 3-D RK4: pressure of the fused stage boundary (r stays in rp)
    void* S = nullptr;
    unsigned long long* cfl_max = nullptr;  // [nx + ny + nz] per-index maxima of |u^a|
    unsigned int* err_flag = nullptr;       // [1]
    double* diag = nullptr;                 // [4]
    unsigned long long* diag_max = nullptr; // [2]
    int lg_tw_x = 0, lg_tw_y = 0, lg_tw_z = 0;
    int kchunk = 32;
    // attached CNN closure (m(u) joins F in rhs, step and step_vjp) and its output buffer
    struct ins_closure* closure = nullptr;
    void* mbuf = nullptr;
    // attached eddy-viscosity model (its term joins F in rhs and step) and its buffers
    int eddy = 0;             // EddyKind
    double eddy_C = 0.0;
    void* eddy_buf = nullptr; // nu_t (N) | term (3N)
    void* eddy_rows = nullptr; // wall y: 1/d_y | 1/h_y | (C D_j)^2 | d_y^2 (ny each, field type)
    // step-VJP workspace (stage states u_2..u_4, the projected cotangent, nu partials),
    // allocated by the first ins_step_vjp call
    void* vjp = nullptr;
    size_t vjp_bytes = 0;
    // CUDA graph of one ins_step, replayed by ins_step_n (captured on a private stream, launched
    // on g->stream); recaptured when the key (pointers, dt, settings) changes
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    unsigned long long step_kernels = 0;   // kernels in the captured step
    std::vector<double> graph_key;
    // launch accounting and opt-in per-kernel CUDA-event timing
    unsigned long long launches = 0;
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    long long prof_dropped = 0;
    std::vector<std::string> names;
    std::vector<int> rec_name;   // per recorded launch: name id (events 2r, 2r+1)
};

struct ins_closure {
    ins_grid* g = nullptr;
    long nvox = 0;
    void* buf = nullptr;
    size_t bytes = 0;
    __nv_bfloat16* wf[4] = {};     // forward weight blobs
    __nv_bfloat16* wt[4] = {};     // data-gradient (transposed) weight blobs
    __nv_bfloat16* x[4] = {};      // layer inputs: x0 (8 ch), x1..x3 (32 ch)
    float* z[3] = {};              // pre-activations of layers 1..3 (32 ch, FP32)
    __nv_bfloat16* ga = nullptr;   // gradient ping-pong buffers (32 ch)
    __nv_bfloat16* gb = nullptr;
    __nv_bfloat16* g4 = nullptr;   // output-side gradient (8 ch)
    const float* bias[4] = {};
    float* gW[4] = {};             // gradient accumulators used by ins_step_vjp
    float* gB[4] = {};
    unsigned int* err = nullptr;
    float* wpart = nullptr;        // partial weight-gradient blocks of k_wgrad_plane (null: not used)
    int params_set = 0;
};

// Closure terms added to F by the step and its pullback (ins_closure.cu; eddy viscosity in ins_eddy.cu).
template <typename T>
ins_status closure_term(ins_grid* g, const T* u, T** m, bool save);
template <typename T>
ins_status closure_pullback(ins_grid* g, const T* w, T* ubar);
template <typename T>
ins_status eddy_term(ins_grid* g, const T* u, T* term);
template <typename T>
ins_status eddy_nut(ins_grid* g, const T* u, T* nut);

namespace {

template <typename T>
Geo<T> make_geo(const ins_grid* g) {
    Geo<T> G;
    G.nx = g->nx;
    G.ny = g->ny;
    G.nz = g->nz;
    G.wall_y = g->wall_y;
    const T* c = reinterpret_cast<const T*>(std::is_same<T, df>::value ? g->coef_df : g->coef);
    G.c[0] = c;
    G.c[1] = c + (size_t)C_COUNT * g->nx;
    G.c[2] = c + (size_t)C_COUNT * (g->nx + g->ny);
    G.fx = (T)g->force[0];
    G.fy = (T)g->force[1];
    G.fz = (T)g->force[2];
    return G;
}

template <typename T>
FftLine<T> make_line(const ins_grid* g, int a) {
    FftLine<T> pl;
    pl.L = a == 0 ? g->nx : (a == 1 ? g->ny : g->nz);
    pl.nst = g->nst[a];
    for (int s = 0; s < FFT_MAX_STAGES; ++s) pl.radix[s] = s < pl.nst ? g->radix[a][s] : 1;
    pl.tw = reinterpret_cast<const cplx<T>*>(std::is_same<T, df>::value ? g->tw_df[a] : g->tw[a]);
    return pl;
}

int prof_begin(ins_grid* g, const char* name) {
    ++g->launches;
    if (!g->prof) return -1;
    if (g->ev_used + 2 > g->ev.size()) {
        ++g->prof_dropped;
        return -1;
    }
    int id = -1;
    for (size_t i = 0; i < g->names.size(); ++i)
        if (g->names[i] == name) id = (int)i;
    if (id < 0) {
        g->names.push_back(name);
        id = (int)g->names.size() - 1;
    }
    const int r = (int)g->rec_name.size();
    g->rec_name.push_back(id);
    cudaEventRecord(g->ev[g->ev_used], g->stream);
    g->ev_used += 2;
    return r;
}

void prof_end(ins_grid* g, int r) { cudaEventRecord(g->ev[2 * (size_t)r + 1], g->stream); }

// Launch a kernel with launch accounting, optional event timing and an error check.
#define KLAUNCH(g, name, ...)                    \
    do {                                         \
        const int pr_ = prof_begin((g), (name)); \
        __VA_ARGS__;                             \
        if (pr_ >= 0) prof_end((g), pr_);        \
        INS_LAUNCHED(name);                      \
    } while (0)

template <typename T>
size_t fft_smem(int L, int lgtw) {
    return 2ull * L * ((1 << lgtw) + 1) * sizeof(cplx<T>);
}

template <typename T>
int choose_lgtw(int L) {
    int lg = sizeof(T) == 8 ? 3 : 4;   // 128-byte rows of complex values
    while (lg > 0 && fft_smem<T>(L, lg) > 100 * 1024) --lg;
    return lg;
}

// ------------------------------------------------------------ Poisson solve
// Register-resident FFT passes for L = R1 R2 in {16, 32, 64, 128, 256}; other lengths use the
// shared-memory Stockham kernels.
// Line lengths of the register FFT kernels. The FP64 x passes of the radix-3 lengths (48, 96,
// 192) stay on the shared-memory Stockham kernel, which measured faster for them (192: 150 vs
// 171 us per pass on the 192 x 128 x 192 channel); the FP64 strided passes and all FP32 passes
// use the register kernels.
bool reg_fft_len(int L, bool fp64_x = false) {
    if (L == 48 || L == 96 || L == 192) return !fp64_x;
    return L == 16 || L == 32 || L == 64 || L == 128 || L == 256;
}

int device_sm_count() {
    static int count = 0;
    if (count == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            count = n;
        else
            count = 148;
    }
    return count;
}

template <typename T, int R1, int R2>
void launch_strided_reg(cudaStream_t st, const cplx<T>* tw, cplx<T>* S, long ncol, long cdiv, long outer,
                        long lstride, int mode, const T* scale) {
    if constexpr (sizeof(T) == 8) {
        // FP64 is bound by the FP64 pipe, not by latency: the one-tile-per-CTA kernel (the
        // pipelined one measured 2 % slower here)
        // one CTA per tile (the double-float square kernels can walk tiles, but as many CTAs as stay
        // resident measured slower: 118.6 against 113.1 us per pass at 256^3)
        using Sh = RegShape<T, R1, R2>;
        const unsigned blocks = (unsigned)((ncol + Sh::TW - 1) / Sh::TW);
        k_fft_strided_reg<T, R1, R2><<<blocks, Sh::NT, 0, st>>>(tw, S, ncol, cdiv, outer, lstride, mode, scale);
    } else {
        // FP32: persistent, double-buffered cp.async variant; the next tile's loads overlap the butterflies
        using Ph = PipeShape<T, R1, R2>;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_fft_strided_pipe<T, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Ph::smem_max());
            attr = true;
        }
        const long ntiles = (ncol + Ph::TW - 1) / Ph::TW;
        const long cap = 2L * device_sm_count();
        const unsigned blocks = (unsigned)(ntiles < cap ? ntiles : cap);
        k_fft_strided_pipe<T, R1, R2><<<blocks, Ph::NT, Ph::smem(mode == 2), st>>>(tw, S, ncol, cdiv, outer, lstride, mode,
                                                                                 scale);
    }
}

template <typename T>
void strided_reg(int L, cudaStream_t st, const cplx<T>* tw, cplx<T>* S, long ncol, long cdiv, long outer,
                 long lstride, int mode, const T* scale) {
    switch (L) {
        case 16: launch_strided_reg<T, 4, 4>(st, tw, S, ncol, cdiv, outer, lstride, mode, scale); break;
        case 32: launch_strided_reg<T, 8, 4>(st, tw, S, ncol, cdiv, outer, lstride, mode, scale); break;
        case 64: launch_strided_reg<T, 8, 8>(st, tw, S, ncol, cdiv, outer, lstride, mode, scale); break;
        case 48: launch_strided_reg<T, 16, 3>(st, tw, S, ncol, cdiv, outer, lstride, mode, scale); break;
        case 96: launch_strided_reg<T, 16, 6>(st, tw, S, ncol, cdiv, outer, lstride, mode, scale); break;
        case 128: launch_strided_reg<T, 16, 8>(st, tw, S, ncol, cdiv, outer, lstride, mode, scale); break;
        case 192: launch_strided_reg<T, 16, 12>(st, tw, S, ncol, cdiv, outer, lstride, mode, scale); break;
        default: launch_strided_reg<T, 16, 16>(st, tw, S, ncol, cdiv, outer, lstride, mode, scale); break;
    }
}

template <typename T, int R1, int R2>
void launch_x_reg(bool forward, cudaStream_t st, const cplx<T>* tw, const T* in, cplx<T>* S, T* out, int lines,
                  int nxh) {
    // FP32 and double-float inverse: persistent double-buffered variant when the spectrum is 16-byte
    // aligned (native FP64 is FP64-pipe bound and keeps the one-tile-per-CTA kernel)
    if constexpr (sizeof(T) == 4 || std::is_same<T, df>::value) {
        if (!forward && reinterpret_cast<uintptr_t>(S) % 16 == 0) {
            using Px = PipeX<T, R1, R2>;
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k_fft_x_c2r_pipe<T, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Px::smem_c2r(Px::L / 2 + 1));
                attr = true;
            }
            const long ntiles = (((long)lines + 1) / 2 + Px::TW - 1) / Px::TW;
            const long cap = 2L * device_sm_count();
            const unsigned blocks = (unsigned)(ntiles < cap ? ntiles : cap);
            k_fft_x_c2r_pipe<T, R1, R2><<<blocks, Px::NT, Px::smem_c2r(nxh), st>>>(tw, S, out, lines, nxh);
            return;
        }
    }
    using Sh = RegShape<T, R1, R2>;
    const long pairs = (lines + 1) / 2;
    const long ntiles = (pairs + Sh::TW - 1) / Sh::TW;
    if (forward) {
        // FP32 and double-float: as many CTAs as stay resident, each walking tiles (FP32: twiddles
        // loaded once per CTA; double-float 256^3: 101.5 against 102.8 us with one CTA per tile)
        long cap = ntiles;
        if (sizeof(T) == 4 || std::is_same<T, df>::value) {
            static int per_sm = 0;
            if (!per_sm) {
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fft_x_r2c_reg<T, R1, R2>, Sh::NT, 0);
                if (per_sm < 1) per_sm = 1;
            }
            cap = (long)per_sm * device_sm_count();
        }
        const unsigned blocks = (unsigned)(ntiles < cap ? ntiles : cap);
        k_fft_x_r2c_reg<T, R1, R2><<<blocks, Sh::NT, 0, st>>>(tw, in, S, lines, nxh);
        return;
    }
    const unsigned blocks = (unsigned)ntiles;
    k_fft_x_c2r_reg<T, R1, R2><<<blocks, Sh::NT, 0, st>>>(tw, S, out, lines, nxh);
}

template <typename T>
void x_reg(int L, bool forward, cudaStream_t st, const cplx<T>* tw, const T* in, cplx<T>* S, T* out, int lines,
           int nxh) {
    switch (L) {
        case 16: launch_x_reg<T, 4, 4>(forward, st, tw, in, S, out, lines, nxh); break;
        case 32: launch_x_reg<T, 8, 4>(forward, st, tw, in, S, out, lines, nxh); break;
        case 64: launch_x_reg<T, 8, 8>(forward, st, tw, in, S, out, lines, nxh); break;
        case 48: launch_x_reg<T, 16, 3>(forward, st, tw, in, S, out, lines, nxh); break;
        case 96: launch_x_reg<T, 16, 6>(forward, st, tw, in, S, out, lines, nxh); break;
        case 128: launch_x_reg<T, 16, 8>(forward, st, tw, in, S, out, lines, nxh); break;
        case 192: launch_x_reg<T, 16, 12>(forward, st, tw, in, S, out, lines, nxh); break;
        default: launch_x_reg<T, 16, 16>(forward, st, tw, in, S, out, lines, nxh); break;
    }
}

// Shared-memory limits of the Stockham FFT kernels. A function attribute set in one translation
// unit does not reach the copy of a template kernel that another unit launches, so every launcher
// calls this first; it sets the attributes once per unit, device and type.
template <typename T>
ins_status set_smem_attrs() {
    static bool done[64] = {};
    int dev = 0;
    INS_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && done[dev]) return INS_OK;
    const int mx = 200 * 1024;   // covers 2 * 2048 * 2 * 16 B (FP64, one line per tile)
    INS_CUDA(cudaFuncSetAttribute(k_fft_x_r2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    INS_CUDA(cudaFuncSetAttribute(k_fft_x_c2r<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    INS_CUDA(cudaFuncSetAttribute(k_fft_strided<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    if constexpr (!std::is_same<T, df>::value)
        INS_CUDA(cudaFuncSetAttribute(k_dct_solve_y<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    if (dev >= 0 && dev < 64) done[dev] = true;
    return INS_OK;
}

// T = df (the double-float FP64 step): the register kernels for their lengths (16 .. 256 powers of
// two, 48, 96, 192), the shared-memory Stockham kernels for the other lengths, with the grid's
// double-float twiddles and spectral table.
template <typename T>
ins_status poisson(ins_grid* g, const T* r, T* p) {
    constexpr bool DF = std::is_same<T, df>::value;
    if (ins_status s0 = set_smem_attrs<T>(); s0 != INS_OK) return s0;
    cudaStream_t st = g->stream;
    const int nx = g->nx, ny = g->ny, nz = g->nz, nxh = g->nxh;
    const long lines = (long)ny * nz;
    cplx<T>* S = reinterpret_cast<cplx<T>*>(g->S);
    FftLine<T> lx = make_line<T>(g, 0);
    if (reg_fft_len(nx, sizeof(T) == 8 && !DF)) {
        KLAUNCH(g, "fft_x_r2c", x_reg<T>(nx, true, st, lx.tw, r, S, nullptr, (int)lines, nxh));
    } else {
        const int lg = g->lg_tw_x;
        const long pairs = (lines + 1) / 2;
        const unsigned blocks = (unsigned)((pairs + (1 << lg) - 1) >> lg);
        KLAUNCH(g, "fft_x_r2c", k_fft_x_r2c<T><<<blocks, FFT_THREADS, fft_smem<T>(nx, lg), st>>>(lx, r, S, (int)lines, nxh, lg));
    }
    auto strided = [&](int a, int mode) -> ins_status {
        FftLine<T> pl = make_line<T>(g, a);
        const int lg = a == 1 ? g->lg_tw_y : g->lg_tw_z;
        long ncol, cdiv, outer, lstride;
        if (a == 1) {
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
            // FP32: the fused pass forms its scale from the eigenvalue sums (no table read)
            const T* sc = sizeof(T) == 4 ? reinterpret_cast<const T*>(g->eig)
                                         : reinterpret_cast<const T*>(DF ? g->scale_df : g->scale);
            KLAUNCH(g, "fft_strided", strided_reg<T>(pl.L, st, pl.tw, S, ncol, cdiv, outer, lstride, mode, sc));
            return INS_OK;
        }
        const unsigned blocks = (unsigned)((ncol + (1 << lg) - 1) >> lg);
        KLAUNCH(g, "fft_strided", k_fft_strided<T><<<blocks, FFT_THREADS, fft_smem<T>(pl.L, lg), st>>>(
            pl, S, ncol, cdiv, outer, lstride, mode, reinterpret_cast<const T*>(DF ? g->scale_df : g->scale), lg));
        return INS_OK;
    };
    ins_status s;
    if (!g->wall_y) {
        if (g->dim == 2) {
            if ((s = strided(1, 2)) != INS_OK) return s;
        } else {
            if ((s = strided(1, 0)) != INS_OK) return s;
            if ((s = strided(2, 2)) != INS_OK) return s;
            if ((s = strided(1, 1)) != INS_OK) return s;
        }
    } else {
        if (g->dim == 3 && (s = strided(2, 0)) != INS_OK) return s;
        const long ncol = (long)nz * nxh;
        const double norm = 1.0 / ((double)nx * (g->dim == 3 ? nz : 1));
        bool dct = false;
        if constexpr (DF) {
            if (g->use_dct) return fail(INS_ERR_UNSUPPORTED, "the DCT wall solve has no double-float pass");
        } else if (g->use_dct) {
            FftLine<T> py = make_line<T>(g, 1);
            const int lg = g->lg_tw_y;
            const unsigned blocks = (unsigned)((ncol + (1 << lg) - 1) >> lg);
            KLAUNCH(g, "dct_solve", k_dct_solve_y<T><<<blocks, FFT_THREADS, fft_smem<T>(ny, lg), st>>>(
                py, S, ncol, nxh, (long)ny * nxh, nxh, reinterpret_cast<const cplx<T>*>(g->dct_qw), g->lam,
                g->lam + nx, g->lam + nx + ny, norm / ny, lg));
            dct = true;
        }
        if (!dct) {
            KLAUNCH(g, "thomas", k_thomas2<T><<<(unsigned)((ncol + TH_COLS - 1) / TH_COLS), 2 * TH_COLS, 0, st>>>(
                S, reinterpret_cast<const typename ThArith<T>::F*>(g->th_lo),
                reinterpret_cast<const typename ThArith<T>::F*>(g->th_up),
                reinterpret_cast<const typename ThArith<T>::F*>(g->th_invm),
                reinterpret_cast<const typename ThArith<T>::F*>(g->th_cp),
                reinterpret_cast<cplx<typename ThArith<T>::A>*>(g->th_d), nxh, ny, ncol));
        }
        if (g->dim == 3 && (s = strided(2, 1)) != INS_OK) return s;
    }
    if (reg_fft_len(nx, sizeof(T) == 8 && !DF)) {
        KLAUNCH(g, "fft_x_c2r", x_reg<T>(nx, false, st, lx.tw, nullptr, S, p, (int)lines, nxh));
    } else {
        const int lg = g->lg_tw_x;
        const long pairs = (lines + 1) / 2;
        const unsigned blocks = (unsigned)((pairs + (1 << lg) - 1) >> lg);
        KLAUNCH(g, "fft_x_c2r", k_fft_x_c2r<T><<<blocks, FFT_THREADS, fft_smem<T>(nx, lg), st>>>(lx, S, p, (int)lines, nxh, lg));
    }
    return INS_OK;
}

// ------------------------------------------------------------ kernels by config
template <typename T>
RhsCoef<T> make_rhs_coef(const ins_grid* g) {
    RhsCoef<T> c;
    c.nx = g->nx;
    c.ny = g->ny;
    c.nz = g->nz;
    double D[3];
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (double w : g->d[a]) s += w;
        D[a] = s / g->d[a].size();
    }
    c.cx = (T)(0.25 / D[0]);
    c.cy = (T)(0.25 / D[1]);
    c.cz = (T)(0.25 / D[2]);
    c.dx = (T)(g->nu / (D[0] * D[0]));
    c.dy = (T)(g->nu / (D[1] * D[1]));
    c.dz = (T)(g->nu / (D[2] * D[2]));
    c.ix = (T)(1.0 / D[0]);
    c.iy = (T)(1.0 / D[1]);
    c.iz = (T)(1.0 / D[2]);
    c.fx = (T)g->force[0];
    c.fy = (T)g->force[1];
    c.fz = (T)g->force[2];
    c.yc = reinterpret_cast<const T*>(g->ycoef);
    c.yc64 = g->dtype == INS_F64 ? reinterpret_cast<const double*>(g->ycoef) : nullptr;
    return c;
}


int device_sm_count();
// z chunk of the pair kernels: the CTAs of a launch run in waves of 2 per SM (their launch
// bounds); a CTA costs about its planes plus two for its prologue (five staged planes without
// an evaluation). Take the chunk that minimises waves x cost per CTA (the last wave counts as a
// full one), or the caller's (ins_set_march_chunk).
// z planes per CTA of a z-marching kernel over `cols` columns: the chunk that minimises
// (waves of `resident` CTAs) x (planes a CTA stages: chunk + halo).
int wave_chunk(long cols, int nz, long resident, int halo) {
    int best_c = nz;
    long best = -1;
    for (int c = 1; c <= nz; ++c) {
        const long ctas = cols * ((nz + c - 1) / c);
        const long cost = (ctas + resident - 1) / resident * (c + halo);
        if (best < 0 || cost < best) {
            best = cost;
            best_c = c;
        }
    }
    return best_c;
}

dim3 pair_grid(const ins_grid* g, int ctas_per_sm = 2) {
    const int nbx = (g->nx + 2 * RBX - 1) / (2 * RBX), nby = (g->ny + RBY - 1) / RBY;
    int kc = g->march_chunk;
    if (kc <= 0) {
        const long resident = (long)ctas_per_sm * device_sm_count();
        long best = -1;
        for (int c = 8; c <= 128; ++c) {
            const long ctas = (long)nbx * nby * ((g->nz + c - 1) / c);
            const long cost = (ctas + resident - 1) / resident * (std::min(c, g->nz) + 2);
            if (best < 0 || cost < best) {
                best = cost;
                kc = c;
            }
            if (c >= g->nz) break;
        }
    }
    kc = std::min(kc, g->nz);
    return dim3(nbx, nby, (g->nz + kc - 1) / kc);
}

// The two-cells-per-thread FP32 kernels (fusion level 2): nx even, 8-byte aligned fields,
// 3 x cells < 2^31.
bool pair_ok(const ins_grid* g, const void* u) {
    return g->fusion == 2 && g->nx % 2 == 0 && 3 * g->N < (1L << 31) && reinterpret_cast<uintptr_t>(u) % 8 == 0;
}

template <bool WALL, bool STAGE, bool STS = false>
ins_status launch_pair(ins_grid* g, const char* name, const float* Fs, const float* p, const float* u0, float* acc,
                       float* F, float* r, const FusedArgs& fa) {
    static bool attr = false;
    if (!attr) {
        INS_CUDA(cudaFuncSetAttribute(k_rhs_div_x2<WALL, STAGE, STS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      PairRegSmem::BYTES));
        attr = true;
    }
    const dim3 grd = pair_grid(g, pair_ctas_per_sm(WALL, STAGE));
    const int kc = (g->nz + grd.z - 1) / grd.z;
    const float* ihy = make_geo<float>(g).c[1] + (size_t)C_INV_H * g->ny;
    KLAUNCH(g, name, (k_rhs_div_x2<WALL, STAGE, STS><<<grd, dim3(RBX, RBY, 1), PairRegSmem::BYTES, g->stream>>>(
                         make_rhs_coef<float>(g), (float)(1.0 / g->h[0][0]), (float)(1.0 / g->h[2][0]), ihy, Fs, p,
                         u0, acc, F, r, fa, kc)));
    return INS_OK;
}

template <typename T, int DIM, bool WALL>
ins_status launch_rhs_div(ins_grid* g, const T* u, T* F, T* r, const T* m = nullptr) {
    if constexpr (DIM == 3 && std::is_same<T, float>::value) {
        if (!m && pair_ok(g, u)) {
            FusedArgs fa{};
            return launch_pair<WALL, false>(g, "rhs_div", nullptr, nullptr, u, nullptr, F, r, fa);
        }
    }
    dim3 blk(RBX, RBY, 1);
    dim3 grd((g->nx + RBX - 1) / RBX, (g->ny + RBY - 1) / RBY, DIM == 3 ? (g->nz + g->kchunk - 1) / g->kchunk : 1);
    KLAUNCH(g, "rhs_div", k_rhs_div<T, DIM, WALL><<<grd, blk, 0, g->stream>>>(make_rhs_coef<T>(g), u, F, r, g->kchunk, m));
    return INS_OK;
}

// F + D F with double-float arithmetic; UI = double for the caller's FP64 field (split by bits
// on load), df for the stage state.
template <int DIM, typename UI, bool WALL = false>
ins_status launch_rhs_div_df(ins_grid* g, const UI* u, df* F, df* r) {
    const dim3 blk(RBX, RBY, 1);
    const dim3 grd((g->nx + RBX - 1) / RBX, (g->ny + RBY - 1) / RBY, DIM == 3 ? (g->nz + g->kchunk - 1) / g->kchunk : 1);
    KLAUNCH(g, "rhs_div", (k_rhs_div<df, DIM, WALL, UI><<<grd, blk, 0, g->stream>>>(make_rhs_coef<df>(g), u, F, r,
                                                                                     g->kchunk, (const df*)nullptr)));
    return INS_OK;
}

template <int DIM, bool LS = false, bool WALL = false>
ins_status rk_update_df(ins_grid* g, const df* F, const df* p, double* u0, df* acc, df* us, const RkArgs& ra,
                        double* uto = nullptr) {
    RkCoefDf c;
    c.nx = g->nx;
    c.ny = g->ny;
    c.nz = g->nz;
    c.ihx = df(1.0 / g->h[0][0]);
    c.ihy = df(1.0 / g->h[1][0]);
    c.ihz = df(DIM == 3 ? 1.0 / g->h[2][0] : 0.0);
    c.ihy_row = WALL ? make_geo<double>(g).c[1] + (size_t)C_INV_H * g->ny : nullptr;
    const int bx = (g->nx / 2 + 31) / 32, by = (g->ny + 7) / 8;
    const int kc = wave_chunk((long)bx * by, g->nz, 4L * device_sm_count(), 1);
    const dim3 grd(bx, by, (g->nz + kc - 1) / kc);
    KLAUNCH(g, "rk_update", (k_rk_update_df<DIM, LS, WALL><<<grd, dim3(32, 8), 0, g->stream>>>(c, F, p, u0, acc, us, ra, kc, uto)));
    return INS_OK;
}

dim3 cell_grid(const ins_grid* g) { return dim3((g->nx + 31) / 32, (g->ny + 7) / 8, g->nz); }

// The vector RK update needs whole 16-byte vectors per row and an aligned caller field.
template <typename T>
bool rk_vec_ok(const ins_grid* g, const void* u) {
    return g->nx % VecT<T>::N == 0 && reinterpret_cast<uintptr_t>(u) % 16 == 0;
}

// Wray's low-storage third-order scheme in two-register form (Butcher tableau a21 = 8/15,
// a31 = 1/4, a32 = 5/12, b = (1/4, 0, 3/4)): u_{s+1} = u_s + dt (gamma_s k_s + zeta_s k_{s-1}).
constexpr double WRAY3_GAMMA[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
constexpr double WRAY3_ZETA[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

template <typename T, int DIM, bool WALL>
struct Impl {
    static ins_status rhs(ins_grid* g, const T* u, T* dudt, T* p) {
        T* F = reinterpret_cast<T*>(g->F);
        T* rp = reinterpret_cast<T*>(g->rp);
        ins_status s;
        T* m = nullptr;
        if ((s = closure_term<T>(g, u, &m, false)) != INS_OK) return s;
        if ((s = launch_rhs_div<T, DIM, WALL>(g, u, F, rp, m)) != INS_OK) return s;
        T* pp = p ? p : rp;
        if ((s = poisson<T>(g, rp, pp)) != INS_OK) return s;
        KLAUNCH(g, "sub_grad", k_sub_grad<T, DIM, WALL><<<cell_grid(g), dim3(32, 8), 0, g->stream>>>(make_geo<T>(g), F, pp, dudt));
        return INS_OK;
    }
    static ins_status project(ins_grid* g, const T* uin, T* uout, T* p) {
        T* rp = reinterpret_cast<T*>(g->rp);
        ins_status s;
        if ((s = div_fast(g, uin, rp)) != INS_OK) return s;
        T* pp = p ? p : rp;
        if ((s = poisson<T>(g, rp, pp)) != INS_OK) return s;
        return sub_grad_fast(g, uin, pp, uout);
    }
    static ins_status divergence(ins_grid* g, const T* u, T* phi) {
        KLAUNCH(g, "divergence", k_divergence<T, DIM, WALL><<<cell_grid(g), dim3(32, 8), 0, g->stream>>>(make_geo<T>(g), u, phi));
        return INS_OK;
    }
    // Vector width of the z-march kernels: VecT<T>::N, or half of it when a row's vector count
    // would leave warps partly idle and the half width fills whole warps (FP32 nx = 192: 48
    // float4 per row, 96 float2).
    static int vec_width(const ins_grid* g) {
        constexpr int V = VecT<T>::N;
        const int nv = g->nx / V;
        return (nv % 32 != 0 && nv < 128 && (g->nx / (V / 2)) % 32 == 0) ? V / 2 : V;
    }
    // z chunk from the wave count of the resident CTAs (the vector kernels keep four 256-thread CTAs
    // per SM; each CTA reads its chunk plus one plane of p or u^z beyond it)
    static dim3 vec_grid(const ins_grid* g, int vw, int* kc) {
        const int bx = (g->nx / vw + 31) / 32, by = (g->ny + 7) / 8;
        const int c = wave_chunk((long)bx * by, g->nz, 4L * device_sm_count(), 1);
        *kc = c;
        return dim3(bx, by, (g->nz + c - 1) / c);
    }
    static RkCoef<T> rk_coef(const ins_grid* g) {
        RkCoef<T> rc;
        rc.nx = g->nx;
        rc.ny = g->ny;
        rc.nz = g->nz;
        rc.ihx = (T)(1.0 / g->h[0][0]);
        rc.ihz = (T)(1.0 / g->h[2][0]);
        rc.ihy = make_geo<T>(g).c[1] + (size_t)C_INV_H * g->ny;
        return rc;
    }
    template <bool LS, int VW>
    static ins_status rk_vec_launch(ins_grid* g, const char* name, const T* F, const T* rp, T* u0, T* acc, T* us,
                                    const RkArgs& ra) {
        int kc;
        const dim3 grd = vec_grid(g, VW, &kc);
        KLAUNCH(g, name, (k_rk_update_vec<T, DIM, WALL, LS, VW><<<grd, dim3(32, 8), 0, g->stream>>>(
                             rk_coef(g), F, rp, u0, acc, us, ra, kc)));
        return INS_OK;
    }
    // Launch the stage update (vector z-march kernel when the rows allow it).
    template <bool LS>
    static ins_status rk_update(ins_grid* g, const T* F, const T* rp, T* u0, T* acc, T* us, const RkArgs& ra) {
        if (rk_vec_ok<T>(g, u0) && (us == nullptr || reinterpret_cast<uintptr_t>(us) % 16 == 0)) {
            constexpr int V = VecT<T>::N;
            if (vec_width(g) == V) return rk_vec_launch<LS, V>(g, "rk_update", F, rp, u0, acc, us, ra);
            return rk_vec_launch<LS, V / 2>(g, "rk_update", F, rp, u0, acc, us, ra);
        }
        KLAUNCH(g, "rk_update", k_rk_update<T, DIM, WALL, LS><<<cell_grid(g), dim3(32, 8), 0, g->stream>>>(
                                    make_geo<T>(g), F, rp, u0, acc, us, ra));
        return INS_OK;
    }
    // phi = D u and out = src - G p through the vector z-march kernels when the rows allow it
    // (the step VJP's P^T and ins_project), else the one-cell kernels.
    template <int VW>
    static ins_status div_vec_launch(ins_grid* g, const T* u, T* phi) {
        DivCoef<T> dc;
        dc.nx = g->nx;
        dc.ny = g->ny;
        dc.nz = g->nz;
        dc.idx = (T)(1.0 / g->d[0][0]);
        dc.idz = (T)(1.0 / g->d[2][0]);
        dc.idy = make_geo<T>(g).c[1] + (size_t)C_INV_D * g->ny;
        int kc;
        const dim3 grd = vec_grid(g, VW, &kc);
        KLAUNCH(g, "divergence", (k_divergence_vec<T, DIM, WALL, VW><<<grd, dim3(32, 8), 0, g->stream>>>(dc, u, phi, kc)));
        return INS_OK;
    }
    static ins_status div_fast(ins_grid* g, const T* u, T* phi) {
        if (rk_vec_ok<T>(g, u) && reinterpret_cast<uintptr_t>(phi) % 16 == 0) {
            constexpr int V = VecT<T>::N;
            return vec_width(g) == V ? div_vec_launch<V>(g, u, phi) : div_vec_launch<V / 2>(g, u, phi);
        }
        KLAUNCH(g, "divergence", (k_divergence<T, DIM, WALL><<<cell_grid(g), dim3(32, 8), 0, g->stream>>>(make_geo<T>(g), u, phi)));
        return INS_OK;
    }
    // The row-scaled P^T passes of the wall-bounded pullback (vector kernels when the rows allow it).
    template <int VW, bool SCL = false>
    static ins_status div_scaled_vec(ins_grid* g, const T* u, T* phi, const double* sdt = nullptr, double sdt_host = 0.0,
                                     double sbeta = 0.0) {
        DivCoef<T> dc;
        dc.nx = g->nx;
        dc.ny = g->ny;
        dc.nz = g->nz;
        dc.idx = (T)(1.0 / g->d[0][0]);
        dc.idz = (T)(1.0 / g->d[2][0]);
        dc.idy = make_geo<T>(g).c[1] + (size_t)C_INV_D * g->ny;
        dc.ihy = make_geo<T>(g).c[1] + (size_t)C_INV_H * g->ny;
        dc.sdt = sdt;
        dc.sdt_host = sdt_host;
        dc.sbeta = sbeta;
        int kc;
        const dim3 grd = vec_grid(g, VW, &kc);
        KLAUNCH(g, "divergence", (k_divergence_vec<T, DIM, WALL, VW, true, SCL><<<grd, dim3(32, 8), 0, g->stream>>>(dc, u, phi, kc)));
        return INS_OK;
    }
    static ins_status div_scaled_fast(ins_grid* g, const T* u, T* phi) {
        if constexpr (WALL) {
            // FP64 keeps the one-cell kernel (its row scalings cost FP64 operations the vector form
            // does not save: 95 vs 109 us on the 192 x 128 x 192 channel)
            if (sizeof(T) == 4 && rk_vec_ok<T>(g, u) && reinterpret_cast<uintptr_t>(phi) % 16 == 0) {
                constexpr int V = VecT<T>::N;
                return vec_width(g) == V ? div_scaled_vec<V>(g, u, phi) : div_scaled_vec<V / 2>(g, u, phi);
            }
            KLAUNCH(g, "divergence", (k_wall_div_scaled<T, DIM><<<cell_grid(g), dim3(32, 8), 0, g->stream>>>(make_geo<T>(g), u, phi)));
        }
        return INS_OK;
    }
    template <int VW, bool SCL = false>
    static ins_status sub_scaled_vec(ins_grid* g, const T* src, const T* p, T* out, const double* hy, const double* dy,
                                     const double* sdt = nullptr, double sdt_host = 0.0, double sbeta = 0.0) {
        RkCoef<T> rc = rk_coef(g);
        rc.idy = make_geo<T>(g).c[1] + (size_t)C_INV_D * g->ny;
        rc.hy = hy;
        rc.dy = dy;
        RkArgs ra;
        ra.dt_dev = sdt;
        ra.dt_host = sdt_host;
        ra.a_next = 0.0;
        ra.b = sbeta;   // SCL: src is read as (dt b) src
        ra.stage = -1;
        ra.last = 0;
        ra.mx = nullptr;
        ra.err_flag = g->err_flag;
        int kc;
        const dim3 grd = vec_grid(g, VW, &kc);
        KLAUNCH(g, "sub_grad", (k_rk_update_vec<T, DIM, WALL, false, VW, true, SCL><<<grd, dim3(32, 8), 0, g->stream>>>(
                                   rc, src, p, nullptr, nullptr, out, ra, kc)));
        return INS_OK;
    }
    static ins_status sub_scaled_fast(ins_grid* g, const T* src, const T* p, T* out, const double* hy, const double* dy) {
        if constexpr (WALL) {
            if (sizeof(T) == 4 && rk_vec_ok<T>(g, src) && reinterpret_cast<uintptr_t>(out) % 16 == 0 &&
                reinterpret_cast<uintptr_t>(p) % 16 == 0) {
                constexpr int V = VecT<T>::N;
                return vec_width(g) == V ? sub_scaled_vec<V>(g, src, p, out, hy, dy)
                                         : sub_scaled_vec<V / 2>(g, src, p, out, hy, dy);
            }
            KLAUNCH(g, "sub_grad",
                    (k_wall_sub_scaled<T, DIM><<<cell_grid(g), dim3(32, 8), 0, g->stream>>>(make_geo<T>(g), src, p, out, hy, dy)));
        }
        return INS_OK;
    }
    // The step VJP's first P^T passes on (dt beta) ybar without forming it: vector kernels only
    // (the caller checks rk_vec_ok on ybar and the alignment of the outputs).
    template <int VW>
    static ins_status div_fold_vec(ins_grid* g, const T* y, T* phi, const double* dt_dev, double dt_host, double beta) {
        DivCoef<T> dc;
        dc.nx = g->nx;
        dc.ny = g->ny;
        dc.nz = g->nz;
        dc.idx = (T)(1.0 / g->d[0][0]);
        dc.idz = (T)(1.0 / g->d[2][0]);
        dc.idy = make_geo<T>(g).c[1] + (size_t)C_INV_D * g->ny;
        dc.sdt = dt_dev;
        dc.sdt_host = dt_host;
        dc.sbeta = beta;
        int kc;
        const dim3 grd = vec_grid(g, VW, &kc);
        KLAUNCH(g, "divergence", (k_divergence_vec<T, DIM, WALL, VW, false, true><<<grd, dim3(32, 8), 0, g->stream>>>(
                                     dc, y, phi, kc)));
        return INS_OK;
    }
    template <int VW>
    static ins_status sub_fold_vec(ins_grid* g, const T* y, const T* p, T* out, const double* dt_dev, double dt_host,
                                   double beta) {
        RkArgs ra;
        ra.dt_dev = dt_dev;
        ra.dt_host = dt_host;
        ra.a_next = 0.0;
        ra.b = beta;
        ra.stage = -1;
        ra.last = 0;
        ra.mx = nullptr;
        ra.err_flag = g->err_flag;
        int kc;
        const dim3 grd = vec_grid(g, VW, &kc);
        KLAUNCH(g, "sub_grad", (k_rk_update_vec<T, DIM, WALL, false, VW, false, true><<<grd, dim3(32, 8), 0, g->stream>>>(
                                   rk_coef(g), y, p, nullptr, nullptr, out, ra, kc)));
        return INS_OK;
    }
    static ins_status sub_grad_fast(ins_grid* g, const T* src, const T* p, T* out) {
        if (rk_vec_ok<T>(g, src) && reinterpret_cast<uintptr_t>(out) % 16 == 0 && reinterpret_cast<uintptr_t>(p) % 16 == 0) {
            RkArgs ra;
            ra.dt_dev = nullptr;
            ra.dt_host = 0.0;
            ra.a_next = 0.0;
            ra.b = 0.0;
            ra.stage = -1;   // out = src - G p only
            ra.last = 0;
            ra.mx = nullptr;
            ra.err_flag = g->err_flag;
            constexpr int V = VecT<T>::N;
            if (vec_width(g) == V) return rk_vec_launch<false, V>(g, "sub_grad", src, p, nullptr, nullptr, out, ra);
            return rk_vec_launch<false, V / 2>(g, "sub_grad", src, p, nullptr, nullptr, out, ra);
        }
        KLAUNCH(g, "sub_grad", (k_sub_grad<T, DIM, WALL><<<cell_grid(g), dim3(32, 8), 0, g->stream>>>(make_geo<T>(g), src, p, out)));
        return INS_OK;
    }
    // defined in impl_step.cuh (RK4, Wray3, FP32 fused stage boundaries)
    static ins_status step_wray3(ins_grid* g, T* u, const double* dt_dev, double dt_host, double* next_dt,
                                 double cfl);
    static ins_status step_fused(ins_grid* g, T* u, const double* dt_dev, double dt_host, double* next_dt,
                                 double cfl);
    static ins_status step(ins_grid* g, T* u, const double* dt_dev, double dt_host, double* next_dt, double cfl);
    // defined in impl_vjp.cuh
    static ins_status step_vjp_wall(ins_grid* g, const T* un, const double* dt_dev, double dt_host, const T* ybar,
                                    T* ubar, double* nubar);
    static ins_status step_vjp(ins_grid* g, const T* un, const double* dt_dev, double dt_host, const T* ybar, T* ubar,
                               double* nubar);
    // defined in impl_diag.cuh
    static ins_status spectrum(ins_grid* g, const T* u, double* E, int kmax);
    static ins_status cfl(ins_grid* g, const T* u, double cfl, double* dt_dev);
    static ins_status diag(ins_grid* g, const T* u, double out[4]);
};

template <typename T, typename Fn>
ins_status dispatch(ins_grid* g, Fn fn) {
    if (g->dim == 2) {
        if (g->wall_y) return fn(Impl<T, 2, true>());
        return fn(Impl<T, 2, false>());
    }
    if (g->wall_y) return fn(Impl<T, 3, true>());
    return fn(Impl<T, 3, false>());
}

template <typename Fn>
ins_status dispatch_dtype(ins_grid* g, Fn fn) {
    if (g->dtype == INS_F64) return fn((double)0);
    return fn((float)0);
}

// ------------------------------------------------------------ creation helpers
template <typename T>
void fill_coefs(const ins_grid* g, std::vector<T>& out) {
    const int n3[3] = {g->nx, g->ny, g->nz};
    out.clear();
    for (int a = 0; a < 3; ++a) {
        const int n = n3[a];
        std::vector<double> c((size_t)C_COUNT * n, 0.0);
        if (a < g->dim) {
            const auto& d = g->d[a];
            const auto& h = g->h[a];
            const bool wall = (a == 1 && g->wall_y);
            for (int i = 0; i < n; ++i) {
                const double dn = (i + 1 < n) ? d[i + 1] : (wall ? d[n - 1] : d[0]);
                const double hp = (i > 0) ? h[i - 1] : g->hlo[a];
                c[C_INV_H * n + i] = 1.0 / h[i];
                c[C_INV_D * n + i] = 1.0 / d[i];
                c[C_CONV_AA * n + i] = 0.25 / h[i];
                c[C_CONV_AB * n + i] = 0.5 / d[i];
                c[C_WL * n + i] = d[i] / (d[i] + dn);
                c[C_WR * n + i] = dn / (d[i] + dn);
                c[C_DIFF_AP * n + i] = g->nu / (dn * h[i]);
                c[C_DIFF_AM * n + i] = g->nu / (d[i] * h[i]);
                c[C_DIFF_BP * n + i] = g->nu / (h[i] * d[i]);
                c[C_DIFF_BM * n + i] = g->nu / (hp * d[i]);
            }
        }
        for (double v : c) out.push_back((T)v);
    }
}

template <typename T>
ins_status upload_twiddles(ins_grid* g, int a, void* dst, int L) {
    std::vector<T> tw(2 * (size_t)L);
    for (int m = 0; m < L; ++m) {
        const double ang = 2.0 * M_PI * (double)m / (double)L;
        tw[2 * m] = (T)std::cos(ang);
        tw[2 * m + 1] = (T)(-std::sin(ang));
    }
    INS_CUDA(cudaMemcpy(dst, tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice));
    return INS_OK;
}

}  // namespace

inline ins_status check_ptr(const ins_grid* g, const void* p, const char* name) {
    if (!p) return fail(INS_ERR_ARG, std::string(name) + " is null");
    const size_t al = g->dtype == INS_F64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(p) % al) return fail(INS_ERR_ARG, std::string(name) + " is misaligned");
    return INS_OK;
}

#define CHECK(x)                        \
    do {                                \
        ins_status s_ = (x);            \
        if (s_ != INS_OK) return s_;    \
    } while (0)

