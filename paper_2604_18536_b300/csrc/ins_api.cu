// libins: C ABI over the B300 kernels (declarations and contracts in include/ins.h).
//
// The grid handle owns: per-direction stencil coefficients (field dtype), FP64
// geometry for the exact CFL rule and diagnostics, FFT twiddle tables, the
// spectral inverse-Laplacian table (all-periodic grids) or the FP64 Thomas
// factors (wall-normal y), and the step workspace (F, RK accumulator, stage
// state, r/p and the half spectrum). Nothing is allocated after creation.
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

using namespace ins;

namespace {

thread_local std::string g_err;

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
    void* ycoef = nullptr;         // T[CY_COUNT][ny]: per-row coefficients of a stretched wall direction
    double* geo64 = nullptr;       // h_x h_y h_z | d_x d_y d_z  (nx+ny+nz each)
    double* one = nullptr;         // a device 1.0 (divisor of an already divided maximum)
    void* tw[3] = {nullptr, nullptr, nullptr};
    int radix[3][FFT_MAX_STAGES];
    int nst[3] = {0, 0, 0};
    void* scale = nullptr;         // T, [nz][ny][nxh] (periodic)
    float* eig = nullptr;          // FP32 periodic: N-scaled eigenvalue sums of the fused pass (see k_fft_strided_pipe)
    double* lam = nullptr;         // FP64 eigenvalues: x (nxh) | y (ny) | z (nz)
    double* th_lo = nullptr;       // Thomas: lo[ny], up[ny]
    double* th_up = nullptr;
    double* th_invm = nullptr;     // [ny][ncol]
    double* th_cp = nullptr;       // [ny][ncol]
    void* th_d = nullptr;          // cplx<double> [ny][ncol]
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

namespace {

template <typename T>
Geo<T> make_geo(const ins_grid* g) {
    Geo<T> G;
    G.nx = g->nx;
    G.ny = g->ny;
    G.nz = g->nz;
    G.wall_y = g->wall_y;
    const T* c = reinterpret_cast<const T*>(g->coef);
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
    pl.tw = reinterpret_cast<const cplx<T>*>(g->tw[a]);
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
        using Sh = RegShape<T, R1, R2>;
        const unsigned blocks = (unsigned)((ncol + Sh::TW - 1) / Sh::TW);
        k_fft_strided_reg<T, R1, R2><<<blocks, Sh::NT, 0, st>>>(tw, S, ncol, cdiv, outer, lstride, mode, scale);
        return;
    }
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
    // FP32 inverse: persistent double-buffered variant when the spectrum is 16-byte aligned (FP64 is
    // FP64-pipe bound and keeps the one-tile-per-CTA kernel)
    if (sizeof(T) == 4 && !forward && reinterpret_cast<uintptr_t>(S) % 16 == 0) {
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
    using Sh = RegShape<T, R1, R2>;
    const long pairs = (lines + 1) / 2;
    const long ntiles = (pairs + Sh::TW - 1) / Sh::TW;
    if (forward) {
        // FP32: as many CTAs as stay resident, each walking tiles (twiddles loaded once per CTA)
        long cap = ntiles;
        if (sizeof(T) == 4) {
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

template <typename T>
ins_status poisson(ins_grid* g, const T* r, T* p) {
    cudaStream_t st = g->stream;
    const int nx = g->nx, ny = g->ny, nz = g->nz, nxh = g->nxh;
    const long lines = (long)ny * nz;
    cplx<T>* S = reinterpret_cast<cplx<T>*>(g->S);
    FftLine<T> lx = make_line<T>(g, 0);
    if (reg_fft_len(nx, sizeof(T) == 8)) {
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
            const T* sc = sizeof(T) == 4 ? reinterpret_cast<const T*>(g->eig) : reinterpret_cast<const T*>(g->scale);
            KLAUNCH(g, "fft_strided", strided_reg<T>(pl.L, st, pl.tw, S, ncol, cdiv, outer, lstride, mode, sc));
            return INS_OK;
        }
        const unsigned blocks = (unsigned)((ncol + (1 << lg) - 1) >> lg);
        KLAUNCH(g, "fft_strided", k_fft_strided<T><<<blocks, FFT_THREADS, fft_smem<T>(pl.L, lg), st>>>(
            pl, S, ncol, cdiv, outer, lstride, mode, reinterpret_cast<const T*>(g->scale), lg));
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
        if (g->use_dct) {
            FftLine<T> py = make_line<T>(g, 1);
            const int lg = g->lg_tw_y;
            const unsigned blocks = (unsigned)((ncol + (1 << lg) - 1) >> lg);
            KLAUNCH(g, "dct_solve", k_dct_solve_y<T><<<blocks, FFT_THREADS, fft_smem<T>(ny, lg), st>>>(
                py, S, ncol, nxh, (long)ny * nxh, nxh, reinterpret_cast<const cplx<T>*>(g->dct_qw), g->lam,
                g->lam + nx, g->lam + nx + ny, norm / ny, lg));
        } else {
            KLAUNCH(g, "thomas", k_thomas2<T><<<(unsigned)((ncol + TH_COLS - 1) / TH_COLS), 2 * TH_COLS, 0, st>>>(
                S, g->th_lo, g->th_up, g->th_invm, g->th_cp, reinterpret_cast<cplx<double>*>(g->th_d), nxh, ny, ncol));
        }
        if (g->dim == 3 && (s = strided(2, 1)) != INS_OK) return s;
    }
    if (reg_fft_len(nx, sizeof(T) == 8)) {
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
    return c;
}

template <typename T>
ins_status closure_term(ins_grid* g, const T* u, T** m, bool save);
template <typename T>
ins_status closure_pullback(ins_grid* g, const T* w, T* ubar);

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
    // Wray's low-storage 3-stage RK (two registers: F and k_{s-1}); u is updated in place.
    static ins_status step_wray3(ins_grid* g, T* u, const double* dt_dev, double dt_host, double* next_dt, double cfl) {
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
    static ins_status step_fused(ins_grid* g, T* u, const double* dt_dev, double dt_host, double* next_dt, double cfl) {
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
    static ins_status step(ins_grid* g, T* u, const double* dt_dev, double dt_host, double* next_dt, double cfl) {
        if (g->scheme == INS_WRAY3) return step_wray3(g, u, dt_dev, dt_host, next_dt, cfl);
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
    // Pullback of one RK4 step (uniform periodic grids): recompute the stage states from the
    // checkpoint u_n, then run the stages in reverse (see ins.h, ins_step_vjp).
    // Pullback of one step on a wall-bounded grid: stage recompute as below, P^T = M Omega P
    // Omega^-1 M, J_F^T in gather form (k_adj_rhs_wall_g); the stored top wall faces of u^y are not
    // unknowns (cotangents there are ignored and returned as 0).
    static ins_status step_vjp_wall(ins_grid* g, const T* un, const double* dt_dev, double dt_host, const T* ybar,
                                    T* ubar, double* nubar) {
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
    static ins_status step_vjp(ins_grid* g, const T* un, const double* dt_dev, double dt_host, const T* ybar,
                               T* ubar, double* nubar) {
        if constexpr (WALL) return step_vjp_wall(g, un, dt_dev, dt_host, ybar, ubar, nubar);
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
    // Shell energy spectrum of a periodic field (see ins.h, ins_spectrum).
    static ins_status spectrum(ins_grid* g, const T* u, double* E, int kmax) {
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
    static ins_status cfl(ins_grid* g, const T* u, double cfl, double* dt_dev) {
        // reuse the stage-4 path's reduction: a read-only pass
        INS_CUDA(cudaMemsetAsync(g->diag, 0, 4 * sizeof(double), g->stream));
        INS_CUDA(cudaMemsetAsync(g->diag_max, 0, 2 * sizeof(unsigned long long), g->stream));
        KLAUNCH(g, "diag", k_diag<T, DIM, WALL><<<cell_grid(g), dim3(32, 8), 0, g->stream>>>(
                               make_geo<T>(g), u, g->geo64, g->diag, g->diag_max));
        // max |u^a|/h_a was reduced into diag_max[1]; finish on the device
        KLAUNCH(g, "cfl_finalize", k_cfl_finalize<<<1, 256, 0, g->stream>>>(g->diag_max + 1, g->one, 1, g->dmin2_nu, cfl, dt_dev));
        return INS_OK;
    }
    static ins_status diag(ins_grid* g, const T* u, double out[4]) {
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
ins_status set_smem_attrs() {
    const int mx = 200 * 1024;   // covers 2 * 2048 * 2 * 16 B (FP64, one line per tile)
    INS_CUDA(cudaFuncSetAttribute(k_fft_x_r2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    INS_CUDA(cudaFuncSetAttribute(k_fft_x_c2r<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    INS_CUDA(cudaFuncSetAttribute(k_fft_strided<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    INS_CUDA(cudaFuncSetAttribute(k_dct_solve_y<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    return INS_OK;
}

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

// =================================================================== C ABI
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
    g->geo64 = reinterpret_cast<double*>(b + o_geo);
    g->one = reinterpret_cast<double*>(b + o_one);
    for (int a = 0; a < 3; ++a) g->tw[a] = b + o_tw[a];
    g->lam = reinterpret_cast<double*>(b + o_lam);
    g->dct_qw = g->wall_dct ? b + o_qw : nullptr;
    g->eig = neig ? reinterpret_cast<float*>(b + o_eig) : nullptr;
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

ins_status ins_workspace_bytes(const ins_grid* g, size_t* bytes) {
    if (!g || !bytes) return fail(INS_ERR_ARG, "null argument");
    *bytes = g->bytes;
    return INS_OK;
}

static ins_status check_ptr(const ins_grid* g, const void* p, const char* name) {
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
                                     (double)g->eddy, g->eddy_C, (double)reinterpret_cast<uintptr_t>(g->closure),
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


// =====================================================================
// CNN closure (see include/ins.h, ins_closure_*)
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

namespace {
constexpr int CL_CIN[4] = {3, 32, 32, 32};
constexpr int CL_COUT[4] = {32, 32, 32, 3};
// blob geometry (N rows, KG channel groups) of the forward and transposed weights
constexpr int CL_FN[4] = {32, 32, 32, 16}, CL_FKG[4] = {2, 4, 4, 4};
constexpr int CL_TN[4] = {16, 32, 32, 32}, CL_TKG[4] = {4, 4, 4, 2};

template <int CG, int N, int EPI>
size_t conv_smem() {
    constexpr int KG = CG == 1 ? 2 : CG;
    return (size_t)CG * CV_CGS + 27 * (size_t)N * KG * 16;
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
    // about one wave of two CTAs per SM: each CTA loads the weights once for ~nz*cols/296 tiles
    // (measured faster than a strictly single wave of longer chunks, which leaves SMs with one CTA)
    const int cols = (g->nx / CV_TX) * (g->ny / CV_TY);
    const int slots = 2 * device_sm_count();
    int zc = (int)(((long)cols * g->nz + slots - 1) / slots);
    zc = zc < 2 ? 2 : (zc > g->nz ? g->nz : zc);
    a.zchunk = zc;
    const dim3 grd(g->nx / CV_TX, g->ny / CV_TY, (g->nz + zc - 1) / zc);
    KLAUNCH(g, "conv3d_tc", k_conv3d_tc<CG, N, EPI><<<grd, CV_THREADS, conv_smem<CG, N, EPI>(), g->stream>>>(a));
    return INS_OK;
}

// Grid of k_wgrad_plane: 16 x 8 columns, z chunks for about one CTA per SM.
dim3 wgrad_plane_grid(const ins_grid* g, int* zchunk) {
    const long cols = (long)(g->nx / WP_TX) * (g->ny / WP_TY);
    const long sms = device_sm_count();
    int zc = (int)((cols * g->nz + sms - 1) / sms);
    zc = zc < 1 ? 1 : (zc > g->nz ? g->nz : zc);
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
            KLAUNCH(g, "wgrad", (k_wgrad_plane<CY><<<grd, 256, WpShape<N>::SMEM, g->stream>>>(
                                    X, dY, g->nx, g->ny, g->nz, cout, zc, part, db, err)));
            const int ncta = (int)(grd.x * grd.y * grd.z);
            KLAUNCH(g, "wgrad_reduce", k_wgrad_reduce<<<(27 * 32 * cout + 255) / 256, 256, 0, g->stream>>>(
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
    KLAUNCH(g, "wgrad", k_wgrad_tc<CX, CY><<<dim3(ngroups, (unsigned)nchunk), WG_THREADS, WgShape<N>::SMEM, g->stream>>>(
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

extern "C" {

ins_status ins_closure_create(ins_grid* g, ins_closure** out);
}  // extern "C"

namespace {
// m(u) of the attached closure into the grid's closure buffer (*m = null when none is attached).
dim3 eddy_grid(const ins_grid* g) { return dim3((g->nx + 31) / 32, (g->ny + 7) / 8, g->nz); }

template <typename T>
EddyCoef<T> eddy_coef(const ins_grid* g) {
    EddyCoef<T> c;
    c.nx = g->nx;
    c.ny = g->ny;
    c.nz = g->nz;
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) {
        const double d = g->d[a][0];
        c.id[a] = (T)(1.0 / d);
        c.w2[a] = (T)(d * d);
        vol *= d;
    }
    const double D = std::cbrt(vol);
    c.CD2 = (T)((g->eddy_C * D) * (g->eddy_C * D));
    c.C2 = (T)(g->eddy == EDDY_CONSTANT ? g->eddy_C : g->eddy_C * g->eddy_C);
    const T* rows = reinterpret_cast<const T*>(g->eddy_rows);
    c.idy = rows;
    c.ihy = rows ? rows + g->ny : nullptr;
    c.cd2y = rows ? rows + 2 * g->ny : nullptr;
    c.w2y = rows ? rows + 3 * g->ny : nullptr;
    return c;
}

// The per-row wall-normal coefficients of the attached model, in the field type.
template <typename T>
cudaError_t eddy_upload_rows(ins_grid* g) {
    const int ny = g->ny;
    std::vector<T> v(4 * (size_t)ny);
    for (int j = 0; j < ny; ++j) {
        const double dy = g->d[1][j];
        const double D = std::cbrt(g->d[0][0] * dy * g->d[2][0]);
        v[j] = (T)(1.0 / dy);
        v[ny + j] = (T)(1.0 / g->h[1][j]);
        v[2 * ny + j] = (T)((g->eddy_C * D) * (g->eddy_C * D));
        v[3 * ny + j] = (T)(dy * dy);
    }
    return cudaMemcpy(g->eddy_rows, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T, bool WALL>
ins_status eddy_nut_launch(ins_grid* g, const T* u, T* nut) {
    const EddyCoef<T> c = eddy_coef<T>(g);
    const dim3 grd = eddy_grid(g), blk(32, 8);
    switch (g->eddy) {
        case EDDY_SMAGORINSKY:
            KLAUNCH(g, "eddy_nut", (k_eddy_nut<T, EDDY_SMAGORINSKY, WALL><<<grd, blk, 0, g->stream>>>(c, u, nut)));
            break;
        case EDDY_WALE: KLAUNCH(g, "eddy_nut", (k_eddy_nut<T, EDDY_WALE, WALL><<<grd, blk, 0, g->stream>>>(c, u, nut))); break;
        case EDDY_QR: KLAUNCH(g, "eddy_nut", (k_eddy_nut<T, EDDY_QR, WALL><<<grd, blk, 0, g->stream>>>(c, u, nut))); break;
        case EDDY_VREMAN:
            KLAUNCH(g, "eddy_nut", (k_eddy_nut<T, EDDY_VREMAN, WALL><<<grd, blk, 0, g->stream>>>(c, u, nut)));
            break;
        default:
            KLAUNCH(g, "eddy_nut", (k_eddy_nut<T, EDDY_CONSTANT, WALL><<<grd, blk, 0, g->stream>>>(c, u, nut)));
            break;
    }
    return INS_OK;
}

template <typename T>
ins_status eddy_nut(ins_grid* g, const T* u, T* nut) {
    if (g->wall_y) return eddy_nut_launch<T, true>(g, u, nut);
    return eddy_nut_launch<T, false>(g, u, nut);
}

template <typename T>
ins_status closure_term(ins_grid* g, const T* u, T** m, bool save) {
    *m = nullptr;
    if (g->eddy) {
        T* nut = reinterpret_cast<T*>(g->eddy_buf);
        T* term = nut + g->N;
        ins_status s = eddy_nut<T>(g, u, nut);
        if (s != INS_OK) return s;
        if (g->wall_y)
            KLAUNCH(g, "eddy_div",
                    (k_eddy_div<T, true><<<eddy_grid(g), dim3(32, 8), 0, g->stream>>>(eddy_coef<T>(g), u, nut, term)));
        else
            KLAUNCH(g, "eddy_div",
                    (k_eddy_div<T, false><<<eddy_grid(g), dim3(32, 8), 0, g->stream>>>(eddy_coef<T>(g), u, nut, term)));
        *m = term;
        return INS_OK;
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
}  // namespace

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

ins_status ins_set_eddy_viscosity(ins_grid* g, int model, double C) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    if (model < INS_EDDY_NONE || model > INS_EDDY_CONSTANT) return fail(INS_ERR_ARG, "unknown eddy-viscosity model");
    if (model == INS_EDDY_NONE) {
        g->eddy = 0;
        return INS_OK;
    }
    if (!(std::isfinite(C) && C >= 0.0)) return fail(INS_ERR_ARG, "C must be finite and >= 0");
    if (g->dim != 3) return fail(INS_ERR_UNSUPPORTED, "eddy-viscosity models: 3-D grids only");
    if (g->nx < 2 || g->ny < 2 || g->nz < 2) return fail(INS_ERR_UNSUPPORTED, "eddy-viscosity models need n >= 2");
    if (g->closure) return fail(INS_ERR_UNSUPPORTED, "a CNN closure is attached (one closure at a time)");
    if (!g->eddy_buf) {
        const size_t bytes = (size_t)4 * g->N * (g->dtype == INS_F64 ? 8 : 4);
        cudaError_t e = cudaMalloc(&g->eddy_buf, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g->eddy_buf = nullptr;
            return fail(INS_ERR_OOM, "eddy-viscosity buffers");
        }
    }
    if (g->wall_y) {
        if (!g->eddy_rows) {
            cudaError_t e = cudaMalloc(&g->eddy_rows, (size_t)4 * g->ny * (g->dtype == INS_F64 ? 8 : 4));
            if (e != cudaSuccess) {
                cudaGetLastError();
                g->eddy_rows = nullptr;
                return fail(INS_ERR_OOM, "eddy-viscosity row coefficients");
            }
        }
        g->eddy_C = C;
        cudaError_t e = g->dtype == INS_F64 ? eddy_upload_rows<double>(g) : eddy_upload_rows<float>(g);
        if (e != cudaSuccess) return fail(INS_ERR_CUDA, cudaGetErrorString(e));
    }
    g->eddy = model;
    g->eddy_C = C;
    return INS_OK;
}

ins_status ins_eddy_viscosity(ins_grid* g, const void* u, void* nut) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    CHECK(check_ptr(g, u, "u"));
    if (!nut) return fail(INS_ERR_ARG, "nut is null");
    if (!g->eddy) return fail(INS_ERR_ARG, "no eddy-viscosity model attached");
    if (g->dtype == INS_F64) return eddy_nut<double>(g, (const double*)u, (double*)nut);
    return eddy_nut<float>(g, (const float*)u, (float*)nut);
}

}  // extern "C"

// =====================================================================
// ins_cfl_dt_noalloc: the CFL time step without a grid handle and without
// any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc -- for example code that
// runs under a memory manager (such as a framework's caching allocator) which
// has already reserved nearly all device memory for its own pool, so a
// cudaMalloc would fail or take memory the pool counts on, or a plug-in inside
// another application that must keep the device memory footprint fixed.
// ins_grid_create allocates the grid's workspace with cudaMalloc, so such
// callers cannot use ins_cfl_dt.
//
// The scratch of the reduction -- the per-index maxima of |u^a| and the FP64
// centre-to-centre distances h_a, both laid out [x: nx | y: ny | z: nz] -- lives
// in one file-scope static device array of fixed size (NOALLOC_NMAX cells per
// direction, 192 KiB), which every GPU that loads this library holds until
// the process exits. The maxima are cleared at the start of every call (and
// again by k_cfl_finalize). Every call shares the array: calls whose work
// overlaps on the GPU (different streams, or different host threads on the
// same device) race and may return wrong time steps.
namespace {

constexpr int NOALLOC_NMAX = 4096;
constexpr int NOALLOC_MAXDEV = 64;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[6 * NOALLOC_NMAX];
std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_ptr[NOALLOC_MAXDEV] = {nullptr};
thread_local double g_noalloc_h[3 * NOALLOC_NMAX];

// Per-index maxima of |u^a| over the other indices (read-only variant of the
// stage-4 reduction of k_rk_update). Block (32, 8); grid (ceil(nx/32), ceil(ny/8), nz).
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_cfl_absmax(int nx, int ny, int nz, const T* __restrict__ u,
                                                    unsigned long long* __restrict__ mx) {
    const long N = (long)nx * ny * nz;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    double q[3] = {0.0, 0.0, 0.0};
    if (i < nx && j < ny) {
        const long a = ((long)k * ny + j) * nx + i;
#pragma unroll
        for (int c = 0; c < DIM; ++c) q[c] = fabs((double)u[c * N + a]);
    }
    __shared__ double sx[8][33];
    const int lane = threadIdx.x, row = threadIdx.y;
    sx[row][lane] = q[0];
    double qy = q[1];
    for (int o = 16; o > 0; o >>= 1) qy = fmax(qy, __shfl_xor_sync(0xffffffffu, qy, o));
    if (lane == 0 && j < ny && qy > 0.0) atomicMax(&mx[nx + j], (unsigned long long)__double_as_longlong(qy));
    double qz = q[2];
    for (int o = 16; o > 0; o >>= 1) qz = fmax(qz, __shfl_xor_sync(0xffffffffu, qz, o));
    if (lane == 0) sx[row][32] = qz;
    __syncthreads();
    if (row == 0) {
        double m = sx[0][lane];
        for (int r = 1; r < 8; ++r) m = fmax(m, sx[r][lane]);
        if (i < nx && m > 0.0) atomicMax(&mx[i], (unsigned long long)__double_as_longlong(m));
        if (DIM == 3 && lane == 0) {
            double z = sx[0][32];
            for (int r = 1; r < 8; ++r) z = fmax(z, sx[r][32]);
            if (z > 0.0) atomicMax(&mx[nx + ny + k], (unsigned long long)__double_as_longlong(z));
        }
    }
}

// Device address of the static scratch on the current device, looked up once per device.
ins_status noalloc_scratch(unsigned long long** out) {
    int dev = 0;
    INS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAXDEV) return fail(INS_ERR_UNSUPPORTED, "device ordinal >= 64");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(static CFL scratch)");
        g_noalloc_ptr[dev] = reinterpret_cast<unsigned long long*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return INS_OK;
}

}  // namespace

extern "C" ins_status ins_cfl_dt_noalloc(const ins_grid_desc* desc, const void* u, double cfl, double* dt_dev,
                                         void* stream) {
    g_err.clear();
    if (!desc || !u || !dt_dev) return fail(INS_ERR_ARG, "ins_cfl_dt_noalloc: null argument");
    const ins_grid_desc& D = *desc;
    if (D.dim != 2 && D.dim != 3) return fail(INS_ERR_ARG, "dim must be 2 or 3");
    if (D.dtype != INS_F32 && D.dtype != INS_F64) return fail(INS_ERR_ARG, "dtype must be INS_F32 or INS_F64");
    if (!(std::isfinite(cfl) && cfl > 0.0)) return fail(INS_ERR_ARG, "cfl must be finite and > 0");
    if (!(D.nu >= 0.0) || !std::isfinite(D.nu)) return fail(INS_ERR_ARG, "nu must be finite and >= 0");
    if (reinterpret_cast<uintptr_t>(u) % (D.dtype == INS_F64 ? 8 : 4)) return fail(INS_ERR_ARG, "u is misaligned");
    if (reinterpret_cast<uintptr_t>(dt_dev) % 8) return fail(INS_ERR_ARG, "dt_dev is misaligned");
    int n3[3] = {1, 1, 1};
    for (int a = 0; a < D.dim; ++a) {
        if (D.n[a] < 2) return fail(INS_ERR_ARG, "n[a] must be >= 2");
        if (D.n[a] > NOALLOC_NMAX)
            return fail(INS_ERR_ARG,
                        "ins_cfl_dt_noalloc: n[a] exceeds the static scratch limit of 4096 cells per direction");
        if (D.bc[a] != INS_PERIODIC && D.bc[a] != INS_WALL) return fail(INS_ERR_ARG, "bc must be PERIODIC or WALL");
        if (!D.face_coords[a]) return fail(INS_ERR_ARG, "face_coords[a] is null");
        n3[a] = D.n[a];
    }
    // FP64 h on the host (periodic: wrap; wall: mirrored ghost), laid out [x | y | z]
    const int nsum = n3[0] + n3[1] + n3[2];
    double dmin = INFINITY;
    int off = 0;
    for (int a = 0; a < 3; ++a) {
        const int n = n3[a];
        for (int i = 0; i < n; ++i) {
            double hv = 1.0;
            if (a < D.dim) {
                const double* f = D.face_coords[a];
                const double w = f[i + 1] - f[i];
                if (!(w > 0.0) || !std::isfinite(w)) return fail(INS_ERR_ARG, "face coordinates must increase");
                dmin = std::fmin(dmin, w);
                const double wn = (i + 1 < n) ? f[i + 2] - f[i + 1] : (D.bc[a] == INS_WALL ? w : f[1] - f[0]);
                hv = 0.5 * (w + wn);
            }
            g_noalloc_h[off + i] = hv;
        }
        off += n;
    }
    const double dmin2_nu = D.nu > 0.0 ? dmin * dmin / D.nu : INFINITY;
    unsigned long long* scr = nullptr;
    CHECK(noalloc_scratch(&scr));
    unsigned long long* mx = scr;
    double* hd = reinterpret_cast<double*>(scr + 3 * NOALLOC_NMAX);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    INS_CUDA(cudaMemcpyAsync(hd, g_noalloc_h, sizeof(double) * nsum, cudaMemcpyHostToDevice, st));
    INS_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * nsum, st));
    const dim3 grd((n3[0] + 31) / 32, (n3[1] + 7) / 8, n3[2]);
    if (D.dtype == INS_F64) {
        if (D.dim == 3) k_cfl_absmax<double, 3><<<grd, dim3(32, 8), 0, st>>>(n3[0], n3[1], n3[2], (const double*)u, mx);
        else k_cfl_absmax<double, 2><<<grd, dim3(32, 8), 0, st>>>(n3[0], n3[1], n3[2], (const double*)u, mx);
    } else {
        if (D.dim == 3) k_cfl_absmax<float, 3><<<grd, dim3(32, 8), 0, st>>>(n3[0], n3[1], n3[2], (const float*)u, mx);
        else k_cfl_absmax<float, 2><<<grd, dim3(32, 8), 0, st>>>(n3[0], n3[1], n3[2], (const float*)u, mx);
    }
    INS_LAUNCHED("cfl_absmax (static scratch)");
    k_cfl_finalize<<<1, 256, 0, st>>>(mx, hd, nsum, dmin2_nu, cfl, dt_dev);
    INS_LAUNCHED("cfl_finalize (static scratch)");
    return INS_OK;
}
