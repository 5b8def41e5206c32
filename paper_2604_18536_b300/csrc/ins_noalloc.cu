#include "ins_internal.cuh"

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

