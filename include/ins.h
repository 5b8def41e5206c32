/*
 * ins.h -- C ABI of libins, the B300 (sm_103a) explicit Runge-Kutta step of the
 * staggered-grid (MAC) finite-volume incompressible Navier-Stokes solver of
 * arXiv 2604.18536 ("A differentiable software suite for accelerated
 * simulation of turbulent flows").
 *
 * Problem (paper Sec. 2.3 and 2.6.1):  du/dt = F(u) - G p,  D u = 0,
 * with L p = D F(u), L = D G, and F(u) = C(u) + nu * diffusion(u) + f.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Cells i in [0, nx), j in [0, ny), k in [0, nz) (nz = 1 in 2-D). Every scalar
 *   field is one contiguous array of nx*ny*nz values, x fastest:
 *   index = (k*ny + j)*nx + i. No ghost cells are stored.
 * - A velocity field is dim such arrays back to back (u^x, u^y[, u^z]).
 *   u^a[i,j,k] lives on the face to the right of cell (i,j,k) in direction a
 *   (Sec. 3.1 convention); p lives at cell centres.
 * - A wall-normal direction (only y may be a wall, x and z then periodic)
 *   stores u^y on the faces above cells 0..ny-1; the last one is the top wall
 *   and holds 0. The bottom wall face is not stored.
 * - Field values are float (INS_F32) or double (INS_F64), as chosen when the
 *   grid was created. Every field pointer is a DEVICE pointer, 16-byte aligned,
 *   owned by the caller. The library never allocates or frees caller buffers.
 * - Calls that launch kernels enqueue them on the grid's stream and return
 *   without synchronising, unless stated otherwise. All argument checks happen
 *   before any launch; on an error nothing is enqueued.
 * - No C++ exception crosses this boundary. Errors return a status code and a
 *   message readable with ins_last_error() (per calling thread).
 */
#ifndef INS_H
#define INS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    INS_OK = 0,
    INS_ERR_ARG = 1,          /* null pointer, bad size, misaligned pointer, bad enum  */
    INS_ERR_UNSUPPORTED = 2,  /* valid request this library does not implement        */
    INS_ERR_OOM = 3,          /* device workspace allocation failed                    */
    INS_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed           */
    INS_ERR_NONFINITE = 5,    /* a NaN/Inf was detected in a result                    */
    INS_ERR_TIMEOUT = 6       /* reserved: no call in this library waits on the device */
} ins_status;

typedef enum { INS_PERIODIC = 0, INS_WALL = 1 } ins_bc;
typedef enum { INS_F32 = 0, INS_F64 = 1 } ins_dtype;
typedef enum { INS_RK4 = 0, INS_WRAY3 = 1 } ins_scheme;

/* Grid description (Sec. 2.1, 2.4, 2.5).
 * dim            2 or 3.
 * n[a]           cells per direction (n[2] ignored in 2-D). Periodic directions
 *                need n[a] = 2^p 3^q 5^r 7^s and n[a] <= 2048 (the FFT radices and
 *                shared-memory line tiles); a wall direction needs n[a] <= 4096.
 * bc[a]          INS_PERIODIC or INS_WALL. Supported: all periodic, or y = WALL
 *                with x (and z) periodic. Other combinations: INS_ERR_UNSUPPORTED.
 * face_coords[a] HOST pointer to n[a]+1 increasing face coordinates, copied at
 *                creation. Periodic directions must be uniformly spaced (the
 *                Poisson solver is spectral there); a wall direction may be
 *                stretched (e.g. the tanh grid of Sec. 2.5).
 * dtype          storage and arithmetic type of the fields.
 * nu             kinematic viscosity (> 0 not required; >= 0).
 * force[a]       constant body force f^a (App. A momentum equation).
 * scheme         time integrator of ins_step (Sec. 2.6.2; 0 = INS_RK4 when the struct is
 *                zero-initialised): INS_RK4, the classic 4-stage RK (three velocity
 *                registers of workspace: F, stage state, accumulator), or INS_WRAY3, Wray's
 *                3-stage third-order low-storage RK (Sec. 3.3, low-storage methods; two
 *                registers: F and the previous stage derivative). */
typedef struct {
    int dim;
    int n[3];
    int bc[3];
    const double* face_coords[3];
    int dtype;
    double nu;
    double force[3];
    int scheme;
} ins_grid_desc;

typedef struct ins_grid ins_grid;

/* Message of the last failed call on this thread ("" if none). Never NULL. */
const char* ins_last_error(void);

/* Library version string. */
const char* ins_version(void);

/* Create a grid: validates *desc, copies the geometry to the device, builds the
 * FFT twiddle tables, the spectral inverse-Laplacian table (periodic) or the
 * Thomas factors (wall direction), and allocates the workspace (about 11 scalar
 * fields of the grid dtype in 3-D with INS_RK4, 8 with INS_WRAY3). stream is a cudaStream_t (NULL = legacy default
 * stream) on which every later call enqueues its work; the current CUDA device
 * must be the one the fields live on. This call synchronises the device. */
ins_status ins_grid_create(const ins_grid_desc* desc, void* stream, ins_grid** out);

/* Free the workspace and the handle (synchronises the grid's stream). NULL is a no-op. */
ins_status ins_grid_destroy(ins_grid* g);

/* Change the stream later calls enqueue on. */
ins_status ins_set_stream(ins_grid* g, void* stream);

/* Bytes of device workspace the grid holds. */
ins_status ins_workspace_bytes(const ins_grid* g, size_t* bytes);

/* Right-hand side of the semi-discrete system (Sec. 2.3, momentum equation):
 * dudt = F(u) - G p with L p = D F(u) (Sec. 2.6.1). u, dudt: dim fields; p:
 * one field or NULL. Wall faces of dudt are 0. */
ins_status ins_rhs(ins_grid* g, const void* u, void* dudt, void* p);

/* Divergence-free projection (Sec. 2.6.1): u_out = u_in - G p with
 * L p = D u_in. u_out may equal u_in. p may be NULL. */
ins_status ins_project(ins_grid* g, const void* u_in, void* u_out, void* p);

/* Divergence (App. B divergence kernel): phi = D u. */
ins_status ins_divergence(ins_grid* g, const void* u, void* phi);

/* One time step of the grid's scheme with a projection at every stage (Sec. 2.6.2);
 * every stage derivative is k_s = F(u_s) - G p_s with L p_s = D F(u_s).
 * INS_RK4: u_s = u_0 + dt a_{s,s-1} k_{s-1}, u_{n+1} = u_0 + dt (k_1/6 + k_2/3 + k_3/3 + k_4/6).
 * INS_WRAY3 (Butcher tableau a21 = 8/15, a31 = 1/4, a32 = 5/12, b = (1/4, 0, 3/4)), run in its
 * two-register form u_{s+1} = u_s + dt (gamma_s k_s + zeta_s k_{s-1}) with
 * gamma = (8/15, 5/12, 3/4), zeta = (0, -17/60, -5/12).
 * u           in/out, dim fields (the step is done in place).
 * dt_dev      DEVICE pointer to one double holding dt, read by the kernels
 *             (no host synchronisation); NULL: dt_host is used.
 * next_dt_dev DEVICE pointer or NULL. If given, receives the CFL time step of
 *             u_{n+1} (see ins_cfl_dt) with factor cfl. It may equal dt_dev
 *             (adaptive stepping entirely on the device).
 * A non-finite value in u_{n+1} sets the grid's error flag (ins_check_finite). */
ins_status ins_step(ins_grid* g, void* u, const double* dt_dev, double dt_host,
                    double* next_dt_dev, double cfl);

/* nsteps consecutive ins_step calls with the same arguments (device-side dt: pass the same
 * pointer as dt_dev and next_dt_dev to advance with the adaptive time step). The first step
 * runs as plain launches; the following ones replay a CUDA graph of one step (captured once on
 * a private stream and launched on g's stream; recaptured when u, the dt arguments, cfl, the
 * stream or a setting of g changes), which removes the per-kernel launch gaps. Results equal
 * nsteps ins_step calls bit for bit. Falls back to plain launches when the step cannot be
 * captured. INS_ERR_ARG for nsteps < 0 and the argument errors of ins_step. */
ins_status ins_step_n(ins_grid* g, void* u, int nsteps, const double* dt_dev, double dt_host, double* next_dt_dev,
                      double cfl);

/* Wall-normal pressure solve of a channel grid (Sec. 2.6.1 and 6): after the x and z FFTs,
 * INS_WALL_THOMAS solves the tridiagonal y system of every (kx, kz) mode in FP64 (any
 * spacing); INS_WALL_DCT diagonalises it with a DCT-II (uniform spacing only: the Neumann
 * rows' eigenvectors are cos(pi k (2j+1)/(2 ny))), computed by one complex FFT of length ny
 * (ny = 2^p 3^q 5^r 7^s <= 2048) and divided by the eigenvalue sum in FP64. Every grid starts
 * with INS_WALL_THOMAS (on this GPU it is faster: two O(ny) sweeps against two FFTs per line).
 * The two give the same velocities; the pressure's mean-mode constant differs (DCT: zero
 * mean, Thomas: p = 0 in the first row of the mean mode). INS_ERR_UNSUPPORTED: no wall
 * direction, or DCT on a grid that does not allow it. */
typedef enum { INS_WALL_THOMAS = 0, INS_WALL_DCT = 1 } ins_wall_solver;
ins_status ins_set_wall_solver(ins_grid* g, int solver);

/* Stage-boundary fusion of ins_step (no counterpart in the paper: an implementation
 * choice). On FP32 3-D INS_RK4 grids without a closure, ins_step by default runs the update
 * of stage s and the evaluation of F and D F of stage s + 1 as one kernel, so the stage
 * state is never stored (the workspace holds one extra scalar field for it); results equal
 * the unfused path's up to the order of FP32 roundings in F. enable = 0 selects the unfused
 * kernels (for comparison), 1 the fused kernels with one cell per thread, 2 (default) the
 * fused kernels with two neighbouring x cells per thread (8-byte accesses; same arithmetic
 * per cell as 1). Other values: INS_ERR_ARG. Other grids ignore the setting. On FP32 3-D
 * periodic grids with even nx, level 2 also selects the two-cells-per-thread pullback
 * stencil of ins_step_vjp (levels 0 and 1: one cell per thread); its results equal the
 * one-cell kernel's up to the order of FP32 roundings. */
ins_status ins_set_step_fusion(ins_grid* g, int enable);

/* Arithmetic of the FP64 step (Sec. 7.3: FP64 is the DNS precision; the arithmetic that
 * reaches it is an implementation choice). INS_ARITH_NATIVE evaluates F, D F, the FFTs of
 * the Poisson solve and the stage updates in FP64 instructions. INS_ARITH_DOUBLE_FLOAT (the
 * default where the grid supports it) evaluates them in double-float arithmetic -- each value
 * the unevaluated sum of two FP32 numbers, about 48 significant bits, error-free
 * transformations on the FP32 pipe -- because this GPU issues FP32 operations 62 times
 * faster than FP64 ones. Storage stays FP64: the caller's velocity is read and written as
 * FP64, the last stage adds the step's increment to it in FP64, and the CFL time step is
 * reduced from the FP64 result exactly as in native mode (bit-identical to the FP64 rule).
 * The step's relative field error against the FP64 oracle stays within the FP64 tolerance
 * (1e-12 per step). It is used by ins_step / ins_step_n (classic RK4 and Wray3; on 3-D
 * channels with the Thomas wall-normal solve) and ins_step_vjp (3-D periodic grids; 3-D
 * channels with classic RK4; the state cotangent accumulates in FP64), without an attached
 * closure or eddy-viscosity model; every other call (ins_rhs, ins_project, 2-D pullbacks, the
 * Wray3 pullback or the DCT solve on a channel, grids with a closure) runs native FP64.
 * Supported grids: FP64, nx even, and either every direction periodic or a 3-D channel
 * (walls in y); elsewhere the setter returns INS_ERR_UNSUPPORTED and the grid stays native.
 * INS_ERR_ARG for other modes. */
typedef enum { INS_ARITH_NATIVE = 0, INS_ARITH_DOUBLE_FLOAT = 1 } ins_arith;
ins_status ins_set_f64_arithmetic(ins_grid* g, int mode);
ins_status ins_get_f64_arithmetic(const ins_grid* g, int* mode);

/* Launch shape of the fused two-cells-per-thread kernels (fusion level 2; no counterpart in
 * the paper): each CTA marches `planes` consecutive z planes of its 64 x 8 column. 0 (default)
 * chooses the chunk from the grid and the number of SMs; results do not depend on it.
 * INS_ERR_ARG for planes < 0. */
ins_status ins_set_march_chunk(ins_grid* g, int planes);

/* Vector-Jacobian product of one ins_step (Sec. 3.4, pullback of a composition;
 * App. B operator pullbacks; the Poisson solve is self-adjoint, Sec. 2.6.1).
 * With u_{n+1} = step(u_n) for a frozen dt, returns
 *   ubar_n = (d u_{n+1} / d u_n)^T ubar_np1   and   *nubar_dev += (d u_{n+1}/d nu) . ubar_np1.
 * The stage states are recomputed from u_n (per-step checkpointing: the caller keeps
 * only the step inputs), then the stages run in reverse: w_s = P kbar_s (P = P^T),
 * ubar_s = J_F(u_s)^T w_s, ubar_n = ubar_np1 + sum_s ubar_s,
 * kbar_{s-1} = dt b_{s-1} ubar_np1 + dt a_{s,s-1} ubar_s (INS_RK4). For INS_WRAY3 the
 * state cotangents chain, Ubar_s = Ubar_{s+1} + ubar_s, and
 * kbar_{s-1} = dt gamma_{s-1} Ubar_s + dt zeta_s Ubar_{s+1} (Ubar_4 = ubar_np1).
 * u_n, ubar_np1: DEVICE, dim fields, not modified. ubar_n: DEVICE, dim fields, must not
 * alias the inputs. dt_dev/dt_host: as in ins_step. nubar_dev: DEVICE double that the
 * result is added to (so it can accumulate over steps), or NULL.
 * Periodic uniform grids use P^T = P and gather-form transposed stencils. Wall-bounded grids
 * (y a no-slip wall, possibly stretched) use P^T = M Omega P Omega^-1 M (Omega the velocity
 * volumes; M zeroes the stored top wall faces of u^y, which are not unknowns: cotangents
 * there are ignored and ubar_n is 0 there) and gather-form transposes (each output value is
 * summed by one thread in a fixed order, no atomics, so repeated calls return the same bits).
 * The first call allocates the
 * step-VJP workspace (3 stage states, two fields, nu partial sums: about 5 velocity fields),
 * kept until ins_grid_destroy; make the first call before any stream capture.
 * The grid's F, r/p and RK accumulator buffers are reused as scratch. */
ins_status ins_step_vjp(ins_grid* g, const void* u_n, const double* dt_dev, double dt_host,
                        const void* ubar_np1, void* ubar_n, double* nubar_dev);

/* Adaptive time step (Sec. 2.6.2, convective and diffusive limits):
 * dt = cfl * min(1 / max_{a,I} |u^a_I| / h_a[i], min_{a,i} d_a[i]^2 / nu)
 * where d are cell widths and h centre-to-centre distances, every operation
 * an IEEE FP64 operation (bit-reproducible). Writes one double to dt_dev. */
ins_status ins_cfl_dt(ins_grid* g, const void* u, double cfl, double* dt_dev);

/* Diagnostics of a velocity field, synchronous. out[0] = kinetic energy
 * (1/|Omega|) 1/2 sum_a sum_I |Omega^a_I| (u^a_I)^2 (FP64 sums); out[1] =
 * max |D u|; out[2] = max |u^a|/h_a; out[3] = number of non-finite values.
 * Returns INS_ERR_NONFINITE (after filling out) if out[3] > 0. */
ins_status ins_diag(ins_grid* g, const void* u, double out[4]);

/* Shell energy spectrum (the closure's error measure; filtered-DNS comparison, Sec. 4):
 * E[k] = sum over wavevectors with floor(|kvec| + 1/2) = k of
 *        1/2 sum_a |uhat_a(kvec)|^2 / Ncells^2, k = 0 .. kmax, uhat the unnormalised DFT,
 * |kvec| in integer wavenumbers (FP64 shell decisions). E_dev: DEVICE, kmax+1 doubles,
 * overwritten. Periodic grids only. Uses the grid's spectral workspace. */
ins_status ins_spectrum(ins_grid* g, const void* u, double* E_dev, int kmax);

/* Channel statistics along the wall-normal y (Sec. 6.2: mean velocity and Reynolds stresses
 * from velocities interpolated to the volume centres, uc_a = (u^a_I + u^a_{I-e_a})/2, the
 * wall value 0 below the first cell for u^y): plane averages over x and z in FP64.
 * out_dev: DEVICE, 9*ny doubles, out[q*ny + j]: q = 0..2 mean u^x, u^y, u^z; q = 3..8 the
 * covariances <uc_a uc_b> - <uc_a><uc_b> for (a,b) = xx, xy, xz, yy, yz, zz.
 * 3-D grids with a wall in y only. */
ins_status ins_wall_profiles(ins_grid* g, const void* u, double* out_dev);

/* Face-averaging filter from a fine grid to one `ratio` times coarser in every
 * direction (filtered DNS for closure training, Sec. 4): the coarse u^a on the face to
 * the right of coarse cell I is the mean of the ratio^(dim-1) fine u^a on the fine faces
 * that tile it. A divergence-free fine field stays divergence free on the coarse grid.
 * n_coarse: coarse cells per direction (host); u_fine: DEVICE, dim fine fields
 * (n_coarse*ratio cells each); u_coarse: DEVICE, dim coarse fields; FP64 sums. */
ins_status ins_filter_face_average(int dim, const int n_coarse[3], int ratio, int dtype, const void* u_fine,
                                   void* u_coarse, void* stream);

/* Reads and clears the grid's device error flag (synchronous).
 * INS_ERR_NONFINITE if a step produced a NaN/Inf since the last check. */
ins_status ins_check_finite(ins_grid* g);

/* CFL time step without a grid handle and without any device allocation.
 * The paper has no counterpart: this is a library convenience for callers that
 * cannot call cudaMalloc (for example code under a memory manager that has
 * reserved nearly all device memory for its own pool, or a plug-in that must
 * keep the device footprint fixed); ins_grid_create, and so ins_cfl_dt, needs
 * cudaMalloc. Result: the same double as ins_cfl_dt on a grid built from *desc
 * (bit for bit). desc: as for ins_grid_create (only dim, n, bc, face_coords,
 * dtype and nu are read; n[a] <= 4096 per direction, else INS_ERR_ARG with a
 * message naming the limit). u: DEVICE velocity field; dt_dev: DEVICE double;
 * stream: cudaStream_t the work is enqueued on.
 * Scratch: a static device array of 192 KiB inside the library (per-index
 * maxima and spacings), held by every GPU that loads the library until the
 * process exits; the call itself allocates and frees nothing. Loading is not
 * free, though: CUDA loads the library's device code and this array into a
 * device's memory lazily, at the first call into the library on that device
 * (this entry point or any other), and that load takes device memory (the
 * code of every kernel plus the 192 KiB). A caller whose memory manager is
 * about to reserve nearly all device memory should therefore make its first
 * call on each device before the pool takes that memory. The first call on
 * each device also looks up that array's device address (cudaGetSymbolAddress);
 * make this first call before any stream capture. Every call shares the array
 * and clears what must start at zero, so calls whose work overlaps on the GPU
 * (other streams, other host threads on the same device) race: serialise them.
 * The spacings are staged in a host buffer of the calling thread and copied
 * with cudaMemcpyAsync from that pageable memory; such a copy has consumed its
 * source when it returns, so the next call may reuse the buffer. */
ins_status ins_cfl_dt_noalloc(const ins_grid_desc* desc, const void* u, double cfl, double* dt_dev,
                              void* stream);

/* ---------------------------------------------------------------- CNN closure
 * A learned closure term m(u) inside F (Sec. 4: neural-network closure models in the
 * right-hand side, trained a posteriori through the unrolled solver). Architecture
 * (a choice; the paper names none): 4 circular 3x3x3 convolutions 3->32->32->32->3,
 * GELU (erf form) after the first three; input channels u^x, u^y, u^z at one storage
 * index, output channel a added to F^a. BF16 weights and activations, FP32 accumulation
 * on the tensor cores (tcgen05) for the forward, the data gradient and the weight gradient.
 * Grids: 3-D, periodic, nx % 8 == 0, ny % 16 == 0, nz >= 2 (else INS_ERR_UNSUPPORTED). */
typedef struct ins_closure ins_closure;

/* Allocate a closure's workspace for grid g (weights blobs, activations). */
ins_status ins_closure_create(ins_grid* g, ins_closure** out);
ins_status ins_closure_destroy(ins_closure* c);

/* Weights W[l]: DEVICE float [27][cin][cout] (tap t = 9(dz+1) + 3(dy+1) + (dx+1),
 * y[co](v) = b[co] + sum_t sum_ci W[t][ci][co] x[ci](v + (dx, dy, dz))), rounded to BF16
 * here; biases b[l]: DEVICE float [cout], read at every use. Call again after every
 * weight update. */
ins_status ins_closure_set_params(ins_closure* c, const float* const W[4], const float* const b[4]);

/* m = closure(u): u and m DEVICE, dim fields of the grid dtype. save != 0 keeps the
 * pre-activations for a following ins_closure_bwd. */
ins_status ins_closure_fwd(ins_grid* g, ins_closure* c, const void* u, void* m, int save);

/* ubar_accum += (dm/du)^T mbar; dW[l] += dL/dW[l], db[l] += dL/db[l] (DEVICE float arrays
 * shaped like W and b; arrays or entries may be NULL). Uses the activations of the last
 * ins_closure_fwd with save != 0. */
ins_status ins_closure_bwd(ins_grid* g, ins_closure* c, const void* mbar, void* ubar_accum, float* const dW[4],
                           float* const db[4]);

/* Where ins_step_vjp accumulates the closure's weight and bias gradients (NULL: not kept). */
ins_status ins_closure_set_grads(ins_closure* c, float* const dW[4], float* const db[4]);

/* Copies (synchronously) the saved BF16 input of layer l (channels-last, 8 channels for
 * l = 0, else 32) and its FP32 pre-activation (32 channels, l < 3) into DEVICE buffers
 * given by the caller (either may be NULL), for inspection. */
ins_status ins_closure_saved(ins_closure* c, int layer, void* x_bf16, float* z);

/* INS_ERR_TIMEOUT if a bounded tensor-core wait gave up since the last check (synchronous). */
ins_status ins_closure_check(ins_closure* c);

/* Attach a closure to g (NULL detaches): ins_rhs, ins_step and ins_step_vjp then use
 * F(u) + m(u). The first attachment allocates one velocity field for m. */
ins_status ins_set_closure(ins_grid* g, ins_closure* c);

/* ---------------------------------------------------------------- eddy-viscosity closures
 * Classical LES closures (App. "Eddy-viscosity models"; the baselines next to the learned
 * closure, Sec. 4 and 6.3). With a model attached, ins_rhs and ins_step add to F the
 * eddy-viscous stress divergence e^a = sum_b delta_b(2 nu_t S_ab), which dissipates energy.
 * S_aa sits at the cell centres, S_ab (a != b) on the cell edges; nu_t is evaluated at the
 * cell centres from the velocity gradient A (off-diagonal entries: mean of the four edge
 * differences around the cell) and averaged from the four neighbouring cells onto an edge.
 * Filter width D = (d_x d_y d_z)^(1/3), per row on a stretched wall-normal axis. Across a
 * wall in y the velocity takes the forward operator's ghosts (odd tangential, zero
 * wall-normal) and nu_t the even ghost (the mirrored cell's value). Models (S = sym A):
 *   INS_EDDY_SMAGORINSKY  nu_t = (C D)^2 sqrt(2 S:S)                    (paper: C = 0.1)
 *   INS_EDDY_WALE         (C D)^2 (Sd:Sd)^(3/2) / ((S:S)^(5/2) + (Sd:Sd)^(5/4)),
 *                         Sd = sym(A A) - tr(A A)/3 I                    (C = 0.5)
 *   INS_EDDY_QR           (C D)^2 |tr(S^3)/3| / (S:S / 2)               (C = sqrt(3/2)/pi)
 *   INS_EDDY_VREMAN       C^2 sqrt(B_beta / (tr(A A^T)/2)),
 *                         beta_ij = sum_m d_m^2 A_im A_jm               (C = sqrt(2.5 * 0.1^2))
 *   INS_EDDY_CONSTANT     nu_t = C (no counterpart in the paper: a diagnostic model for which
 *                         the term equals C (diffusion + G D) u)
 * nu_t = 0 where the model's denominator vanishes. */
typedef enum {
    INS_EDDY_NONE = 0,
    INS_EDDY_SMAGORINSKY = 1,
    INS_EDDY_WALE = 2,
    INS_EDDY_QR = 3,
    INS_EDDY_VREMAN = 4,
    INS_EDDY_CONSTANT = 5
} ins_eddy_model;

/* Attach model with constant C (INS_EDDY_NONE detaches). 3-D grids (periodic, or walls in y)
 * with n >= 2 (INS_ERR_UNSUPPORTED otherwise, and while a CNN closure is attached). The first
 * attachment allocates four scalar fields (nu_t and the term) and, on a wall grid, four rows
 * of ny coefficients, uploaded by a blocking copy (a set-up call: not while g's stream is
 * being captured). ins_step_vjp returns INS_ERR_UNSUPPORTED while a model is attached. */
ins_status ins_set_eddy_viscosity(ins_grid* g, int model, double C);

/* nu_t of the attached model at every cell centre: u DEVICE, dim fields; nut DEVICE, one
 * field of the grid dtype. INS_ERR_ARG without an attached model. */
ins_status ins_eddy_viscosity(ins_grid* g, const void* u, void* nut);

/* ---------------------------------------------------------------- measurement
 * Tracing support (the paper describes none; these calls serve benchmarking). */

/* Number of kernels this grid has launched since creation (every call above
 * that launches work counts each kernel once). */
ins_status ins_launch_count(const ins_grid* g, unsigned long long* n);

/* Per-kernel timing with CUDA events recorded on the grid's stream around every
 * launch (off by default). Enabling creates an event pool of 8192 launches;
 * read the profile before it fills. Enabling again clears pending records. */
ins_status ins_profile_enable(ins_grid* g, int on);

typedef struct {
    char name[32];        /* kernel family, e.g. "rhs_div", "fft_strided"     */
    long long launches;   /* launches recorded since the last read              */
    double total_ms;      /* sum of their event-measured durations             */
} ins_kernel_stat;

/* Synchronises the stream, fills up to cap entries, sets *n_out, and clears the
 * records. INS_ERR_ARG if launches were dropped because the pool was full. */
ins_status ins_profile_read(ins_grid* g, ins_kernel_stat* out, int cap, int* n_out);

/* Measures the device's dependent-FMA throughput for dtype (INS_F32/INS_F64)
 * with a ~0.1 s kernel on stream, in FLOP/s (one FMA = 2 FLOP). Allocates and
 * frees a small scratch buffer; synchronous. */
ins_status ins_measure_fma_rate(int dtype, void* stream, double* flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* INS_H */
