"""Python face of libins: torch tensors in, pointers out. Argument marshalling only.

Every computation runs in the CUDA kernels of libins; PyTorch only owns the
device memory and the stream. A velocity field is a tensor of shape
(dim, nz, ny, nx) in 3-D or (dim, ny, nx) in 2-D (x fastest), contiguous, on
the grid's device and in the grid's dtype; a scalar field drops the first axis.
"""

import ctypes
import math

import numpy as np
import torch

from . import _lib
from ._lib import GridDesc, check, lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def measure_fma_rate(dtype=torch.float64, device=None):
    """Dependent-FMA throughput of the current device in FLOP/s (ins_measure_fma_rate)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    out = ctypes.c_double()
    with torch.cuda.device(dev):
        st = torch.cuda.current_stream(dev).cuda_stream
        check(lib().ins_measure_fma_rate(_lib.INS_F64 if dtype == torch.float64 else _lib.INS_F32,
                                         ctypes.c_void_p(st), ctypes.byref(out)), "ins_measure_fma_rate")
    return out.value


def filter_face_average(u_fine, ratio):
    """Face-averaging filter to a grid `ratio` times coarser (ins_filter_face_average).

    u_fine: CUDA tensor (dim, [nz,] ny, nx), float32 or float64; returns the coarse field."""
    dim = u_fine.shape[0]
    fine = tuple(reversed(u_fine.shape[1:]))
    if any(n % ratio for n in fine) or not u_fine.is_contiguous() or not u_fine.is_cuda:
        raise ValueError("fine sizes must be multiples of ratio; contiguous CUDA tensor expected")
    nc = [n // ratio for n in fine] + [1] * (3 - len(fine))
    out = torch.empty((dim,) + tuple(reversed(nc[:dim])), dtype=u_fine.dtype, device=u_fine.device)
    arr = (ctypes.c_int * 3)(*nc)
    dt = _lib.INS_F64 if u_fine.dtype == torch.float64 else _lib.INS_F32
    st = torch.cuda.current_stream(u_fine.device).cuda_stream
    check(lib().ins_filter_face_average(dim, arr, int(ratio), dt, _ptr(u_fine), _ptr(out), ctypes.c_void_p(st)),
          "ins_filter_face_average")
    return out


class Grid:
    """A staggered grid and its device workspace (``ins_grid_create``).

    faces: list of dim 1-D arrays of face coordinates (n_a + 1 each, host FP64)
    bc:    list of "periodic" | "wall" (only y may be a wall)
    nu, force: viscosity and constant body force
    dtype: torch.float32 or torch.float64
    scheme: "rk4" (classic RK4) or "wray3" (Wray's low-storage third-order RK)
    """

    SCHEMES = {"rk4": _lib.INS_RK4, "wray3": _lib.INS_WRAY3}

    def __init__(self, faces, bc, nu, force=None, dtype=torch.float64, device=None, scheme="rk4"):
        self.dim = len(faces)
        if scheme not in self.SCHEMES:
            raise ValueError(f"scheme must be one of {sorted(self.SCHEMES)}")
        self.scheme = scheme
        self.faces = [np.ascontiguousarray(f, dtype=np.float64) for f in faces]
        self.n = tuple(len(f) - 1 for f in self.faces)
        self.shape = tuple(reversed(self.n))
        self.bc = list(bc)
        self.nu = float(nu)
        self.force = [0.0] * self.dim if force is None else [float(x) for x in force]
        if dtype not in (torch.float32, torch.float64):
            raise ValueError("dtype must be torch.float32 or torch.float64")
        self.dtype = dtype
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        d = GridDesc()
        d.dim = self.dim
        for a in range(3):
            d.n[a] = self.n[a] if a < self.dim else 1
            d.bc[a] = (_lib.INS_WALL if self.bc[a] == "wall" else _lib.INS_PERIODIC) if a < self.dim else 0
            d.face_coords[a] = (self.faces[a].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                                if a < self.dim else None)
            d.force[a] = self.force[a] if a < self.dim else 0.0
        d.dtype = _lib.INS_F64 if dtype == torch.float64 else _lib.INS_F32
        d.nu = self.nu
        d.scheme = self.SCHEMES[scheme]
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().ins_grid_create(ctypes.byref(d), ctypes.c_void_p(self._stream()), ctypes.byref(h)),
                  "ins_grid_create")
        self._h = h

    # ------------------------------------------------------------ plumbing
    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def _sync_stream(self):
        check(lib().ins_set_stream(self._h, ctypes.c_void_p(self._stream())), "ins_set_stream")

    def _check_u(self, u, name="u"):
        want = (self.dim,) + self.shape
        if tuple(u.shape) != want or u.dtype != self.dtype or not u.is_cuda or not u.is_contiguous():
            raise ValueError(f"{name}: expected contiguous {self.dtype} CUDA tensor of shape {want}, got "
                             f"{tuple(u.shape)} {u.dtype} {u.device}")

    def _check_p(self, p, name="p"):
        if tuple(p.shape) != self.shape or p.dtype != self.dtype or not p.is_cuda or not p.is_contiguous():
            raise ValueError(f"{name}: expected contiguous {self.dtype} CUDA tensor of shape {self.shape}")

    def close(self):
        if getattr(self, "_h", None):
            lib().ins_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_velocity(self):
        return torch.zeros((self.dim,) + self.shape, dtype=self.dtype, device=self.device)

    def new_scalar(self):
        return torch.zeros(self.shape, dtype=self.dtype, device=self.device)

    # model constants of the paper's channel LES (Sec. 6.3)
    EDDY_DEFAULT_C = {"smagorinsky": 0.1, "wale": 0.5, "qr": math.sqrt(1.5) / math.pi,
                      "vreman": math.sqrt(2.5 * 0.1 ** 2)}

    def set_eddy_viscosity(self, model, C=None):
        """Attach an eddy-viscosity closure ("smagorinsky", "wale", "qr", "vreman", "constant") or
        detach it (None / "none"); C defaults to the paper's constant (ins_set_eddy_viscosity)."""
        name = "none" if model is None else model
        if name not in _lib.INS_EDDY:
            raise ValueError(f"model must be one of {sorted(_lib.INS_EDDY)}")
        c = self.EDDY_DEFAULT_C.get(name, 0.0) if C is None else float(C)
        check(lib().ins_set_eddy_viscosity(self._h, _lib.INS_EDDY[name], c), "ins_set_eddy_viscosity")
        self.eddy = None if name == "none" else (name, c)

    def eddy_viscosity(self, u, out=None):
        """nu_t of the attached model at the cell centres (ins_eddy_viscosity)."""
        self._check_u(u)
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=u.device)
        self._sync_stream()
        check(lib().ins_eddy_viscosity(self._h, _ptr(u), _ptr(out)), "ins_eddy_viscosity")
        return out

    def set_wall_solver(self, solver):
        """Channel grids: "thomas" (any y spacing) or "dct" (uniform y) wall-normal pressure solve."""
        code = {"thomas": 0, "dct": 1}[solver]
        check(lib().ins_set_wall_solver(self._h, code), "ins_set_wall_solver")

    def set_f64_arithmetic(self, mode):
        """FP64 step arithmetic (ins_set_f64_arithmetic): "native" FP64 instructions or "double-float"
        (pairs of FP32 values, the default on the grids that support it)."""
        code = {"native": 0, "double-float": 1}[mode]
        check(lib().ins_set_f64_arithmetic(self._h, code), "ins_set_f64_arithmetic")

    def f64_arithmetic(self):
        m = ctypes.c_int()
        check(lib().ins_get_f64_arithmetic(self._h, ctypes.byref(m)), "ins_get_f64_arithmetic")
        return "double-float" if m.value == 1 else "native"

    def set_march_chunk(self, planes):
        """z planes per CTA of the fused pair kernels (ins_set_march_chunk; 0 = automatic)."""
        check(lib().ins_set_march_chunk(self._h, int(planes)), "ins_set_march_chunk")

    def set_step_fusion(self, enable):
        """FP32 3-D RK4 stage boundaries (ins_set_step_fusion): False/0 separate kernels, 1 fused
        with one cell per thread, True/2 (default) fused with two cells per thread."""
        level = (2 if enable else 0) if isinstance(enable, bool) else int(enable)
        check(lib().ins_set_step_fusion(self._h, level), "ins_set_step_fusion")

    def workspace_bytes(self):
        b = ctypes.c_size_t()
        check(lib().ins_workspace_bytes(self._h, ctypes.byref(b)), "ins_workspace_bytes")
        return b.value

    # ------------------------------------------------------------ operators
    def rhs(self, u, out=None, p=None):
        """dudt = F(u) - G p with L p = D F(u)   (ins_rhs)."""
        self._check_u(u)
        out = self.new_velocity() if out is None else out
        self._check_u(out, "out")
        if p is not None:
            self._check_p(p)
        self._sync_stream()
        check(lib().ins_rhs(self._h, _ptr(u), _ptr(out), _ptr(p)), "ins_rhs")
        return out

    def project(self, u, out=None, p=None):
        """u - G p with L p = D u   (ins_project). out may be u itself."""
        self._check_u(u)
        out = self.new_velocity() if out is None else out
        self._check_u(out, "out")
        if p is not None:
            self._check_p(p)
        self._sync_stream()
        check(lib().ins_project(self._h, _ptr(u), _ptr(out), _ptr(p)), "ins_project")
        return out

    def divergence(self, u, out=None):
        self._check_u(u)
        out = self.new_scalar() if out is None else out
        self._check_p(out, "out")
        self._sync_stream()
        check(lib().ins_divergence(self._h, _ptr(u), _ptr(out)), "ins_divergence")
        return out

    def step(self, u, dt=None, dt_dev=None, next_dt_dev=None, cfl=0.3):
        """One RK4 step in place (ins_step). dt: host float, or dt_dev: a CUDA float64 tensor of one element."""
        self._check_u(u)
        if dt_dev is None and dt is None:
            raise ValueError("give dt or dt_dev")
        for t in (dt_dev, next_dt_dev):
            if t is not None and (t.dtype != torch.float64 or not t.is_cuda or t.numel() < 1):
                raise ValueError("dt tensors must be CUDA float64")
        self._sync_stream()
        check(lib().ins_step(self._h, _ptr(u), _ptr(dt_dev), float(dt if dt is not None else 0.0),
                             _ptr(next_dt_dev), float(cfl)), "ins_step")
        return u

    def step_n(self, u, nsteps, dt=None, dt_dev=None, next_dt_dev=None, cfl=0.3):
        """nsteps RK4 steps in place (ins_step_n: the steps after the first replay a CUDA graph of one
        step). Same arguments as step; results equal nsteps calls of step."""
        self._check_u(u)
        if dt_dev is None and dt is None:
            raise ValueError("give dt or dt_dev")
        for t in (dt_dev, next_dt_dev):
            if t is not None and (t.dtype != torch.float64 or not t.is_cuda or t.numel() < 1):
                raise ValueError("dt tensors must be CUDA float64")
        self._sync_stream()
        check(lib().ins_step_n(self._h, _ptr(u), int(nsteps), _ptr(dt_dev), float(dt if dt is not None else 0.0),
                               _ptr(next_dt_dev), float(cfl)), "ins_step_n")
        return u

    def step_vjp(self, u_n, ubar_np1, dt=None, dt_dev=None, ubar_n=None, nubar=None):
        """Pullback of one step (ins_step_vjp): returns (ubar_n, nubar) with nubar a CUDA float64
        tensor of one element that the nu-derivative is added to (a new zero tensor if None)."""
        self._check_u(u_n, "u_n")
        self._check_u(ubar_np1, "ubar_np1")
        if dt_dev is None and dt is None:
            raise ValueError("give dt or dt_dev")
        ubar_n = self.new_velocity() if ubar_n is None else ubar_n
        self._check_u(ubar_n, "ubar_n")
        nubar = torch.zeros(1, dtype=torch.float64, device=self.device) if nubar is None else nubar
        self._sync_stream()
        check(lib().ins_step_vjp(self._h, _ptr(u_n), _ptr(dt_dev), float(dt if dt is not None else 0.0),
                                 _ptr(ubar_np1), _ptr(ubar_n), _ptr(nubar)), "ins_step_vjp")
        return ubar_n, nubar

    def spectrum(self, u, kmax=None):
        """Shell energy spectrum E[0..kmax] as a CUDA float64 tensor (ins_spectrum)."""
        self._check_u(u)
        kmax = min(self.n) // 2 if kmax is None else int(kmax)
        E = torch.empty(kmax + 1, dtype=torch.float64, device=self.device)
        self._sync_stream()
        check(lib().ins_spectrum(self._h, _ptr(u), _ptr(E), kmax), "ins_spectrum")
        return E

    def wall_profiles(self, u):
        """Channel statistics (ins_wall_profiles): (mean (3, ny), cov (6, ny)) float64 CUDA tensors."""
        self._check_u(u)
        out = torch.empty((9, self.n[1]), dtype=torch.float64, device=self.device)
        self._sync_stream()
        check(lib().ins_wall_profiles(self._h, _ptr(u), _ptr(out)), "ins_wall_profiles")
        return out[:3], out[3:]

    def cfl_dt(self, u, cfl, out=None):
        self._check_u(u)
        out = torch.zeros(1, dtype=torch.float64, device=self.device) if out is None else out
        self._sync_stream()
        check(lib().ins_cfl_dt(self._h, _ptr(u), float(cfl), _ptr(out)), "ins_cfl_dt")
        return out

    def diag(self, u, raise_nonfinite=True):
        """{'ke', 'max_div', 'max_u_over_h', 'nonfinite'} (synchronous)."""
        self._check_u(u)
        out = (ctypes.c_double * 4)()
        self._sync_stream()
        st = lib().ins_diag(self._h, _ptr(u), out)
        if st != _lib.INS_ERR_NONFINITE or raise_nonfinite:
            check(st, "ins_diag")
        return {"ke": out[0], "max_div": out[1], "max_u_over_h": out[2], "nonfinite": int(out[3])}

    @property
    def N(self):
        n = 1
        for v in self.n:
            n *= v
        return n

    def set_closure(self, closure):
        """Attach a closure (F(u) + m(u) in rhs, step, step_vjp); None detaches."""
        check(lib().ins_set_closure(self._h, closure._h if closure is not None else None), "ins_set_closure")
        self._closure = closure

    # ------------------------------------------------------------ measurement
    def launch_count(self):
        n = ctypes.c_ulonglong()
        check(lib().ins_launch_count(self._h, ctypes.byref(n)), "ins_launch_count")
        return n.value

    def profile(self, on=True):
        check(lib().ins_profile_enable(self._h, int(bool(on))), "ins_profile_enable")

    def profile_read(self):
        """{kernel name: (launches, total_ms)} since the last read (synchronous)."""
        cap = 64
        arr = (_lib.KernelStat * cap)()
        n = ctypes.c_int()
        self._sync_stream()
        check(lib().ins_profile_read(self._h, arr, cap, ctypes.byref(n)), "ins_profile_read")
        return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n.value)}

    def check_finite(self):
        self._sync_stream()
        check(lib().ins_check_finite(self._h), "ins_check_finite")
