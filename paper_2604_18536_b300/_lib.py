"""ctypes declarations of libins (include/ins.h). Argument marshalling only.

The shared library is loaded from this package directory. There is no
fallback: if it is missing or cannot be loaded, ``lib()`` raises.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libins.so")

INS_OK = 0
INS_ERR_ARG = 1
INS_ERR_UNSUPPORTED = 2
INS_ERR_OOM = 3
INS_ERR_CUDA = 4
INS_ERR_NONFINITE = 5
INS_ERR_TIMEOUT = 6
STATUS_NAMES = {0: "INS_OK", 1: "INS_ERR_ARG", 2: "INS_ERR_UNSUPPORTED", 3: "INS_ERR_OOM", 4: "INS_ERR_CUDA",
                5: "INS_ERR_NONFINITE", 6: "INS_ERR_TIMEOUT"}

INS_PERIODIC = 0
INS_WALL = 1
INS_ARITH_NATIVE, INS_ARITH_DOUBLE_FLOAT = 0, 1
INS_F32 = 0
INS_F64 = 1
INS_RK4 = 0
INS_WRAY3 = 1
INS_EDDY = {"none": 0, "smagorinsky": 1, "wale": 2, "qr": 3, "vreman": 4, "constant": 5}

# every entry point the header declares, with (restype, argtypes)
_c = ctypes
_vp = _c.c_void_p
_dp = _c.POINTER(_c.c_double)


class GridDesc(_c.Structure):
    _fields_ = [
        ("dim", _c.c_int),
        ("n", _c.c_int * 3),
        ("bc", _c.c_int * 3),
        ("face_coords", _dp * 3),
        ("dtype", _c.c_int),
        ("nu", _c.c_double),
        ("force", _c.c_double * 3),
        ("scheme", _c.c_int),
    ]


class KernelStat(_c.Structure):
    _fields_ = [("name", _c.c_char * 32), ("launches", _c.c_longlong), ("total_ms", _c.c_double)]


SIGNATURES = {
    "ins_last_error": (_c.c_char_p, []),
    "ins_version": (_c.c_char_p, []),
    "ins_grid_create": (_c.c_int, [_c.POINTER(GridDesc), _vp, _c.POINTER(_vp)]),
    "ins_grid_destroy": (_c.c_int, [_vp]),
    "ins_set_stream": (_c.c_int, [_vp, _vp]),
    "ins_workspace_bytes": (_c.c_int, [_vp, _c.POINTER(_c.c_size_t)]),
    "ins_rhs": (_c.c_int, [_vp, _vp, _vp, _vp]),
    "ins_project": (_c.c_int, [_vp, _vp, _vp, _vp]),
    "ins_divergence": (_c.c_int, [_vp, _vp, _vp]),
    "ins_set_step_fusion": (_c.c_int, [_vp, _c.c_int]),
    "ins_set_march_chunk": (_c.c_int, [_vp, _c.c_int]),
    "ins_set_wall_solver": (_c.c_int, [_vp, _c.c_int]),
    "ins_set_f64_arithmetic": (_c.c_int, [_vp, _c.c_int]),
    "ins_get_f64_arithmetic": (_c.c_int, [_vp, _vp]),
    "ins_set_eddy_viscosity": (_c.c_int, [_vp, _c.c_int, _c.c_double]),
    "ins_eddy_viscosity": (_c.c_int, [_vp, _vp, _vp]),
    "ins_step": (_c.c_int, [_vp, _vp, _vp, _c.c_double, _vp, _c.c_double]),
    "ins_step_n": (_c.c_int, [_vp, _vp, _c.c_int, _vp, _c.c_double, _vp, _c.c_double]),
    "ins_cfl_dt": (_c.c_int, [_vp, _vp, _c.c_double, _vp]),
    "ins_step_vjp": (_c.c_int, [_vp, _vp, _vp, _c.c_double, _vp, _vp, _vp]),
    "ins_spectrum": (_c.c_int, [_vp, _vp, _vp, _c.c_int]),
    "ins_wall_profiles": (_c.c_int, [_vp, _vp, _vp]),
    "ins_filter_face_average": (_c.c_int, [_c.c_int, _c.POINTER(_c.c_int), _c.c_int, _c.c_int, _vp, _vp, _vp]),
    "ins_diag": (_c.c_int, [_vp, _vp, _dp]),
    "ins_check_finite": (_c.c_int, [_vp]),
    "ins_launch_count": (_c.c_int, [_vp, _c.POINTER(_c.c_ulonglong)]),
    "ins_profile_enable": (_c.c_int, [_vp, _c.c_int]),
    "ins_profile_read": (_c.c_int, [_vp, _c.POINTER(KernelStat), _c.c_int, _c.POINTER(_c.c_int)]),
    "ins_measure_fma_rate": (_c.c_int, [_c.c_int, _vp, _dp]),
    "ins_closure_create": (_c.c_int, [_vp, _c.POINTER(_vp)]),
    "ins_closure_destroy": (_c.c_int, [_vp]),
    "ins_closure_set_params": (_c.c_int, [_vp, _c.POINTER(_vp), _c.POINTER(_vp)]),
    "ins_closure_fwd": (_c.c_int, [_vp, _vp, _vp, _vp, _c.c_int]),
    "ins_closure_bwd": (_c.c_int, [_vp, _vp, _vp, _vp, _c.POINTER(_vp), _c.POINTER(_vp)]),
    "ins_closure_set_grads": (_c.c_int, [_vp, _c.POINTER(_vp), _c.POINTER(_vp)]),
    "ins_closure_saved": (_c.c_int, [_vp, _c.c_int, _vp, _vp]),
    "ins_closure_check": (_c.c_int, [_vp]),
    "ins_set_closure": (_c.c_int, [_vp, _vp]),
    "ins_cfl_dt_noalloc": (_c.c_int, [_c.POINTER(GridDesc), _vp, _c.c_double, _vp, _vp]),
}

_LIB = None


class InsError(RuntimeError):
    def __init__(self, status, where, msg):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def lib():
    """The loaded libins (raises if it is missing: there is no CPU fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libins.so not built at {LIB_PATH}; run `python -m paper_2604_18536_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def check(status, where):
    if status != INS_OK:
        msg = lib().ins_last_error().decode(errors="replace")
        raise InsError(status, where, msg)
