"""Host-side checks of libins: it loads, exports every symbol include/ins.h declares,
and rejects bad arguments before touching the device (no GPU needed)."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2604_18536_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ins_\w+)\s*\(", txt, re.M))
    return names


def test_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert set(_lib.SIGNATURES) >= names


def test_version(L):
    assert b"libins" in L.ins_version()


def _desc(dim=3, n=(8, 8, 8), bc=(0, 0, 0), faces=None, dtype=1, nu=0.01):
    d = _lib.GridDesc()
    d.dim = dim
    keep = []
    for a in range(3):
        d.n[a] = n[a]
        d.bc[a] = bc[a]
        f = np.linspace(0, 1, n[a] + 1) if faces is None else faces[a]
        keep.append(f)
        d.face_coords[a] = f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if f is not None else None
    d.dtype = dtype
    d.nu = nu
    return d, keep


@pytest.mark.parametrize("case,want", [
    ("dim4", _lib.INS_ERR_ARG),
    ("n1", _lib.INS_ERR_ARG),
    ("badbc", _lib.INS_ERR_ARG),
    ("nullfaces", _lib.INS_ERR_ARG),
    ("dtype", _lib.INS_ERR_ARG),
    ("nu", _lib.INS_ERR_ARG),
    ("wallx", _lib.INS_ERR_UNSUPPORTED),
    ("nonuniform_periodic", _lib.INS_ERR_UNSUPPORTED),
    ("radix11", _lib.INS_ERR_UNSUPPORTED),
    ("decreasing", _lib.INS_ERR_ARG),
])
def test_create_rejects_bad_descriptors(L, case, want):
    kw = {}
    if case == "dim4":
        kw["dim"] = 4
    elif case == "n1":
        kw["n"] = (1, 8, 8)
    elif case == "badbc":
        kw["bc"] = (0, 7, 0)
    elif case == "dtype":
        kw["dtype"] = 5
    elif case == "nu":
        kw["nu"] = float("nan")
    elif case == "wallx":
        kw["bc"] = (1, 0, 0)
    elif case == "nonuniform_periodic":
        f = np.linspace(0, 1, 9)
        f[3] += 0.01
        kw["faces"] = [f, np.linspace(0, 1, 9), np.linspace(0, 1, 9)]
    elif case == "radix11":
        kw["n"] = (11, 8, 8)
    elif case == "decreasing":
        f = np.linspace(0, 1, 9)[::-1].copy()
        kw["faces"] = [np.linspace(0, 1, 9), f, np.linspace(0, 1, 9)]
        kw["bc"] = (0, 1, 0)
    d, keep = _desc(**kw)
    if case == "nullfaces":
        d.face_coords[1] = None
    h = ctypes.c_void_p()
    st = L.ins_grid_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == want, L.ins_last_error()
    assert h.value is None
    assert len(L.ins_last_error()) > 0


def test_null_arguments(L):
    assert L.ins_grid_create(None, None, None) == _lib.INS_ERR_ARG
    assert L.ins_rhs(None, None, None, None) == _lib.INS_ERR_ARG
    assert L.ins_step(None, None, None, 0.1, None, 0.3) == _lib.INS_ERR_ARG
    assert L.ins_grid_destroy(None) == _lib.INS_OK
