"""ins_cfl_dt_noalloc: the CFL time step for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- code under a memory manager that has
reserved nearly all device memory for its own pool, or a plug-in that must keep
the device footprint fixed -- so they cannot create a grid (which allocates its
workspace). This entry point keeps its scratch in a static device array inside
the library instead. Its answer must equal ins_cfl_dt's bit for bit (the CFL
tests elsewhere are bit-exact too), also on the second of two calls in a row,
which shares the static array with the first.

This file is collected last on purpose, so a run that stops at its first
failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_2604_18536_b300 import inputs, _lib
from paper_2604_18536_b300.solver import Grid

pytestmark = pytest.mark.gpu


def _desc(faces, bc, nu, dtype):
    d = _lib.GridDesc()
    d.dim = len(faces)
    keep = [np.ascontiguousarray(f, dtype=np.float64) for f in faces]
    for a in range(3):
        d.n[a] = len(keep[a]) - 1 if a < d.dim else 1
        d.bc[a] = (_lib.INS_WALL if bc[a] == "wall" else _lib.INS_PERIODIC) if a < d.dim else 0
        d.face_coords[a] = keep[a].ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a < d.dim else None
    d.dtype = _lib.INS_F64 if dtype == torch.float64 else _lib.INS_F32
    d.nu = nu
    return d, keep


def _noalloc(desc, u, cfl, out):
    st = torch.cuda.current_stream().cuda_stream
    return _lib.lib().ins_cfl_dt_noalloc(ctypes.byref(desc), ctypes.c_void_p(u.data_ptr()), cfl,
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st))


CASES = {
    "periodic3_f64": (lambda: inputs.periodic_box(40, 3), ["periodic"] * 3, 1 / 1600, torch.float64),
    "channel3_f32": (lambda: inputs.channel_faces(36, 20, 28), ["periodic", "wall", "periodic"], 1 / 180,
                     torch.float32),
    "periodic2_f64": (lambda: [inputs.uniform_faces(72, 0, 2 * np.pi), inputs.uniform_faces(40, 0, 3.0)],
                      ["periodic"] * 2, 0.01, torch.float64),
}


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_matches_cfl_dt_on_two_calls(name):
    mk, bc, nu, dtype = CASES[name]
    faces = mk()
    g = Grid(faces, bc, nu, dtype=dtype)
    desc, keep = _desc(faces, bc, nu, dtype)
    shape = (len(faces),) + g.shape
    # first call with a large field, second with a smaller one: stale maxima would show
    fields = [inputs.random_field(shape, 1, 5.0), inputs.random_field(shape, 2, 1.0)]
    for f in fields:
        if "wall" in bc:
            f[1][..., -1, :] = 0.0
        u = torch.tensor(f, dtype=dtype, device="cuda")
        want = g.cfl_dt(u, 0.3).item()
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(desc, u, 0.3, out) == _lib.INS_OK, _lib.lib().ins_last_error()
        assert out.item() == want
    g.close()


def test_noalloc_allocates_no_device_memory():
    faces = inputs.periodic_box(32, 3)
    desc, keep = _desc(faces, ["periodic"] * 3, 0.01, torch.float64)
    u = torch.tensor(inputs.random_field((3, 32, 32, 32), 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(desc, u, 0.5, out) == _lib.INS_OK      # first call on this device: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _noalloc(desc, u, 0.5, out) == _lib.INS_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_the_limit():
    faces = [inputs.uniform_faces(5000, 0, 1.0), inputs.uniform_faces(8, 0, 1.0)]
    desc, keep = _desc(faces, ["periodic"] * 2, 0.01, torch.float64)
    u = torch.zeros((2, 8, 5000), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(desc, u, 0.3, out) == _lib.INS_ERR_ARG
    assert b"4096" in _lib.lib().ins_last_error()


_FIRST_CALL_SCRIPT = r"""
import ctypes, json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2604_18536_b300 import inputs, _lib
torch.cuda.init()
faces = inputs.periodic_box(32, 3)
keep = [np.ascontiguousarray(f, dtype=np.float64) for f in faces]
d = _lib.GridDesc()
d.dim = 3
for a in range(3):
    d.n[a] = 32
    d.bc[a] = _lib.INS_PERIODIC
    d.face_coords[a] = keep[a].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
d.dtype = _lib.INS_F64
d.nu = 0.01
u = torch.tensor(inputs.random_field((3, 32, 32, 32), 3), dtype=torch.float64, device="cuda")
out = torch.zeros(1, dtype=torch.float64, device="cuda")
lib = _lib.lib()
st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
torch.cuda.synchronize()
free = [torch.cuda.mem_get_info()[0]]
for _ in range(4):
    rc = lib.ins_cfl_dt_noalloc(ctypes.byref(d), ctypes.c_void_p(u.data_ptr()), 0.5,
                                ctypes.c_void_p(out.data_ptr()), st)
    assert rc == _lib.INS_OK, lib.ins_last_error()
    torch.cuda.synchronize()
    free.append(torch.cuda.mem_get_info()[0])
print(json.dumps({"free": free, "dt": out.item()}))
"""


def test_noalloc_first_call_in_fresh_process():
    """In a process that has not called the library yet, the first call loads the library's device
    code and static array (CUDA loads modules lazily), which takes device memory; later calls take
    none. The drop is recorded so that memory-constrained callers know what to set aside."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_SCRIPT, root], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    free = res["free"]
    first_drop = free[0] - free[1]
    print(f"first call on the device: {first_drop / 2**20:.1f} MiB of device memory (module load)")
    assert first_drop >= 0
    assert first_drop < 512 * 2**20
    assert free[1] == free[2] == free[3] == free[4]
    assert res["dt"] > 0.0
