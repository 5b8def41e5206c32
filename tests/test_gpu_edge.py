"""Edge cases of the step against the oracle: smallest and largest supported sizes, degenerate
fields and parameters.

* n = 2 in every direction (the smallest grid; neighbours wrap onto each other);
* the largest periodic FFT length (2048) and the largest wall-normal size (4096 rows);
* FFT lengths with every radix at odd products (3 * 5 * 7 = 105) on the shared-memory path;
* a zero field (stays zero without forcing; the CFL step is the diffusive limit, bit for bit);
* inviscid flow (nu = 0: no diffusive limit) and a field at rest with nu = 0 (dt = inf).
Tolerances as in test_gpu_parity (FP64 relative L2 <= 1e-12, FP32 <= 2e-5; CFL bit-exact).
"""

import math

import numpy as np
import pytest
import torch

from oracle import timestep, poisson
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300.solver import Grid
from test_gpu_parity import rounded, dev, host, rel, TOL, DTYPES

pytestmark = pytest.mark.gpu
U = inputs.uniform_faces
PI = np.pi


def pair(faces, bc, nu, dtype, force=None):
    return OGrid(faces, bc, nu, force), Grid(faces, bc, nu, force, dtype=dtype)


def step_parity(og, gg, dtype, seed):
    u0 = inputs.random_field((og.dim,) + og.shape, seed)
    for a in range(og.dim):
        u0[a] *= og.face_mask(a)
    u0, _ = poisson.project(og, u0)
    u0 = rounded(u0, dtype)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ut = dev(u0, dtype)
    gg.step(ut, dt=dt)
    ref = timestep.rk4_step(og, u0, dt)
    return rel(host(ut), ref)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("dim", [2, 3])
def test_smallest_periodic_grid(dim, dtype):
    og, gg = pair([U(2, 0, 1.0)] * dim, ["periodic"] * dim, 0.05, dtype)
    assert step_parity(og, gg, dtype, 1) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_smallest_channel_grid(dtype):
    og, gg = pair([U(2, 0, 1.0), inputs.tanh_faces(2, 0, 2, 1.5), U(2, 0, 1.0)], ["periodic", "wall", "periodic"],
                  0.05, dtype, force=[1.0, 0.0, 0.0])
    assert step_parity(og, gg, dtype, 2) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_largest_periodic_fft_length(dtype):
    og, gg = pair([U(2048, 0, 2 * PI), U(6, 0, 1.0), U(4, 0, 1.0)], ["periodic"] * 3, 0.01, dtype)
    assert step_parity(og, gg, dtype, 3) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_largest_wall_normal_size(dtype):
    og, gg = pair([U(4, 0, 1.0), inputs.tanh_faces(4096, 0, 2, 1.5), U(2, 0, 1.0)], ["periodic", "wall", "periodic"],
                  1.0 / 180, dtype, force=[1.0, 0.0, 0.0])
    assert step_parity(og, gg, dtype, 4) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_odd_radix_lengths(dtype):
    og, gg = pair([U(105, 0, 2 * PI), U(9, 0, 1.0), U(25, 0, 3.0)], ["periodic"] * 3, 0.02, dtype)
    assert step_parity(og, gg, dtype, 5) <= TOL[dtype]


def test_oversize_grids_are_rejected():
    from paper_2604_18536_b300._lib import InsError
    with pytest.raises(InsError):
        Grid([U(4096, 0, 1.0), U(4, 0, 1.0)], ["periodic"] * 2, 0.1)      # periodic n > 2048
    with pytest.raises(InsError):
        Grid([U(4, 0, 1.0), U(4097, 0, 1.0)], ["periodic", "wall"], 0.1)  # n > 4096
    with pytest.raises(InsError):
        Grid([U(22, 0, 1.0), U(4, 0, 1.0)], ["periodic"] * 2, 0.1)        # 22 = 2 * 11: no radix 11


@pytest.mark.parametrize("dtype", DTYPES)
def test_zero_field_stays_zero_and_cfl_is_diffusive_limit(dtype):
    og, gg = pair([U(16, 0, 2 * PI), U(8, 0, 1.0), U(12, 0, 3.0)], ["periodic"] * 3, 0.02, dtype)
    u = torch.zeros((3,) + og.shape, dtype=dtype, device="cuda")
    dt = gg.cfl_dt(u, 0.3)
    assert dt.item() == timestep.cfl_dt(og, np.zeros((3,) + og.shape), 0.3)
    dmin = min(float(np.min(og.d[a])) for a in range(3))
    assert dt.item() == 0.3 * (dmin * dmin / 0.02)
    gg.step(u, dt_dev=dt, next_dt_dev=dt, cfl=0.3)
    assert torch.count_nonzero(u).item() == 0
    assert dt.item() == timestep.cfl_dt(og, np.zeros((3,) + og.shape), 0.3)


def test_inviscid_step_and_rest_state():
    og, gg = pair([U(16, 0, 2 * PI), U(8, 0, 1.0), U(12, 0, 3.0)], ["periodic"] * 3, 0.0, torch.float64)
    assert step_parity(og, gg, torch.float64, 6) <= 1e-12
    u = torch.zeros((3,) + og.shape, dtype=torch.float64, device="cuda")
    dt = gg.cfl_dt(u, 0.3)
    assert math.isinf(dt.item()) and math.isinf(timestep.cfl_dt(og, np.zeros((3,) + og.shape), 0.3))
