"""Wray's low-storage three-stage RK (grid scheme "wray3") on the GPU against the oracle.

The GPU runs the two-register form u_{s+1} = u_s + dt (gamma_s k_s + zeta_s k_{s-1}) in place;
the oracle evaluates the Butcher tableau directly. Tolerances as for RK4: relative L2 field
error <= 1e-12 per step (FP64), <= 1e-10 after 100 steps, <= 2e-5 per step (FP32 on
FP32-rounded inputs); the next CFL time step is compared bit for bit. The step VJP is
compared with the oracle's Butcher-form pullback.
"""

import numpy as np
import pytest
import torch

from oracle import adjoint, timestep
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300.solver import Grid
from test_gpu_parity import case, rand_u, rounded, dev, host, rel, TOL, DTYPES

pytestmark = pytest.mark.gpu


def grids(name, dtype):
    c = case(name)
    og = OGrid(c["faces"], c["bc"], c["nu"], c["force"])
    gg = Grid(c["faces"], c["bc"], c["nu"], c["force"], dtype=dtype, scheme="wray3")
    return og, gg


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", ["p2", "p3", "p3tiny", "p3reg", "p3reg2", "c3", "c3reg", "c2"])
def test_wray3_step_parity(name, dtype):
    og, gg = grids(name, dtype)
    u0 = rounded(rand_u(og, 14, project=True), dtype)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ut = dev(u0, dtype)
    gg.step(ut, dt=dt)
    ref = timestep.wray3_step(og, u0, dt)
    assert rel(host(ut), ref) <= TOL[dtype], rel(host(ut), ref)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", ["p3", "c3"])
def test_wray3_device_dt_and_cfl_bitexact(name, dtype):
    og, gg = grids(name, dtype)
    u0 = rounded(rand_u(og, 15, project=True), dtype)
    ut = dev(u0, dtype)
    dt_dev = gg.cfl_dt(ut, 0.3)
    dt0 = dt_dev.item()
    assert dt0 == timestep.cfl_dt(og, u0, 0.3)
    gg.step(ut, dt_dev=dt_dev, next_dt_dev=dt_dev, cfl=0.3)
    u1 = host(ut)
    assert rel(u1, timestep.wray3_step(og, u0, dt0)) <= TOL[dtype]
    assert dt_dev.item() == timestep.cfl_dt(og, u1, 0.3)


def test_wray3_100_steps_fp64():
    og, gg = grids("p3tiny", torch.float64)
    u0 = rand_u(og, 16, project=True)
    dt = 0.3 * timestep.cfl_dt(og, u0, 0.3)
    ut = dev(u0, torch.float64)
    for _ in range(100):
        gg.step(ut, dt=dt)
    ref = timestep.integrate(og, u0, dt, 100, scheme="wray3")
    assert rel(host(ut), ref) <= 1e-10


@pytest.mark.parametrize("dtype", DTYPES)
def test_wray3_workspace_is_one_register_smaller(dtype):
    c = case("p3")
    g4 = Grid(c["faces"], c["bc"], c["nu"], c["force"], dtype=dtype)
    g3 = Grid(c["faces"], c["bc"], c["nu"], c["force"], dtype=dtype, scheme="wray3")
    scalar = 40 * 24 * 36 * (8 if dtype == torch.float64 else 4)
    # an FP32 3-D RK4 grid also holds the pressure field of its fused stage boundaries
    saved_want = 3 * scalar + (scalar if dtype == torch.float32 else 0)
    saved = g4.workspace_bytes() - g3.workspace_bytes()
    assert saved_want <= saved <= saved_want + 512
    g4.close()
    g3.close()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", ["p3", "p3reg", "p2"])
def test_wray3_step_vjp_matches_oracle(name, dtype):
    og, gg = grids(name, dtype)
    u0 = rounded(rand_u(og, 17, project=True), dtype)
    ybar = rounded(rand_u(og, 18), dtype)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ub, nb = gg.step_vjp(dev(u0, dtype), dev(ybar, dtype), dt=dt)
    ub_o, nb_o = adjoint.wray3_step_vjp(og, u0, dt, ybar)
    assert rel(host(ub), ub_o) <= TOL[dtype]
    assert abs(nb.item() - nb_o) <= 50 * TOL[dtype] * abs(nb_o)
