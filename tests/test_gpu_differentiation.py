"""Differentiation of a 16-step unroll at 128^3 (3-D periodic decaying turbulence).

Loss L(u0, nu) = mean over the field of (u_16 - u_target)^2, u_16 the 16th RK4 step from u0 and
u_target the 16th step from the seeded spectrum field u*; u0 = u* + 0.1 x an independent projected
field (the gradient vanishes at u* itself). The time step is frozen from the CFL rule on u*.
The gradient comes from torch.autograd over ins_step (per-step checkpoints, stage recomputation,
the hand-written step VJP) and is checked in FP64 against central differences (eps = 1e-6) of the
GPU forward map along 20 seeded directions, for u0 and for nu. FP32 gradients are compared with the
FP64 ones.
"""

import math

import numpy as np
import pytest
import torch

from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300 import autograd as ag
from paper_2604_18536_b300.solver import Grid

pytestmark = pytest.mark.gpu

N = 128
NU = 1.0 / 1000
NSTEPS = 16


def _grid(dtype, nu=NU):
    return Grid(inputs.periodic_box(N, 3), ["periodic"] * 3, nu, dtype=dtype)


def _field(g, seed, dtype):
    u = torch.tensor(inputs.spectrum_velocity_raw(N, 3, seed=seed, k0=4.0, kmax=32), dtype=dtype, device="cuda")
    g.project(u, out=u)
    u.mul_(1.0 / math.sqrt(g.diag(u)["ke"]))
    return u


@pytest.fixture(scope="module")
def problem():
    g = _grid(torch.float64)
    ustar = _field(g, 0, torch.float64)
    dt = float(g.cfl_dt(ustar, 0.3).item())
    target = ustar.clone()
    for _ in range(NSTEPS):
        g.step(target, dt=dt)
    u0 = ustar + 0.1 * _field(g, 1, torch.float64)
    return g, u0, target, dt


def _loss(g, u0, target, dt, nu=None):
    u = u0.detach().clone().requires_grad_(True)
    nut = torch.tensor(g.nu if nu is None else nu, dtype=torch.float64, device="cuda", requires_grad=True)
    states = ag.rollout(u, g, dt, NSTEPS, nut)
    loss = ((states[-1] - target) ** 2).mean()
    loss.backward()
    return loss.item(), u.grad.detach(), nut.grad.item()


def _forward_loss(g, u0, target, dt):
    u = u0.clone()
    for _ in range(NSTEPS):
        g.step(u, dt=dt)
    return float(((u - target) ** 2).double().mean())


def test_gradient_central_differences_fp64(problem):
    g, u0, target, dt = problem
    L0, gu, gnu = _loss(g, u0, target, dt)
    assert L0 > 0 and torch.isfinite(gu).all()
    eps = 1e-6
    rms = float(u0.pow(2).mean().sqrt())
    for seed in range(1, 21):
        v = torch.tensor(inputs.random_field(tuple(u0.shape), 1000 + seed), dtype=torch.float64, device="cuda")
        v.mul_(rms / float(v.pow(2).mean().sqrt()))
        fd = (_forward_loss(g, u0 + eps * v, target, dt) - _forward_loss(g, u0 - eps * v, target, dt)) / (2 * eps)
        ad = float((gu * v).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-12 * L0, (seed, fd, ad)
    # viscosity: two grids at nu +- h (the grid's coefficients depend on nu)
    h = 1e-6 * NU
    gp, gm = _grid(torch.float64, NU + h), _grid(torch.float64, NU - h)
    fd_nu = (_forward_loss(gp, u0, target, dt) - _forward_loss(gm, u0, target, dt)) / (2 * h)
    gp.close()
    gm.close()
    assert abs(fd_nu - gnu) <= 1e-6 * abs(gnu), (fd_nu, gnu)


def test_gradient_fp32_against_fp64(problem):
    g, u0, target, dt = problem
    _, gu64, gnu64 = _loss(g, u0, target, dt)
    g32 = _grid(torch.float32)
    _, gu32, gnu32 = _loss(g32, u0.float(), target.float(), dt)
    g32.close()
    err = float(torch.linalg.norm((gu32.double() - gu64).ravel()) / torch.linalg.norm(gu64.ravel()))
    assert err <= 1e-3, err
    assert abs(gnu32 - gnu64) <= 1e-3 * abs(gnu64), (gnu32, gnu64)
