"""Step VJP (ins_step_vjp) against the oracle's pullback and against finite differences.

FP64: relative error <= 1e-12 against the oracle's VJP of the same step; central
finite differences (eps = 1e-6) of the GPU forward step on seeded directions.
FP32: the FP64 oracle on the FP32-rounded inputs, relative error <= 2e-5.
"""

import numpy as np
import pytest
import torch

from oracle import adjoint, poisson, timestep
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300 import autograd as ag
from paper_2604_18536_b300.solver import Grid
from paper_2604_18536_b300._lib import InsError

pytestmark = pytest.mark.gpu
U = inputs.uniform_faces
PI = np.pi


def case(name):
    if name == "p3":        # generic FFT lengths
        return [U(24, 0, 2 * PI), U(20, 0, 1.5 * PI), U(14, 0, 3.0)], 0.03
    if name == "p3reg":     # register FFT lengths
        return [U(32, 0, 2 * PI), U(16, 0, 1.0), U(64, 0, 3.0)], 0.02
    if name == "p2":
        return [U(40, 0, 2 * PI), U(24, 0, 1.5 * PI)], 0.05
    if name == "p3odd":     # odd nx: the one-cell-per-thread adjoint march
        return [U(15, 0, 2 * PI), U(12, 0, 1.5 * PI), U(10, 0, 3.0)], 0.03
    if name == "p3wide":    # nx = 140: two full 64-wide pair tiles and a ragged one
        return [U(140, 0, 2 * PI), U(9, 0, 1.5 * PI), U(6, 0, 3.0)], 0.03
    raise KeyError(name)


def setup(name, dtype, seed=1):
    faces, nu = case(name)
    og = OGrid(faces, ["periodic"] * len(faces), nu)
    gg = Grid(faces, ["periodic"] * len(faces), nu, dtype=dtype)
    u0, _ = poisson.project(og, inputs.random_field((og.dim,) + og.shape, seed))
    ybar = inputs.random_field((og.dim,) + og.shape, seed + 100)
    if dtype == torch.float32:
        u0 = u0.astype(np.float32).astype(np.float64)
        ybar = ybar.astype(np.float32).astype(np.float64)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    return og, gg, u0, ybar, dt


def dev(x, dtype):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


TOL = {torch.float64: 1e-12, torch.float32: 2e-5}


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("name", ["p3", "p3reg", "p2"])
def test_step_vjp_matches_oracle(name, dtype):
    og, gg, u0, ybar, dt = setup(name, dtype)
    ub, nb = gg.step_vjp(dev(u0, dtype), dev(ybar, dtype), dt=dt)
    ub_o, nb_o = adjoint.rk4_step_vjp(og, u0, dt, ybar)
    assert rel(ub.double().cpu().numpy(), ub_o) <= TOL[dtype]
    assert abs(nb.item() - nb_o) <= 50 * TOL[dtype] * abs(nb_o)


@pytest.mark.parametrize("level", [0, 2])
@pytest.mark.parametrize("name", ["p3", "p3reg", "p3odd", "p3wide"])
def test_step_vjp_fp32_adjoint_kernels(name, level):
    """FP32: the two-cells-per-thread adjoint march (fusion level 2, even nx) and the one-cell
    march (level 0, or odd nx) both against the oracle, and against each other."""
    og, gg, u0, ybar, dt = setup(name, torch.float32, seed=7)
    gg.set_step_fusion(level)
    ub, nb = gg.step_vjp(dev(u0, torch.float32), dev(ybar, torch.float32), dt=dt)
    ub_o, nb_o = adjoint.rk4_step_vjp(og, u0, dt, ybar)
    assert rel(ub.double().cpu().numpy(), ub_o) <= TOL[torch.float32]
    assert abs(nb.item() - nb_o) <= 50 * TOL[torch.float32] * abs(nb_o)
    gg.set_step_fusion(2 - level)
    ub2, _ = gg.step_vjp(dev(u0, torch.float32), dev(ybar, torch.float32), dt=dt)
    assert rel(ub2.double().cpu().numpy(), ub.double().cpu().numpy()) <= 1e-6


def test_step_vjp_inputs_untouched_and_device_dt():
    og, gg, u0, ybar, dt = setup("p3reg", torch.float64, seed=3)
    u = dev(u0, torch.float64)
    y = dev(ybar, torch.float64)
    u_c, y_c = u.clone(), y.clone()
    dtd = torch.tensor([dt], dtype=torch.float64, device="cuda")
    nub = torch.full((1,), 2.0, dtype=torch.float64, device="cuda")
    ub, nb = gg.step_vjp(u, y, dt_dev=dtd, nubar=nub)
    assert torch.equal(u, u_c) and torch.equal(y, y_c)
    ub_o, nb_o = adjoint.rk4_step_vjp(og, u0, dt, ybar)
    assert rel(ub.cpu().numpy(), ub_o) <= 1e-12
    assert abs((nb.item() - 2.0) - nb_o) <= 1e-10 * abs(nb_o)     # added to the given value


def test_step_vjp_central_differences():
    """<ubar, v> against (L(u + eps v) - L(u - eps v)) / 2 eps with L = <c, step(u)>, eps = 1e-6."""
    og, gg, u0, c, dt = setup("p3reg", torch.float64, seed=5)
    ub, _ = gg.step_vjp(dev(u0, torch.float64), dev(c, torch.float64), dt=dt)
    ub = ub.cpu().numpy()
    eps = 1e-6

    def L(u):
        t = dev(u, torch.float64)
        gg.step(t, dt=dt)
        return float(np.sum(c * t.cpu().numpy()))

    for seed in range(5):
        v, _ = poisson.project(og, inputs.random_field(u0.shape, 200 + seed))
        fd = (L(u0 + eps * v) - L(u0 - eps * v)) / (2 * eps)
        assert abs(fd - np.sum(ub * v)) <= 1e-7 * max(1.0, abs(fd))


def test_autograd_rollout_matches_oracle_chain():
    """Three differentiable steps through torch.autograd: dL/du0 and dL/dnu against the oracle."""
    og, gg, u0, c, dt = setup("p3", torch.float64, seed=7)
    u = dev(u0, torch.float64).requires_grad_(True)
    nu = torch.tensor(og.nu, dtype=torch.float64, device="cuda", requires_grad=True)
    states = ag.rollout(u, gg, dt, 3, nu)
    loss = (states[-1] * dev(c, torch.float64)).sum()
    loss.backward()
    # oracle: chain the step pullbacks
    us = [u0]
    for _ in range(2):
        us.append(timestep.rk4_step(og, us[-1], dt))
    ybar, nub = c, 0.0
    for k in range(2, -1, -1):
        ybar, nb = adjoint.rk4_step_vjp(og, us[k], dt, ybar)
        nub += nb
    assert rel(u.grad.cpu().numpy(), ybar) <= 1e-12
    assert abs(nu.grad.item() - nub) <= 1e-10 * abs(nub)
