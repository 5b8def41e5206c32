"""Step VJP on wall-bounded (channel) grids against the oracle's pullback and finite differences.

Cases span several tiles with ragged tails, tanh-stretched y and register-path FFT lengths.
FP64: relative L2 error <= 1e-12 against the oracle's VJP of the same step (cotangents masked
on the stored wall faces); FP32: the FP64 oracle on FP32-rounded inputs, <= 2e-5. Central
differences (eps = 1e-6) of the GPU forward step along seeded masked directions.
"""

import numpy as np
import pytest
import torch

from oracle import adjoint, poisson, timestep
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300.solver import Grid
from test_gpu_parity import case, rand_u, rounded, dev, host, rel, TOL

pytestmark = pytest.mark.gpu


def setup(name, dtype, scheme="rk4", seed=1):
    c = case(name)
    og = OGrid(c["faces"], c["bc"], c["nu"], c["force"])
    gg = Grid(c["faces"], c["bc"], c["nu"], c["force"], dtype=dtype, scheme=scheme)
    u0 = rounded(rand_u(og, seed, project=True), dtype)
    ybar = rounded(rand_u(og, seed + 100), dtype)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    return og, gg, u0, ybar, dt


@pytest.mark.parametrize("scheme", ["rk4", "wray3"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("name", ["c3", "c3reg", "c2"])
def test_step_vjp_wall_matches_oracle(name, dtype, scheme):
    og, gg, u0, ybar, dt = setup(name, dtype, scheme)
    ub, nb = gg.step_vjp(dev(u0, dtype), dev(ybar, dtype), dt=dt)
    vjp = adjoint.rk4_step_vjp if scheme == "rk4" else adjoint.wray3_step_vjp
    ub_o, nb_o = vjp(og, u0, dt, ybar)
    assert rel(host(ub), ub_o) <= TOL[dtype], rel(host(ub), ub_o)
    assert abs(nb.item() - nb_o) <= 50 * TOL[dtype] * abs(nb_o)
    top = host(ub)[1][..., -1, :]
    assert np.all(top == 0.0)


def test_step_vjp_wall_central_differences():
    og, gg, u0, c, dt = setup("c3", torch.float64, seed=5)
    ub = host(gg.step_vjp(dev(u0, torch.float64), dev(c, torch.float64), dt=dt)[0])
    eps = 1e-6

    def L(u):
        t = dev(u, torch.float64)
        gg.step(t, dt=dt)
        return float(np.sum(c * host(t)))

    for seed in range(4):
        v, _ = poisson.project(og, rand_u(og, 300 + seed))
        fd = (L(u0 + eps * v) - L(u0 - eps * v)) / (2 * eps)
        assert abs(fd - np.sum(ub * v)) <= 1e-7 * max(1.0, abs(fd))
