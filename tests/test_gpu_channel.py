"""Turbulent-channel configuration on the GPU against the oracle (32^3 on 4 pi x 2 x 4 pi/3,
tanh-stretched y with gamma = 1.5, nu = 1/180, f = (1, 0, 0)): laminar profile plus a seeded
perturbation, projected; several RK4 steps with the CFL time step; mean-velocity and
Reynolds-stress profiles."""

import numpy as np
import pytest
import torch

from oracle import diagnostics, poisson, timestep
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300.solver import Grid

pytestmark = pytest.mark.gpu


def channel(n=32, dtype=torch.float64):
    faces = inputs.channel_faces(n, n, n)
    bc = ["periodic", "wall", "periodic"]
    og = OGrid(faces, bc, 1 / 180, [1.0, 0.0, 0.0])
    gg = Grid(faces, bc, 1 / 180, [1.0, 0.0, 0.0], dtype=dtype)
    u0, _ = poisson.project(og, inputs.channel_velocity_raw(faces, seed=3))
    return og, gg, u0


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_profiles_match_oracle():
    og, gg, u0 = channel()
    mean, cov = gg.wall_profiles(torch.tensor(u0, device="cuda"))
    m_or, c_or = diagnostics.wall_profiles(og, u0)
    for a in range(3):
        assert np.allclose(mean[a].cpu().numpy(), m_or[a], rtol=1e-12, atol=1e-12 * np.max(np.abs(m_or[0])))
    keys = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for q, k in enumerate(keys):
        assert np.allclose(cov[q].cpu().numpy(), c_or[k], rtol=1e-10, atol=1e-10 * np.max(np.abs(c_or[(0, 0)])))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 1e-4)])
def test_ten_cfl_steps_and_profiles(dtype, tol):
    og, gg, u0 = channel(dtype=dtype)
    if dtype == torch.float32:
        u0 = u0.astype(np.float32).astype(np.float64)
    ut = torch.tensor(u0, dtype=dtype, device="cuda")
    dt = gg.cfl_dt(ut, 0.3)
    u = u0
    assert dt.item() == timestep.cfl_dt(og, u0, 0.3)            # identical input: same bits
    for _ in range(10):
        d = dt.item()
        # the trajectories differ at round-off, so the CFL steps agree to round-off
        assert abs(d - timestep.cfl_dt(og, u, 0.3)) <= 1e3 * tol * d
        gg.step(ut, dt_dev=dt, next_dt_dev=dt, cfl=0.3)
        u = timestep.rk4_step(og, u, d)
    assert rel(ut.double().cpu().numpy(), u) <= tol
    mean, _ = gg.wall_profiles(ut)
    m_or, _ = diagnostics.wall_profiles(og, u)
    assert rel(mean[0].cpu().numpy(), m_or[0]) <= tol
    assert np.all(ut[1][:, -1, :].cpu().numpy() == 0.0)      # top wall stays closed
