"""Face-averaging filter and shell spectrum on the GPU against the oracle."""

import numpy as np
import pytest
import torch

from oracle import diagnostics, operators as op, poisson
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300.solver import Grid, filter_face_average

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("dim,nf,m", [(3, (32, 24, 16), 4), (3, (12, 12, 12), 3), (2, (40, 24), 2)])
def test_filter_matches_oracle_and_keeps_divergence_free(dim, nf, m, dtype):
    faces = [inputs.uniform_faces(n, 0, 2 * np.pi) for n in nf]
    og = OGrid(faces, ["periodic"] * dim, 0.0)
    u, _ = poisson.project(og, inputs.random_field((dim,) + og.shape, 3))
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
    uc = filter_face_average(torch.tensor(u, dtype=dtype, device="cuda"), m).double().cpu().numpy()
    ref = diagnostics.face_average_filter(u, dim, m)
    tol = 1e-15 if dtype == torch.float64 else 1e-7
    assert np.max(np.abs(uc - ref)) <= tol * np.max(np.abs(ref)) * 4
    gc = OGrid([inputs.uniform_faces(n // m, 0, 2 * np.pi) for n in nf], ["periodic"] * dim, 0.0)
    if dtype == torch.float64:
        assert np.max(np.abs(op.divergence(gc, uc))) < 1e-11 * np.max(np.abs(u)) * max(nf)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [32, 24])
def test_spectrum_matches_oracle(n, dtype):
    faces = inputs.periodic_box(n, 3)
    g = Grid(faces, ["periodic"] * 3, 0.01, dtype=dtype)
    og = OGrid(faces, ["periodic"] * 3, 0.01)
    u, _ = poisson.project(og, inputs.spectrum_velocity_raw(n, 3, seed=2, k0=4.0))
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
    E = g.spectrum(torch.tensor(u, dtype=dtype, device="cuda")).cpu().numpy()
    ref = diagnostics.shell_spectrum(u)
    tol = 1e-12 if dtype == torch.float64 else 2e-5
    assert np.max(np.abs(E - ref)) <= tol * np.max(ref)
    # total energy: sum_k E(k) = 1/2 mean |u|^2 summed over components (Parseval)
    assert abs(E.sum() - 0.5 * np.sum(np.mean(u ** 2, axis=(1, 2, 3)))) <= 1e-3 * E.sum() + (1e-12 if dtype == torch.float64 else 1e-5)
