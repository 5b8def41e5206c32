"""Eddy-viscosity closures (ins_set_eddy_viscosity) on the GPU against the oracle.

nu_t fields, the right-hand side and one RK4 step with the model in F, element by element on
seeded fields: FP64 relative L2 error <= 1e-12, FP32 (oracle on the FP32-rounded input)
<= 2e-5 for F and the step, 1e-5 for nu_t. The grids span several 32 x 8 tiles with ragged
tails and unequal spacings: a triply periodic box and a channel (walls in y, tanh-stretched
rows, the wall ghost rules of the velocity and of nu_t).
"""

import numpy as np
import pytest
import torch

from oracle import eddy, poisson, timestep, diagnostics
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300.solver import Grid
from paper_2604_18536_b300._lib import InsError
from test_gpu_parity import rounded, dev, host, rel

pytestmark = pytest.mark.gpu
U = inputs.uniform_faces
MODELS = ["smagorinsky", "wale", "qr", "vreman", "constant"]
TOL = {torch.float64: 1e-12, torch.float32: 2e-5}
NUT_TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


KINDS = ["periodic", "channel"]


def grids(dtype, nu=0.01, kind="periodic"):
    if kind == "channel":
        faces, bc, force = inputs.channel_faces(36, 20, 28), ["periodic", "wall", "periodic"], [1.0, 0.0, 0.0]
    else:
        faces, bc, force = [U(40, 0, 2 * np.pi), U(24, 0, 1.5 * np.pi), U(12, 0, 1.0)], ["periodic"] * 3, None
    og = OGrid(faces, bc, nu, force)
    gg = Grid(faces, bc, nu, force, dtype=dtype)
    return og, gg


def field(og, seed, dtype):
    u = inputs.random_field((3,) + og.shape, seed)
    for a in range(3):
        u[a] *= og.face_mask(a)
    u, _ = poisson.project(og, u)
    return rounded(u, dtype)


def oc(model):
    return Grid.EDDY_DEFAULT_C.get(model, 0.02)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("model", MODELS)
def test_eddy_viscosity_field(model, dtype, kind):
    og, gg = grids(dtype, kind=kind)
    u = field(og, 31, dtype)
    gg.set_eddy_viscosity(model, oc(model))
    nu = host(gg.eddy_viscosity(dev(u, dtype)))
    ref = eddy.eddy_viscosity(og, u, model, oc(model))
    assert rel(nu, ref) <= NUT_TOL[dtype], rel(nu, ref)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("model", MODELS)
def test_rhs_with_eddy_model(model, dtype, kind):
    og, gg = grids(dtype, kind=kind)
    u = field(og, 32, dtype)
    gg.set_eddy_viscosity(model, oc(model))
    dudt = gg.rhs(dev(u, dtype))
    ref, _ = poisson.rhs(og, u, eddy.closure(og, model, oc(model)))
    assert rel(host(dudt), ref) <= TOL[dtype], rel(host(dudt), ref)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("model", ["smagorinsky", "wale"])
def test_step_with_eddy_model(model, dtype, kind):
    og, gg = grids(dtype, kind=kind)
    u = field(og, 33, dtype)
    dt = 0.5 * timestep.cfl_dt(og, u, 0.3)
    gg.set_eddy_viscosity(model, oc(model))
    ut = dev(u, dtype)
    gg.step(ut, dt=dt)
    ref = timestep.rk4_step(og, u, dt, eddy.closure(og, model, oc(model)))
    assert rel(host(ut), ref) <= TOL[dtype], rel(host(ut), ref)


def test_eddy_model_rules():
    og, gg = grids(torch.float64)
    u = dev(field(og, 34, torch.float64), torch.float64)
    with pytest.raises(InsError):
        gg.eddy_viscosity(u)                      # no model attached
    gg.set_eddy_viscosity("smagorinsky")
    with pytest.raises(InsError):
        gg.step_vjp(u, u.clone(), dt=1e-3)        # no pullback for eddy models
    a = u.clone()
    gg.step(a, dt=1e-3)
    gg.set_eddy_viscosity(None)                   # detached: the plain step again
    b = u.clone()
    c = u.clone()
    gg.step(b, dt=1e-3)
    g2 = Grid(og.faces, ["periodic"] * 3, og.nu, dtype=torch.float64)
    g2.step(c, dt=1e-3)
    assert torch.equal(b, c) and not torch.equal(a, b)
    flat = Grid([U(8, 0, 1.0), U(8, 0, 1.0)], ["periodic"] * 2, 0.01, dtype=torch.float64)
    with pytest.raises(InsError):
        flat.set_eddy_viscosity("wale")           # 3-D grids only


def test_eddy_models_dissipate_energy():
    """Inviscid LES of a random field: every model removes energy, the no-model run keeps it."""
    og, gg = grids(torch.float64, nu=0.0)
    u0 = field(og, 35, torch.float64)
    dt = 0.3 * timestep.cfl_dt(og, u0, 0.3)
    ke0 = diagnostics.kinetic_energy(og, u0)
    kes = {}
    for model in [None, "smagorinsky", "wale", "qr", "vreman"]:
        gg.set_eddy_viscosity(model)
        u = dev(u0, torch.float64)
        for _ in range(5):
            gg.step(u, dt=dt)
        kes[model] = diagnostics.kinetic_energy(og, host(u))
    assert abs(kes[None] - ke0) <= 1e-3 * ke0      # the no-model scheme conserves energy up to O(dt^4)
    for model in ["smagorinsky", "wale", "qr", "vreman"]:
        assert kes[model] < kes[None] - 1e-6 * ke0, model
