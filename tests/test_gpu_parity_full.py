"""GPU versus the FP64 oracle at the workloads' full sizes, in the launch configuration of the benchmark.

The small parity cases elsewhere span tiles, chunks and ragged tails; these run the sizes whose
launch shapes the benchmark times (z chunks from the wave count of resident CTAs, persistent FFT
CTAs walking many tiles, the half-width vector variants at nx = 192):

* one RK4 step of the 256^3 isotropic-turbulence field (nu = 1/1600, spectrum k0 = 4, unit KE,
  CFL 0.3 with the device-side time step), FP64 and FP32, through ins_step_n as the benchmark calls it;
* one RK4 step of the 192 x 128 x 192 tanh channel (nu = 1/180, f = (1, 0, 0)), FP64 and FP32;
* the step VJP of the 128^3 differentiation field (nu = 1/1000, u* + 0.1 perturbation);
* the CNN closure forward on a batch of eight 64^3 fields, samples 0 and 7 against the oracle.

Each input is rounded to FP32 once, so that the FP64 and FP32 runs and the oracle all start from
the same values and one oracle evaluation serves both precisions. Tolerances are those of the
small cases: relative L2 field error <= 1e-12 (FP64) and <= 2e-5 (FP32) per step; the CFL time
step bit for bit.
"""

import math

import numpy as np
import pytest
import torch

from oracle import adjoint, poisson, timestep, diagnostics, closure as oc
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300.closure import Closure, init_params
from paper_2604_18536_b300.solver import Grid

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}
DTYPES = [torch.float64, torch.float32]
CFL = 0.3


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def dev(x, dtype):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# ------------------------------------------------------------------ 256^3 isotropic turbulence
@pytest.fixture(scope="module")
def hit256():
    n, nu = 256, 1.0 / 1600
    faces = inputs.periodic_box(n, 3)
    og = OGrid(faces, ["periodic"] * 3, nu)
    u0, _ = poisson.project(og, inputs.spectrum_velocity_raw(n, 3, seed=0, k0=4.0))
    u0 = f32(u0 / math.sqrt(diagnostics.kinetic_energy(og, u0)))
    dt = timestep.cfl_dt(og, u0, CFL)
    ref = timestep.rk4_step(og, u0, dt)
    return dict(faces=faces, nu=nu, og=og, u0=u0, dt=dt, ref=ref)


@pytest.mark.parametrize("dtype", DTYPES)
def test_hit256_step_matches_oracle(hit256, dtype):
    h = hit256
    g = Grid(h["faces"], ["periodic"] * 3, h["nu"], dtype=dtype)
    u = dev(h["u0"], dtype)
    dt = g.cfl_dt(u, CFL)
    assert dt.item() == h["dt"]                                   # bit for bit
    g.step_n(u, 1, dt_dev=dt, next_dt_dev=dt, cfl=CFL)            # the benchmark's call
    u1 = host(u)
    err = rel(u1, h["ref"])
    print(f"256^3 {dtype}: relative error {err:.3e} after one step")
    assert err <= TOL[dtype]
    assert dt.item() == timestep.cfl_dt(h["og"], u1, CFL)         # next dt from u_{n+1}, bit for bit
    g.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_hit256_graph_replay_equals_plain_steps(hit256, dtype):
    """ins_step_n (graph replay after the first step) gives the bits of the same number of ins_step calls."""
    h = hit256
    g = Grid(h["faces"], ["periodic"] * 3, h["nu"], dtype=dtype)
    ua, ub = dev(h["u0"], dtype), dev(h["u0"], dtype)
    da, db = g.cfl_dt(ua, CFL), g.cfl_dt(ub, CFL)
    g.step_n(ua, 3, dt_dev=da, next_dt_dev=da, cfl=CFL)
    for _ in range(3):
        g.step(ub, dt_dev=db, next_dt_dev=db, cfl=CFL)
    assert torch.equal(ua, ub) and torch.equal(da, db)
    g.close()


# ------------------------------------------------------------------ 192 x 128 x 192 channel
@pytest.fixture(scope="module")
def channel192():
    faces = inputs.channel_faces(192, 128, 192)
    bc = ["periodic", "wall", "periodic"]
    og = OGrid(faces, bc, 1.0 / 180, [1.0, 0.0, 0.0])
    u0, _ = poisson.project(og, inputs.channel_velocity_raw(faces, seed=0))
    u0 = f32(u0)
    dt = timestep.cfl_dt(og, u0, CFL)
    ref = timestep.rk4_step(og, u0, dt)
    return dict(faces=faces, bc=bc, og=og, u0=u0, dt=dt, ref=ref)


@pytest.mark.parametrize("dtype", DTYPES)
def test_channel192_step_matches_oracle(channel192, dtype):
    c = channel192
    g = Grid(c["faces"], c["bc"], 1.0 / 180, [1.0, 0.0, 0.0], dtype=dtype)
    u = dev(c["u0"], dtype)
    dt = g.cfl_dt(u, CFL)
    assert dt.item() == c["dt"]
    g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=CFL)                 # the benchmark's call
    u1 = host(u)
    err = rel(u1, c["ref"])
    print(f"channel 192x128x192 {dtype}: relative error {err:.3e} after one step")
    assert err <= TOL[dtype]
    assert dt.item() == timestep.cfl_dt(c["og"], u1, CFL)
    assert np.all(u1[1][:, -1, :] == 0.0)                         # top wall faces of u^y stay 0
    g.close()


# ------------------------------------------------------------------ 128^3 step VJP
@pytest.fixture(scope="module")
def vjp128():
    n, nu = 128, 1.0 / 1000
    faces = inputs.periodic_box(n, 3)
    og = OGrid(faces, ["periodic"] * 3, nu)
    ustar, _ = poisson.project(og, inputs.spectrum_velocity_raw(n, 3, seed=0, k0=4.0, kmax=n // 4))
    ustar /= math.sqrt(diagnostics.kinetic_energy(og, ustar))
    pert, _ = poisson.project(og, inputs.spectrum_velocity_raw(n, 3, seed=1, k0=4.0, kmax=n // 4))
    pert *= 0.1 / math.sqrt(diagnostics.kinetic_energy(og, pert))
    u0 = f32(ustar + pert)
    dt = timestep.cfl_dt(og, f32(ustar), CFL)
    ybar = f32(inputs.random_field((3,) + og.shape, 11))
    ubar, nubar = adjoint.rk4_step_vjp(og, u0, dt, ybar)
    return dict(faces=faces, nu=nu, u0=u0, dt=dt, ybar=ybar, ubar=ubar, nubar=nubar)


@pytest.mark.parametrize("dtype", DTYPES)
def test_vjp128_matches_oracle(vjp128, dtype):
    v = vjp128
    g = Grid(v["faces"], ["periodic"] * 3, v["nu"], dtype=dtype)
    dtd = torch.tensor([v["dt"]], dtype=torch.float64, device="cuda")
    ub, nb = g.step_vjp(dev(v["u0"], dtype), dev(v["ybar"], dtype), dt_dev=dtd)
    err = rel(host(ub), v["ubar"])
    print(f"128^3 step VJP {dtype}: relative error {err:.3e}")
    assert err <= TOL[dtype]
    assert abs(nb.item() - v["nubar"]) <= 50 * TOL[dtype] * abs(v["nubar"])
    g.close()


# ------------------------------------------------------------------ closure, batch of 8 x 64^3
def test_closure_forward_batch8_64():
    """Eight 64^3 fields through the closure one after another (the training batch's calls);
    samples 0 and 7 against the oracle's network on the same parameters. Independent BF16
    roundings on both sides let single activations differ by one BF16 ulp, so the outputs are
    compared in relative L2 norm with the bound of the smaller end-to-end test."""
    n = 64
    faces = inputs.periodic_box(n, 3)
    g = Grid(faces, ["periodic"] * 3, 1.0 / 2000, dtype=torch.float32)
    W, b = init_params(0, 1.0)
    for bb in b:
        bb.copy_(torch.linspace(-0.1, 0.1, bb.numel()))
    c = Closure(g)
    c.set_params(W, b)
    params = [(oc.bf16(w.double().cpu().numpy()), bb.double().cpu().numpy()) for w, bb in zip(W, b)]
    us, ms = [], []
    for s in range(8):
        raw = inputs.spectrum_velocity_raw(n, 3, seed=s, k0=4.0, kmax=n // 2 - 1)
        raw = f32(raw / math.sqrt(np.mean(raw ** 2)))
        us.append(raw)
        ms.append(c.forward(dev(raw, torch.float32)))
    c.check()
    torch.cuda.synchronize()
    for s in (0, 7):
        want = oc.forward(params, us[s])
        err = rel(host(ms[s]), want)
        print(f"closure 64^3 sample {s}: relative error {err:.3e}")
        assert err <= 5e-3
    c.close()
    g.close()
