"""The FP64 step in double-float arithmetic (ins_set_f64_arithmetic) against the FP64 oracle.

Double-float keeps F, the Poisson FFTs and the stage updates on the FP32 pipe with about 48
significant bits; storage, the final update of the caller's field and the CFL rule stay FP64.
It must meet the FP64 tolerances of the native path: relative field error <= 1e-12 per step and
<= 1e-10 after 100 steps against the oracle, the next CFL time step bit for bit, and graph
replay (ins_step_n) bit-identical to plain steps. FFT lengths without register kernels run the
shared-memory Stockham passes in double-float; grids with odd nx keep native FP64 and refuse
the setting.
"""

import numpy as np
import pytest
import torch

from oracle import poisson, timestep, diagnostics
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300.solver import Grid
from paper_2604_18536_b300._lib import InsError, INS_ERR_UNSUPPORTED

pytestmark = pytest.mark.gpu
U = inputs.uniform_faces
PI = np.pi

CASES = {
    "p3reg": ([U(32, 0, 2 * PI), U(16, 0, 1.0), U(64, 0, 3.0)], 0.02),
    "p3r12": ([U(48, 0, 2 * PI), U(96, 0, 1.5 * PI), U(16, 0, 2 * PI)], 0.02),   # radix-3 lengths
    "p3ragged": ([U(192, 0, 2 * PI), U(16, 0, 1.0), U(128, 0, 2 * PI)], 0.01),
    "p2r12": ([U(192, 0, 2 * PI), U(96, 0, 1.5 * PI)], 0.02),
    "p2pow": ([U(256, 0, 2 * PI), U(64, 0, 2 * PI)], 0.01),
    # y and z lines of 256 in the strided passes (64 in p3reg and p2pow)
    "p3r4y": ([U(16, 0, 2 * PI), U(256, 0, 2 * PI), U(16, 0, 1.0)], 0.02),
    "p3r4z": ([U(32, 0, 2 * PI), U(16, 0, 1.0), U(256, 0, 3.0)], 0.02),
    # lengths without register kernels: the shared-memory Stockham passes in double-float
    "p3stock": ([U(40, 0, 2 * PI), U(24, 0, 1.5 * PI), U(36, 0, 3.0)], 0.02),
    "p3stock7": ([U(14, 0, 2 * PI), U(20, 0, 1.5 * PI), U(42, 0, 3.0)], 0.02),
}


def make(name, seed=3, spectrum=False):
    faces, nu = CASES[name]
    bc = ["periodic"] * len(faces)
    og = OGrid(faces, bc, nu)
    g = Grid(faces, bc, nu, dtype=torch.float64)
    if spectrum and len(faces) == 3 and len({len(f) for f in faces}) == 1:
        raw = inputs.spectrum_velocity_raw(len(faces[0]) - 1, 3, seed=seed, k0=4.0)
    else:
        raw = inputs.random_field((og.dim,) + og.shape, seed)
    u0, _ = poisson.project(og, raw)
    u0 /= np.sqrt(2 * diagnostics.kinetic_energy(og, u0))
    return og, g, u0


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("name", list(CASES))
def test_default_is_double_float_where_supported(name):
    og, g, u0 = make(name)
    assert g.f64_arithmetic() == "double-float"
    g.close()


@pytest.mark.parametrize("mode", ["double-float", "native"])
@pytest.mark.parametrize("name", list(CASES))
def test_step_matches_oracle(name, mode):
    og, g, u0 = make(name)
    g.set_f64_arithmetic(mode)
    u = dev(u0)
    dt = g.cfl_dt(u, 0.3)
    assert dt.item() == timestep.cfl_dt(og, u0, 0.3)
    g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=0.3)
    u1 = u.cpu().numpy()
    ref = timestep.rk4_step(og, u0, timestep.cfl_dt(og, u0, 0.3))
    err = rel(u1, ref)
    assert err <= 1e-12, (mode, err)
    assert dt.item() == timestep.cfl_dt(og, u1, 0.3)       # next dt from the FP64 result, bit for bit
    g.close()


def test_double_float_differs_from_native_only_at_rounding_level():
    og, g, u0 = make("p3reg", seed=8)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ua, ub = dev(u0), dev(u0)
    g.step(ua, dt=dt)
    g.set_f64_arithmetic("native")
    g.step(ub, dt=dt)
    d = rel(ua.cpu().numpy(), ub.cpu().numpy())
    assert 0.0 < d <= 1e-13, d        # different arithmetic, same FP64-level result
    g.close()


@pytest.mark.parametrize("name", ["p3reg", "p2pow", "p3r4z", "p3stock"])
def test_100_steps(name):
    """<= 1e-10 after 100 steps against the oracle (fixed dt)."""
    og, g, u0 = make(name, seed=4)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    u = dev(u0)
    g.step_n(u, 100, dt=dt)
    ref = timestep.integrate(og, u0, dt, 100)
    err = rel(u.cpu().numpy(), ref)
    assert err <= 1e-10, err
    g.close()


def test_graph_replay_is_bit_identical():
    og, g, u0 = make("p3r12", seed=5)
    ua, ub = dev(u0), dev(u0)
    da, db = g.cfl_dt(ua, 0.3), g.cfl_dt(ub, 0.3)
    g.step_n(ua, 4, dt_dev=da, next_dt_dev=da, cfl=0.3)
    for _ in range(4):
        g.step(ub, dt_dev=db, next_dt_dev=db, cfl=0.3)
    assert torch.equal(ua, ub) and torch.equal(da, db)
    g.close()


def test_unsupported_grids_stay_native():
    faces = [U(45, 0, 2 * PI), U(24, 0, 1.5 * PI), U(36, 0, 3.0)]    # odd nx (the two-cell update)
    g = Grid(faces, ["periodic"] * 3, 0.02, dtype=torch.float64)
    assert g.f64_arithmetic() == "native"
    with pytest.raises(InsError) as e:
        g.set_f64_arithmetic("double-float")
    assert e.value.status == INS_ERR_UNSUPPORTED
    g.close()
    c2 = Grid([U(32, 0, 4 * PI), inputs.tanh_faces(12, 0, 2, 1.5)], ["periodic", "wall"], 0.05, [1.0, 0],
              dtype=torch.float64)                                         # 2-D channels stay native
    assert c2.f64_arithmetic() == "native"
    c2.close()
    g32 = Grid(inputs.periodic_box(32, 3), ["periodic"] * 3, 0.01, dtype=torch.float32)
    assert g32.f64_arithmetic() == "native"
    g32.close()


def test_non_finite_flag_and_wray3():
    """A NaN in the field sets the non-finite flag as in native mode; Wray's low-storage step in
    double-float arithmetic is within 1e-12 of the oracle and its CFL maxima are bit-exact."""
    og, g, u0 = make("p3reg", seed=6)
    u0[0, 3, 4, 5] = np.nan
    u = dev(u0)
    g.step(u, dt=1e-3)
    with pytest.raises(InsError):
        g.check_finite()
    g.close()
    faces, nu = CASES["p3reg"]
    gw = Grid(faces, ["periodic"] * 3, nu, dtype=torch.float64, scheme="wray3")
    ow = OGrid(faces, ["periodic"] * 3, nu)
    _, _, v0 = make("p3reg", seed=7)
    dt = 0.5 * timestep.cfl_dt(ow, v0, 0.3)
    assert gw.f64_arithmetic() == "double-float"
    v = dev(v0)
    dtd = torch.tensor([dt], dtype=torch.float64, device="cuda")
    gw.step(v, dt_dev=dtd, next_dt_dev=dtd, cfl=0.3)
    v1 = v.cpu().numpy()
    assert rel(v1, timestep.wray3_step(ow, v0, dt)) <= 1e-12
    assert dtd.item() == timestep.cfl_dt(ow, v1, 0.3)
    w = dev(v0)
    gw.step_n(w, 50, dt=dt)
    assert rel(w.cpu().numpy(), timestep.integrate(ow, v0, dt, 50, scheme="wray3")) <= 1e-10
    gw.close()


@pytest.mark.parametrize("mode", ["double-float", "native"])
@pytest.mark.parametrize("name", ["p3reg", "p3r12", "p3ragged", "p3r4y", "p3r4z", "p3stock"])
def test_step_vjp_matches_oracle(name, mode):
    """The step pullback in double-float arithmetic (3-D grids): ubar within 1e-12 of the oracle's,
    nubar within 5e-11 relative."""
    from oracle import adjoint
    og, g, u0 = make(name, seed=9)
    g.set_f64_arithmetic(mode)
    ybar = inputs.random_field((og.dim,) + og.shape, 109)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ub, nb = g.step_vjp(dev(u0), dev(ybar), dt=dt)
    ub_o, nb_o = adjoint.rk4_step_vjp(og, u0, dt, ybar)
    err = rel(ub.cpu().numpy(), ub_o)
    assert err <= 1e-12, (mode, err)
    assert abs(nb.item() - nb_o) <= 5e-11 * abs(nb_o)
    g.close()


def test_step_vjp_central_differences_double_float():
    """<ubar, v> against central differences of the double-float forward step (eps = 1e-6)."""
    og, g, u0 = make("p3reg", seed=10)
    c = inputs.random_field((og.dim,) + og.shape, 110)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ub, _ = g.step_vjp(dev(u0), dev(c), dt=dt)
    ub = ub.cpu().numpy()
    eps = 1e-6

    def L(u):
        t = dev(u)
        g.step(t, dt=dt)
        return float(np.sum(c * t.cpu().numpy()))

    for seed in range(3):
        v, _ = poisson.project(og, inputs.random_field(u0.shape, 210 + seed))
        fd = (L(u0 + eps * v) - L(u0 - eps * v)) / (2 * eps)
        assert abs(fd - np.sum(ub * v)) <= 1e-7 * max(1.0, abs(fd))
    g.close()


def test_wray3_step_vjp_matches_oracle():
    """The Wray3 step pullback in double-float arithmetic against the oracle's (<= 1e-12)."""
    from oracle import adjoint
    faces, nu = CASES["p3r12"]
    g = Grid(faces, ["periodic"] * 3, nu, dtype=torch.float64, scheme="wray3")
    og = OGrid(faces, ["periodic"] * 3, nu)
    _, _, u0 = make("p3r12", seed=12)
    ybar = inputs.random_field((3,) + og.shape, 112)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ub, nb = g.step_vjp(dev(u0), dev(ybar), dt=dt)
    ub_o, nb_o = adjoint.wray3_step_vjp(og, u0, dt, ybar)
    assert rel(ub.cpu().numpy(), ub_o) <= 1e-12
    assert abs(nb.item() - nb_o) <= 5e-11 * abs(nb_o)
    g.close()


# ---------------------------------------------------------------- channels (walls in y)
# The double-float step also runs on 3-D channels whose periodic x and z lengths have register FFT
# kernels: stretched wall-normal rows, wall ghosts and the top wall face of u^y in double-float, the
# wall-normal Poisson solve by the double-float Thomas sweep.
CHB = ["periodic", "wall", "periodic"]
CH_CASES = {
    "c3df": [U(64, 0, 4 * PI), inputs.tanh_faces(20, 0, 2, 1.5), U(32, 0, 4 * PI / 3)],
    "c3dfodd": [U(96, 0, 4 * PI), inputs.tanh_faces(15, 0, 2, 1.5), U(16, 0, 4 * PI / 3)],
    "c3dfstock": [U(40, 0, 4 * PI), inputs.tanh_faces(12, 0, 2, 1.5), U(20, 0, 4 * PI / 3)],   # Stockham x, z
}


def make_channel(name, seed):
    faces = CH_CASES[name]
    og = OGrid(faces, CHB, 1 / 180, [1.0, 0.0, 0.0])
    g = Grid(faces, CHB, 1 / 180, [1.0, 0.0, 0.0], dtype=torch.float64)
    u0, _ = poisson.project(og, inputs.channel_velocity_raw(faces, seed=seed))
    return og, g, u0


@pytest.mark.parametrize("mode", ["double-float", "native"])
@pytest.mark.parametrize("name", list(CH_CASES))
def test_channel_step_matches_oracle(name, mode):
    og, g, u0 = make_channel(name, 21)
    assert g.f64_arithmetic() == "double-float"
    g.set_f64_arithmetic(mode)
    u = dev(u0)
    dt = g.cfl_dt(u, 0.3)
    assert dt.item() == timestep.cfl_dt(og, u0, 0.3)
    g.step(u, dt_dev=dt, next_dt_dev=dt, cfl=0.3)
    u1 = u.cpu().numpy()
    err = rel(u1, timestep.rk4_step(og, u0, timestep.cfl_dt(og, u0, 0.3)))
    assert err <= 1e-12, (mode, err)
    assert dt.item() == timestep.cfl_dt(og, u1, 0.3)
    assert np.all(u1[1][:, -1, :] == 0.0)    # the top wall face of u^y stays 0
    g.close()


def test_channel_100_steps_and_graph_replay():
    """<= 1e-10 after 100 steps against the oracle (fixed dt); ins_step_n bit-identical to plain steps."""
    og, g, u0 = make_channel("c3df", 22)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    u = dev(u0)
    g.step_n(u, 100, dt=dt)
    assert rel(u.cpu().numpy(), timestep.integrate(og, u0, dt, 100)) <= 1e-10
    ua, ub = dev(u0), dev(u0)
    da, db = g.cfl_dt(ua, 0.3), g.cfl_dt(ub, 0.3)
    g.step_n(ua, 4, dt_dev=da, next_dt_dev=da, cfl=0.3)
    for _ in range(4):
        g.step(ub, dt_dev=db, next_dt_dev=db, cfl=0.3)
    assert torch.equal(ua, ub) and torch.equal(da, db)
    g.close()


def test_channel_double_float_differs_from_native_only_at_rounding_level():
    og, g, u0 = make_channel("c3dfodd", 23)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ua, ub = dev(u0), dev(u0)
    g.step(ua, dt=dt)
    g.set_f64_arithmetic("native")
    g.step(ub, dt=dt)
    d = rel(ua.cpu().numpy(), ub.cpu().numpy())
    assert 0.0 < d <= 1e-13, d
    g.close()


@pytest.mark.parametrize("mode", ["double-float", "native"])
@pytest.mark.parametrize("name", list(CH_CASES))
def test_channel_step_vjp_matches_oracle(name, mode):
    """The channel step pullback in double-float arithmetic: ubar within 1e-12 of the oracle's (the
    stored top wall faces of u^y returned as 0), nubar within 5e-11 relative."""
    from oracle import adjoint
    og, g, u0 = make_channel(name, 24)
    g.set_f64_arithmetic(mode)
    ybar = inputs.random_field((3,) + og.shape, 124)
    ybar[1][:, -1, :] = 0.0                  # the top wall faces of u^y are no unknowns
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ub, nb = g.step_vjp(dev(u0), dev(ybar), dt=dt)
    ub_o, nb_o = adjoint.rk4_step_vjp(og, u0, dt, ybar)
    ub = ub.cpu().numpy()
    assert rel(ub, ub_o) <= 1e-12, (mode, rel(ub, ub_o))
    assert abs(nb.item() - nb_o) <= 5e-11 * abs(nb_o)
    assert np.all(ub[1][:, -1, :] == 0.0)
    g.close()


def test_channel_step_vjp_central_differences_double_float():
    """<ubar, v> against central differences of the double-float channel step (eps = 1e-6). The
    directions v keep the stored top wall faces of u^y at 0: they are no unknowns, and the pullback
    returns 0 there."""
    og, g, u0 = make_channel("c3df", 25)
    c = inputs.random_field((3,) + og.shape, 125)
    c[1][:, -1, :] = 0.0
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ub = g.step_vjp(dev(u0), dev(c), dt=dt)[0].cpu().numpy()
    eps = 1e-6

    def L(u):
        t = dev(u)
        g.step(t, dt=dt)
        return float(np.sum(c * t.cpu().numpy()))

    for seed in range(3):
        v, _ = poisson.project(og, inputs.random_field(u0.shape, 225 + seed))
        v[1][:, -1, :] = 0.0
        fd = (L(u0 + eps * v) - L(u0 - eps * v)) / (2 * eps)
        assert abs(fd - np.sum(ub * v)) <= 1e-7 * max(1.0, abs(fd))
    g.close()


def test_channel_wray3_double_float():
    """Wray's low-storage RK3 on a channel in double-float arithmetic: within 1e-12 of the oracle per
    step (the next CFL step bit-exact, the top wall face of u^y kept at 0) and 1e-10 after 50 steps."""
    faces = CH_CASES["c3df"]
    og = OGrid(faces, CHB, 1 / 180, [1.0, 0.0, 0.0])
    g = Grid(faces, CHB, 1 / 180, [1.0, 0.0, 0.0], dtype=torch.float64, scheme="wray3")
    assert g.f64_arithmetic() == "double-float"
    u0, _ = poisson.project(og, inputs.channel_velocity_raw(faces, seed=26))
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    u = dev(u0)
    dtd = torch.tensor([dt], dtype=torch.float64, device="cuda")
    g.step(u, dt_dev=dtd, next_dt_dev=dtd, cfl=0.3)
    u1 = u.cpu().numpy()
    assert rel(u1, timestep.wray3_step(og, u0, dt)) <= 1e-12
    assert dtd.item() == timestep.cfl_dt(og, u1, 0.3)
    assert np.all(u1[1][:, -1, :] == 0.0)
    w = dev(u0)
    g.step_n(w, 50, dt=dt)
    assert rel(w.cpu().numpy(), timestep.integrate(og, u0, dt, 50, scheme="wray3")) <= 1e-10
    g.close()
