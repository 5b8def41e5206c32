"""GPU (libins, sm_103a) versus the FP64 oracle, element by element on seeded inputs.

Tolerances (relative L2 field error): FP64 <= 1e-12 per call/step and <= 1e-10 after
100 steps; FP32 <= 2e-5 per call/step (the FP32 path is compared with the FP64 oracle
run on the same FP32-rounded input). The CFL time step is compared bit for bit.
Sizes span several 32 x 8 stencil tiles and z chunks with ragged tails, and FFT
lengths with every radix (2, 3, 4, 5, 7, 8) and the register-path lengths (16 .. 256, 48, 96, 192).
"""

import numpy as np
import pytest
import torch

from oracle import operators as op, poisson, timestep, diagnostics
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300.solver import Grid
from paper_2604_18536_b300._lib import InsError, INS_ERR_NONFINITE

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}
PI = np.pi


def case(name):
    U = inputs.uniform_faces
    if name == "p2":
        return dict(faces=[U(72, 0, 2 * PI), U(40, 0, 1.5 * PI)], bc=["periodic"] * 2, nu=0.05, force=None)
    if name == "p3":
        return dict(faces=[U(40, 0, 2 * PI), U(24, 0, 1.5 * PI), U(36, 0, 3.0)], bc=["periodic"] * 3, nu=0.02,
                    force=None)
    if name == "p3tiny":
        return dict(faces=[U(6, 0, 1.0), U(10, 0, 2.0), U(14, 0, 1.5)], bc=["periodic"] * 3, nu=0.01, force=None)
    if name == "p3reg":     # register-path FFT lengths 32 (8x4), 16 (4x4), 64 (8x8)
        return dict(faces=[U(32, 0, 2 * PI), U(16, 0, 1.0), U(64, 0, 3.0)], bc=["periodic"] * 3, nu=0.02,
                    force=None)
    if name == "p3reg2":    # 256 (16x16) and 128 (16x8)
        return dict(faces=[U(256, 0, 2 * PI), U(8, 0, 1.0), U(128, 0, 2 * PI)], bc=["periodic"] * 3, nu=0.01,
                    force=None)
    if name == "p3r12":     # register-path lengths with radix-3 and radix-12 butterflies: 48 (16x3), 192 (16x12)
        return dict(faces=[U(48, 0, 2 * PI), U(8, 0, 1.0), U(192, 0, 2 * PI)], bc=["periodic"] * 3, nu=0.02,
                    force=None)
    if name == "p2r12":     # 192 (16x12) in x, 96 (16x6) in the fused y pass
        return dict(faces=[U(192, 0, 2 * PI), U(96, 0, 1.5 * PI)], bc=["periodic"] * 2, nu=0.02, force=None)
    if name == "c3r12":     # channel with x 96 (16x6) and z 48 (16x3)
        return dict(faces=[U(96, 0, 4 * PI), inputs.tanh_faces(12, 0, 2, 1.5), U(48, 0, 4 * PI / 3)],
                    bc=["periodic", "wall", "periodic"], nu=1 / 180, force=[1.0, 0.0, 0.0])
    if name == "c3odd":     # odd wall-normal size: the two-ended wall solve meets at an interior row
        return dict(faces=[U(24, 0, 4 * PI), inputs.tanh_faces(15, 0, 2, 1.5), U(20, 0, 4 * PI / 3)],
                    bc=["periodic", "wall", "periodic"], nu=1 / 180, force=[1.0, 0.0, 0.0])
    if name == "c2odd":
        return dict(faces=[U(28, 0, 4 * PI), inputs.tanh_faces(7, 0, 2, 1.5)], bc=["periodic", "wall"], nu=0.05,
                    force=[1.0, 0.0])
    if name == "c3reg":     # channel with register-path x and z
        return dict(faces=[U(64, 0, 4 * PI), inputs.tanh_faces(20, 0, 2, 1.5), U(32, 0, 4 * PI / 3)],
                    bc=["periodic", "wall", "periodic"], nu=1 / 180, force=[1.0, 0.0, 0.0])
    if name == "c3":
        return dict(faces=inputs.channel_faces(36, 20, 28), bc=["periodic", "wall", "periodic"], nu=1 / 180,
                    force=[1.0, 0.0, 0.0])
    if name == "c2":
        return dict(faces=[U(30, 0, 4 * PI), inputs.tanh_faces(18, 0, 2, 1.5)], bc=["periodic", "wall"], nu=0.05,
                    force=[1.0, 0.0])
    if name == "cu3":       # uniform wall-normal spacing: the DCT-II wall solve
        return dict(faces=[U(40, 0, 4 * PI), U(24, 0, 2.0), U(20, 0, 4 * PI / 3)],
                    bc=["periodic", "wall", "periodic"], nu=1 / 180, force=[1.0, 0.0, 0.0])
    if name == "cu2":
        return dict(faces=[U(30, 0, 4 * PI), U(18, 0, 2.0)], bc=["periodic", "wall"], nu=0.05, force=[1.0, 0.0])
    raise KeyError(name)


CASES = ["p2", "p3", "p3tiny", "p3reg", "p3reg2", "p3r12", "p2r12", "c3", "c3reg", "c3r12", "c3odd", "c2", "c2odd",
         "cu3", "cu2", "cu3dct", "cu2dct"]
DTYPES = [torch.float64, torch.float32]


def grids(name, dtype):
    dct = name.endswith("dct")          # the uniform-y channel cases with the DCT-II y solve
    c = case(name[:-3] if dct else name)
    og = OGrid(c["faces"], c["bc"], c["nu"], c["force"])
    gg = Grid(c["faces"], c["bc"], c["nu"], c["force"], dtype=dtype)
    if dct:
        gg.set_wall_solver("dct")
    return og, gg


def rand_u(og, seed, project=False, scale=1.0):
    u = inputs.random_field((og.dim,) + og.shape, seed, scale)
    for a in range(og.dim):
        u[a] *= og.face_mask(a)
    if project:
        u, _ = poisson.project(og, u)
    return u


def dev(x, dtype):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rounded(x, dtype):
    """The input as the GPU sees it (FP32 rounding), in FP64 for the oracle."""
    return x.astype(np.float32).astype(np.float64) if dtype == torch.float32 else x


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def demean(og, p):
    v = og.cell_volume()
    return p - np.sum(v * p) / np.sum(v)


# ------------------------------------------------------------------ operators
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", CASES)
def test_rhs_parity(name, dtype):
    og, gg = grids(name, dtype)
    u = rounded(rand_u(og, 1), dtype)
    p = gg.new_scalar()
    du = host(gg.rhs(dev(u, dtype), p=p))
    du_o, p_o = poisson.rhs(og, u)
    assert rel(du, du_o) <= TOL[dtype], rel(du, du_o)
    pd = demean(og, host(p))
    po = demean(og, p_o)
    assert rel(pd, po) <= 5 * TOL[dtype], rel(pd, po)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", CASES)
def test_project_parity(name, dtype):
    og, gg = grids(name, dtype)
    u = rounded(rand_u(og, 2), dtype)
    ut = dev(u, dtype)
    out = host(gg.project(ut))
    ref, _ = poisson.project(og, u)
    assert rel(out, ref) <= TOL[dtype], rel(out, ref)
    # divergence of the projected field at round-off: relative to the input divergence,
    # with room for the conditioning of L (the oracle's own projection reaches ~30 eps)
    eps = np.finfo(np.float64 if dtype == torch.float64 else np.float32).eps
    assert np.max(np.abs(op.divergence(og, out))) < 1000 * eps * np.max(np.abs(op.divergence(og, u)))
    # in place
    gg.project(ut, out=ut)
    assert rel(host(ut), ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", CASES)
def test_divergence_parity(name, dtype):
    og, gg = grids(name, dtype)
    u = rounded(rand_u(og, 3), dtype)
    d = host(gg.divergence(dev(u, dtype)))
    assert rel(d, op.divergence(og, u)) <= TOL[dtype]


# ------------------------------------------------------------------ RK4 step
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", CASES)
def test_step_parity(name, dtype):
    og, gg = grids(name, dtype)
    u0 = rand_u(og, 4, project=True)
    u0 = rounded(u0, dtype)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ut = dev(u0, dtype)
    gg.step(ut, dt=dt)
    ref = timestep.rk4_step(og, u0, dt)
    assert rel(host(ut), ref) <= TOL[dtype], rel(host(ut), ref)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", ["p3", "c3"])
def test_step_device_dt_and_cfl_bitexact(name, dtype):
    og, gg = grids(name, dtype)
    u0 = rounded(rand_u(og, 5, project=True), dtype)
    ut = dev(u0, dtype)
    dt_dev = gg.cfl_dt(ut, 0.3)
    assert dt_dev.item() == timestep.cfl_dt(og, u0, 0.3)          # bit for bit
    dt0 = dt_dev.item()
    gg.step(ut, dt_dev=dt_dev, next_dt_dev=dt_dev, cfl=0.3)     # adaptive, all on the device
    u1 = host(ut)
    assert rel(u1, timestep.rk4_step(og, u0, dt0)) <= TOL[dtype]
    assert dt_dev.item() == timestep.cfl_dt(og, u1, 0.3)          # next dt from u_{n+1}, bit for bit


def test_taylor_green_100_steps_fp64():
    """Config: 2-D TGV 64^2 FP64, dt = 0.01, 100 steps: <= 1e-10 against the oracle."""
    n, nu, dt = 64, 0.01, 0.01
    faces = inputs.periodic_box(n, 2)
    og = OGrid(faces, ["periodic"] * 2, nu)
    gg = Grid(faces, ["periodic"] * 2, nu, dtype=torch.float64)
    u0 = inputs.taylor_green_2d(faces)
    ut = dev(u0, torch.float64)
    for _ in range(100):
        gg.step(ut, dt=dt)
    ref = timestep.integrate(og, u0, dt, 100)
    assert rel(host(ut), ref) <= 1e-10
    exact = inputs.taylor_green_2d(faces, t=1.0, nu=nu)
    assert rel(host(ut), exact) < 2e-3       # O(D^2) spatial error


def test_random_3d_100_steps_fp64():
    og, gg = grids("p3tiny", torch.float64)
    u0 = rand_u(og, 6, project=True)
    dt = 0.3 * timestep.cfl_dt(og, u0, 0.3)
    ut = dev(u0, torch.float64)
    for _ in range(100):
        gg.step(ut, dt=dt)
    ref = timestep.integrate(og, u0, dt, 100)
    assert rel(host(ut), ref) <= 1e-10


# ------------------------------------------------------------------ diagnostics, failure paths
@pytest.mark.parametrize("name", ["p3", "c3"])
def test_diag(name):
    og, gg = grids(name, torch.float64)
    u = rand_u(og, 7)
    d = gg.diag(dev(u, torch.float64))
    assert abs(d["ke"] - diagnostics.kinetic_energy(og, u)) <= 1e-12 * diagnostics.kinetic_energy(og, u)
    assert abs(d["max_div"] - np.max(np.abs(op.divergence(og, u)))) <= 1e-12 * d["max_div"]
    assert d["max_u_over_h"] == timestep.max_u_over_h(og, u)
    assert d["nonfinite"] == 0


def test_nonfinite_input_is_reported():
    """Host-side fault injection: a NaN in the input sets the device error flag."""
    og, gg = grids("p3tiny", torch.float64)
    u = rand_u(og, 8, project=True)
    u[0, 1, 2, 3] = np.nan
    ut = dev(u, torch.float64)
    gg.step(ut, dt=1e-3)
    with pytest.raises(InsError) as e:
        gg.check_finite()
    assert e.value.status == INS_ERR_NONFINITE
    gg.check_finite()          # the flag was cleared
    with pytest.raises(InsError):
        gg.diag(ut)


def test_step_is_deterministic():
    og, gg = grids("p3", torch.float64)
    u0 = rand_u(og, 10, project=True)
    a = dev(u0, torch.float64)
    b = dev(u0, torch.float64)
    for t in (a, b):
        gg.step(t, dt=1e-2)
    assert torch.equal(a, b)


def test_bad_tensor_arguments():
    og, gg = grids("p3tiny", torch.float64)
    with pytest.raises(ValueError):
        gg.rhs(torch.zeros((3, 4, 4, 4), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        gg.rhs(gg.new_velocity().float())


# ------------------------------------------------------------------ FP32 stage-boundary fusion
@pytest.mark.parametrize("name", ["p3", "p3reg", "p3reg2", "c3", "c3reg"])
def test_fp32_unfused_step_parity(name):
    """The unfused FP32 kernels (ins_set_step_fusion(0)) against the oracle, like the fused default."""
    og, gg = grids(name, torch.float32)
    gg.set_step_fusion(False)
    u0 = rounded(rand_u(og, 4, project=True), torch.float32)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ut = dev(u0, torch.float32)
    gg.step(ut, dt=dt)
    assert rel(host(ut), timestep.rk4_step(og, u0, dt)) <= TOL[torch.float32]


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("name", ["p3reg2", "c3"])
def test_fp32_fused_matches_unfused(name, level):
    """Fused and unfused stage boundaries differ only by FP32 rounding order (10 steps)."""
    og, gg = grids(name, torch.float32)
    u0 = rounded(rand_u(og, 21, project=True), torch.float32)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    a = dev(u0, torch.float32)
    b = dev(u0, torch.float32)
    for _ in range(10):
        gg.set_step_fusion(level)
        gg.step(a, dt=dt)
        gg.set_step_fusion(False)
        gg.step(b, dt=dt)
    assert rel(host(a), host(b)) <= 1e-6


@pytest.mark.parametrize("name", ["p3", "p3reg", "p3reg2", "c3", "c3reg", "cu3"])
def test_fp32_pair_and_single_cell_fusion_agree(name):
    """Two cells per thread (level 2) and one cell per thread (level 1) run the same arithmetic
    per cell: one step agrees bit for bit, and both match the oracle."""
    og, gg = grids(name, torch.float32)
    u0 = rounded(rand_u(og, 22, project=True), torch.float32)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    out = {}
    for level in (1, 2):
        gg.set_step_fusion(level)
        ut = dev(u0, torch.float32)
        gg.step(ut, dt=dt)
        out[level] = ut
    assert torch.equal(out[1], out[2])
    assert rel(host(out[2]), timestep.rk4_step(og, u0, dt)) <= TOL[torch.float32]


@pytest.mark.parametrize("shape", [(4, 3, 2), (60, 9, 5), (72, 9, 5)])
@pytest.mark.parametrize("bc", ["periodic", "wall"])
def test_pair_kernels_on_small_and_ragged_grids(shape, bc):
    """The two-cells-per-thread kernels on grids narrower than one 64-wide tile, with a ragged
    second tile, ragged rows and few planes: bit-identical to the one-cell kernels, and the
    oracle's step within the FP32 tolerance."""
    nx, ny, nz = shape
    U = inputs.uniform_faces
    if bc == "wall":
        faces, bcs, force = [U(nx, 0, 4 * PI), inputs.tanh_faces(ny, 0, 2, 1.5), U(nz, 0, 2.0)], \
            ["periodic", "wall", "periodic"], [1.0, 0.0, 0.0]
    else:
        faces, bcs, force = [U(nx, 0, 2 * PI), U(ny, 0, 1.5), U(nz, 0, 1.0)], ["periodic"] * 3, None
    og = OGrid(faces, bcs, 0.02, force)
    gg = Grid(faces, bcs, 0.02, force, dtype=torch.float32)
    u0 = rounded(rand_u(og, 31, project=True), torch.float32)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    out = {}
    for level in (1, 2):
        gg.set_step_fusion(level)
        ut = dev(u0, torch.float32)
        gg.step(ut, dt=dt)
        out[level] = ut
    assert torch.equal(out[1], out[2])
    assert rel(host(out[2]), timestep.rk4_step(og, u0, dt)) <= TOL[torch.float32]


def test_fusion_level_is_checked():
    from paper_2604_18536_b300._lib import InsError
    _, gg = grids("p3", torch.float32)
    with pytest.raises(InsError):
        gg.set_step_fusion(3)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", ["cu3", "cu2"])
def test_dct_and_thomas_wall_solves_agree(name, dtype):
    """On a uniform wall-normal grid both y solves give the same step (velocities)."""
    og, gg = grids(name, dtype)
    u0 = rounded(rand_u(og, 41, project=True), dtype)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    a = dev(u0, dtype)
    b = dev(u0, dtype)
    gg.set_wall_solver("dct")
    gg.step(a, dt=dt)
    gg.set_wall_solver("thomas")
    gg.step(b, dt=dt)
    assert rel(host(a), host(b)) <= (1e-13 if dtype == torch.float64 else 1e-6)
    with pytest.raises(InsError):
        grids("c3", dtype)[1].set_wall_solver("dct")     # stretched y: no DCT


@pytest.mark.parametrize("name", ["p3", "c3"])
def test_march_chunk_is_launch_shape_only(name):
    """The z chunk of the pair kernels (ins_set_march_chunk) changes no bit of the step, including
    chunks that split z raggedly and chunks longer than nz; negative chunks are rejected."""
    from paper_2604_18536_b300._lib import InsError
    og, gg = grids(name, torch.float32)
    u0 = rounded(rand_u(og, 23, project=True), torch.float32)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    out = []
    for kc in (0, 1, 5, 64):
        gg.set_march_chunk(kc)
        ut = dev(u0, torch.float32)
        gg.step(ut, dt=dt)
        out.append(ut)
    assert all(torch.equal(out[0], o) for o in out[1:])
    with pytest.raises(InsError):
        gg.set_march_chunk(-1)


# ------------------------------------------------------------------ square x-y planes, thin z
# FP32 periodic 3-D grids with square x-y planes of the register FFT lengths 64, 128 and 256 and a
# few odd z planes (the z pass on a ragged length with the Stockham kernel).
@pytest.mark.parametrize("nxy,nz", [(64, 9), (128, 5), (256, 3)])
def test_fp32_square_plane_projection_and_step(nxy, nz):
    U = inputs.uniform_faces
    faces = [U(nxy, 0, 2 * PI), U(nxy, 0, 1.5 * PI), U(nz, 0, 0.5)]
    og = OGrid(faces, ["periodic"] * 3, 0.02)
    gg = Grid(faces, ["periodic"] * 3, 0.02, dtype=torch.float32)
    u = rounded(rand_u(og, 21), torch.float32)
    out = host(gg.project(dev(u, torch.float32)))
    ref, _ = poisson.project(og, u)
    assert rel(out, ref) <= 2e-5, rel(out, ref)
    u0 = rounded(rand_u(og, 22, project=True), torch.float32)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ut = dev(u0, torch.float32)
    gg.step(ut, dt=dt)
    assert rel(host(ut), timestep.rk4_step(og, u0, dt)) <= 2e-5
    gg.close()
