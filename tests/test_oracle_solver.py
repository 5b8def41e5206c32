"""Pins of the oracle's Poisson solvers, RK4 step, CFL rule, adjoints and diagnostics."""

import numpy as np
import pytest

from oracle import operators as op, poisson, timestep, adjoint, diagnostics
from oracle.grid import Grid, uniform_faces, tanh_faces
from paper_2604_18536_b300 import inputs
from test_oracle_operators import (periodic_grid, stretched_periodic_grid, channel_grid, random_u,
                                   dense_matrix)


# ------------------------------------------------------------------ Poisson
@pytest.mark.parametrize("kind", ["periodic2", "periodic3", "channel2", "channel3"])
def test_poisson_matches_dense_solve(kind):
    """Brute force: p equals the dense solve of the assembled L = D G (mean removed)."""
    if kind == "periodic2":
        g = periodic_grid(6, 2)
    elif kind == "periodic3":
        g = periodic_grid(4, 3)
    elif kind == "channel2":
        g = Grid([uniform_faces(6, 0, 3.0), tanh_faces(5, 0, 2, 1.5)], ["periodic", "wall"], 0.1)
    else:
        g = channel_grid(6, 4, 6)
    npts = int(np.prod(g.shape))
    L = dense_matrix(g, lambda e: poisson.laplacian(g, e.reshape(g.shape)), npts, npts)
    # a consistent right-hand side: the divergence of a random field with zero wall flux
    r = op.divergence(g, random_u(g, 7))
    p = poisson.solve(g, r)
    # augmented system (Sec. 2.6.1, direct solver): [L e; e^T 0][p; l] = [r; 0]
    vol = g.cell_volume().ravel()
    A = np.zeros((npts + 1, npts + 1))
    A[:npts, :npts] = L
    A[:npts, npts] = vol
    A[npts, :npts] = vol
    rhs = np.concatenate([r.ravel(), [0.0]])
    pd = np.linalg.solve(A, rhs)[:npts].reshape(g.shape)
    pm = p - np.sum(vol.reshape(g.shape) * p) / vol.sum()
    np.testing.assert_allclose(pm, pd, atol=1e-11 * np.max(np.abs(pd)))


@pytest.mark.parametrize("kind", ["periodic3", "channel"])
def test_projection_properties(kind):
    """max|D P u| at round-off, P idempotent, Poisson residual at round-off (Sec. 5.8)."""
    g = periodic_grid(12, 3) if kind == "periodic3" else channel_grid(8, 12, 6)
    u = random_u(g, 9)
    Pu, p = poisson.project(g, u)
    umax = np.max(np.abs(u))
    dmin = min(np.min(g.d[a]) for a in range(g.dim))
    assert np.max(np.abs(op.divergence(g, Pu))) < 200 * np.finfo(float).eps * umax / dmin
    PPu, _ = poisson.project(g, Pu)
    np.testing.assert_allclose(PPu, Pu, atol=1e-13 * umax)
    r = op.divergence(g, u)
    res = poisson.laplacian(g, p) - r
    assert np.linalg.norm(res) < 1e-12 * np.linalg.norm(r)


# ---------------------------------------------------------- time stepping
@pytest.mark.parametrize("dim", [2, 3])
def test_shear_wave_rk4_amplification(dim):
    """u^x = sin(m y): convection vanishes, the projection is the identity and one RK4
    step multiplies the field by R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24,
    z = -dt nu (4/D^2) sin^2(m D/2)."""
    n, m, nu, dt = 16, 3, 0.2, 0.01
    g = periodic_grid(n, dim, nu=nu)
    D = 2 * np.pi / n
    u = g.zeros_u()
    y = g.face_coords(0)[1]
    u[0] = np.sin(m * y) * np.ones(g.shape)
    z = -dt * nu * (4 / D ** 2) * np.sin(m * D / 2) ** 2
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    u1 = timestep.rk4_step(g, u, dt)
    np.testing.assert_allclose(u1[0], R * u[0], atol=1e-14)
    np.testing.assert_allclose(u1[1:], 0.0, atol=1e-14)


def poiseuille_discrete(g):
    """Discrete steady channel flow nu (diffusion_y u)(y) = -f: a 1-D dense solve of the
    operator's own y-stencil, which the full RK4 step must leave unchanged."""
    ny = g.n[1]

    def apply(col):
        u = g.zeros_u()
        u[0] = col.reshape(1, ny, 1) * np.ones(g.shape)
        return op.diffusion(g, u)[0][0, :, 0]

    A = dense_matrix(g, apply, ny, ny)
    return np.linalg.solve(g.nu * A, -g.force[0] * np.ones(ny))


def test_poiseuille_is_steady_on_tanh_grid():
    g = channel_grid(4, 16, 4)
    ux = poiseuille_discrete(g)
    u = g.zeros_u()
    u[0] = ux.reshape(1, -1, 1) * np.ones(g.shape)
    u1 = timestep.rk4_step(g, u, 1e-3)
    np.testing.assert_allclose(u1, u, atol=1e-12 * np.max(np.abs(ux)))


def test_poiseuille_converges_to_parabola_second_order():
    """The discrete steady state approaches u = y(2-y)/(2 nu) at second order in 1/N."""
    errs = []
    for ny in (16, 32, 64):
        g = channel_grid(4, ny, 4)
        ux = poiseuille_discrete(g)
        yc = g.xc[1]
        exact = yc * (2 - yc) / (2 * g.nu)
        errs.append(np.max(np.abs(ux - exact)) / np.max(exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


def taylor_green_error(n, t_end=1.0, dt=0.01, nu=0.01):
    g = periodic_grid(n, 2, nu=nu)
    faces = g.faces
    u = inputs.taylor_green_2d(faces)
    steps = int(round(t_end / dt))
    u = timestep.integrate(g, u, dt, steps)
    ex = inputs.taylor_green_2d(faces, t=t_end, nu=nu)
    return np.sqrt(np.mean((u - ex) ** 2)), u, g


def test_taylor_green_second_order():
    """2-D Taylor-Green vortex at t = 1 (Sec. 7.4): second-order spatial convergence."""
    errs = [taylor_green_error(n)[0] for n in (8, 16, 32)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9) and np.all(rates < 2.2), (errs, rates)


def test_taylor_green_energy_decay():
    """KE(t)/KE(0) = exp(-4 nu t) up to the O(D^2) discretisation error."""
    err, u, g = taylor_green_error(32)
    u0 = inputs.taylor_green_2d(g.faces)
    ratio = diagnostics.kinetic_energy(g, u) / diagnostics.kinetic_energy(g, u0)
    assert abs(ratio - np.exp(-4 * 0.01)) < 5e-3 * (2 * np.pi / 32) ** 2 * 10


def test_cfl_rule():
    g = channel_grid(6, 8, 4, nu=0.5)
    u = random_u(g, 2)
    dt = timestep.cfl_dt(g, u, 0.3)
    m = 0.0
    for a in range(g.dim):
        for idx in np.ndindex(g.shape):
            i = idx[g.axis(a)]
            m = max(m, abs(u[a][idx]) / g.h[a][i])
    dmin = min(np.min(g.d[a]) for a in range(g.dim))
    assert dt == 0.3 * min(1.0 / m, dmin * dmin / 0.5)


def test_rk4_order_in_time():
    """Temporal order 4: halving dt cuts the one-interval error by ~16."""
    g = periodic_grid(8, 2, nu=0.05)
    u0, _ = poisson.project(g, random_u(g, 12))
    ref = timestep.integrate(g, u0, 0.2 / 64, 64)
    e1 = np.max(np.abs(timestep.integrate(g, u0, 0.2 / 4, 4) - ref))
    e2 = np.max(np.abs(timestep.integrate(g, u0, 0.2 / 8, 8) - ref))
    assert 12 < e1 / e2 < 20


@pytest.mark.parametrize("dim", [2, 3])
def test_shear_wave_wray3_amplification(dim):
    """Every three-stage third-order explicit RK has the stability function
    R(z) = 1 + z + z^2/2 + z^3/6: on the shear wave (no convection, identity projection)
    one Wray step multiplies the field by it."""
    n, m, nu, dt = 16, 3, 0.2, 0.01
    g = periodic_grid(n, dim, nu=nu)
    D = 2 * np.pi / n
    u = g.zeros_u()
    y = g.face_coords(0)[1]
    u[0] = np.sin(m * y) * np.ones(g.shape)
    z = -dt * nu * (4 / D ** 2) * np.sin(m * D / 2) ** 2
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6
    u1 = timestep.wray3_step(g, u, dt)
    np.testing.assert_allclose(u1[0], R * u[0], atol=1e-14)
    np.testing.assert_allclose(u1[1:], 0.0, atol=1e-14)


def test_wray3_order_in_time():
    """Temporal order 3 on a nonlinear (convective) flow: halving dt cuts the error by ~8.
    A wrong tableau entry (for example a32 = 1/2) drops the order and fails the ratio."""
    g = periodic_grid(8, 2, nu=0.05)
    u0, _ = poisson.project(g, random_u(g, 12))
    ref = timestep.integrate(g, u0, 0.2 / 64, 64)        # RK4, error far below the Wray errors
    e1 = np.max(np.abs(timestep.integrate(g, u0, 0.2 / 4, 4, scheme="wray3") - ref))
    e2 = np.max(np.abs(timestep.integrate(g, u0, 0.2 / 8, 8, scheme="wray3") - ref))
    assert 6.5 < e1 / e2 < 9.5


def test_wray3_tableau_low_storage_form():
    """The tableau equals the two-register recurrence u_{s+1} = u_s + dt (g_s k_s + z_s k_{s-1})
    with g = (8/15, 5/12, 3/4), z = (0, -17/60, -5/12): a_{s+1,t} = a_{s,t} for t < s - 1,
    a_{s+1,s-1} = a_{s,s-1} + z_s, a_{s+1,s} = g_s (b as the fourth row)."""
    from fractions import Fraction as Fr
    gam = (Fr(8, 15), Fr(5, 12), Fr(3, 4))
    zet = (Fr(0), Fr(-17, 60), Fr(-5, 12))
    rows = [[]]
    for s in range(3):
        prev = rows[-1] + [Fr(0)]
        new = list(prev)
        new[s] = gam[s]
        if s > 0:
            new[s - 1] = prev[s - 1] + zet[s]
        rows.append(new)
    A = [[Fr(x).limit_denominator(1000) for x in r] for r in timestep.WRAY3_A]
    assert rows[1][:1] == A[1] and rows[2][:2] == A[2]
    assert rows[3] == [Fr(x).limit_denominator(1000) for x in timestep.WRAY3_B]
    # third-order conditions
    b = rows[3]
    c = [Fr(0), sum(A[1]), sum(A[2])]
    assert sum(b) == 1 and sum(bi * ci for bi, ci in zip(b, c)) == Fr(1, 2)
    assert sum(bi * ci * ci for bi, ci in zip(b, c)) == Fr(1, 3)
    assert b[2] * A[2][1] * c[1] == Fr(1, 6)


# ------------------------------------------------------------------ adjoints
def _dot(a, b):
    return float(np.sum(a * b))


@pytest.mark.parametrize("stretched", [False, True])
def test_linear_adjoints_dot_product(stretched):
    """<J v, w> = <v, J^T w> for D, G and the diffusion (App. B pullbacks)."""
    g = stretched_periodic_grid(7, 3) if stretched else periodic_grid(6, 3)
    v = random_u(g, 1)
    w = random_u(g, 2)
    q = inputs.random_field(g.shape, 3)
    assert abs(_dot(op.divergence(g, v), q) - _dot(v, adjoint.divergence_T(g, q))) < 1e-12
    assert abs(_dot(op.gradient(g, q), w) - _dot(q, adjoint.gradient_T(g, w))) < 1e-12
    s = max(1.0, abs(_dot(op.diffusion(g, v), w)))
    assert abs(_dot(op.diffusion(g, v), w) - _dot(v, adjoint.diffusion_T(g, w))) < 1e-12 * s


@pytest.mark.parametrize("stretched", [False, True])
def test_convection_adjoint_dot_product(stretched):
    """Bilinear form: <B(v, t), w> = <v, B_adv^T w> = <t, B_tra^T w>; J v = B(v,u) + B(u,v)."""
    g = stretched_periodic_grid(6, 3) if stretched else periodic_grid(5, 3)
    u = random_u(g, 4)
    v = random_u(g, 5)
    w = random_u(g, 6)
    ab, tb = adjoint.convection_bilinear_T(g, v, u, w)
    ref1 = _dot(op.convection_bilinear(g, v, u), w)
    ab2, _ = adjoint.convection_bilinear_T(g, u, u, w)
    # linear in the advecting argument: <B(v,u), w> = <v, d/dadv <w,B(adv,u)>>
    assert abs(_dot(op.convection_bilinear(g, v, u), w) - _dot(v, ab2)) < 1e-11 * max(1, abs(ref1))
    _, tb2 = adjoint.convection_bilinear_T(g, u, u, w)
    assert abs(_dot(op.convection_bilinear(g, u, v), w) - _dot(v, tb2)) < 1e-11 * max(1, abs(ref1))
    Jv = op.convection_bilinear(g, v, u) + op.convection_bilinear(g, u, v)
    assert abs(_dot(Jv, w) - _dot(v, adjoint.convection_vjp(g, u, w))) < 1e-11 * max(1, abs(_dot(Jv, w)))


def test_step_vjp_dot_product_and_fd():
    """RK4 step VJP against central finite differences (eps = 1e-6) in u0 and nu (Sec. 3.4)."""
    g = periodic_grid(6, 3, nu=0.05)
    u0, _ = poisson.project(g, random_u(g, 21))
    dt = 0.05
    c = random_u(g, 22)

    def loss(u, nu):
        gg = periodic_grid(6, 3, nu=nu)
        return _dot(c, timestep.rk4_step(gg, u, dt))

    ubar, nubar = adjoint.rk4_step_vjp(g, u0, dt, c)
    eps = 1e-6
    for seed in range(3):
        du = random_u(g, 100 + seed)
        fd = (loss(u0 + eps * du, g.nu) - loss(u0 - eps * du, g.nu)) / (2 * eps)
        assert abs(fd - _dot(ubar, du)) < 1e-7 * max(1, abs(fd))
    fdn = (loss(u0, g.nu + eps) - loss(u0, g.nu - eps)) / (2 * eps)
    assert abs(fdn - nubar) < 1e-6 * max(1, abs(fdn))


def test_erk_vjp_reduces_to_rk4_vjp():
    """The generic Butcher-form pullback with the RK4 tableau is the RK4 step pullback."""
    g = periodic_grid(6, 3, nu=0.05)
    u0, _ = poisson.project(g, random_u(g, 31))
    c = random_u(g, 32)
    A = ((), (0.5,), (0.0, 0.5), (0.0, 0.0, 1.0))
    ub1, nb1 = adjoint.erk_step_vjp(g, u0, 0.05, c, A, timestep.RK4_B)
    ub2, nb2 = adjoint.rk4_step_vjp(g, u0, 0.05, c)
    np.testing.assert_allclose(ub1, ub2, rtol=0, atol=1e-13 * np.max(np.abs(ub2)))
    assert abs(nb1 - nb2) <= 1e-12 * abs(nb2)


def test_wray3_step_vjp_fd():
    """Wray step VJP against central finite differences (eps = 1e-6) in u0 and nu."""
    g = periodic_grid(6, 3, nu=0.05)
    u0, _ = poisson.project(g, random_u(g, 41))
    dt = 0.05
    c = random_u(g, 42)

    def loss(u, nu):
        return _dot(c, timestep.wray3_step(periodic_grid(6, 3, nu=nu), u, dt))

    ubar, nubar = adjoint.wray3_step_vjp(g, u0, dt, c)
    eps = 1e-6
    for seed in range(3):
        du = random_u(g, 140 + seed)
        fd = (loss(u0 + eps * du, g.nu) - loss(u0 - eps * du, g.nu)) / (2 * eps)
        assert abs(fd - _dot(ubar, du)) < 1e-7 * max(1, abs(fd))
    fdn = (loss(u0, g.nu + eps) - loss(u0, g.nu - eps)) / (2 * eps)
    assert abs(fdn - nubar) < 1e-6 * max(1, abs(fdn))


# ------------------------------------------------------------------ diagnostics
def test_filter_keeps_divergence_free():
    """Face averaging maps a divergence-free fine field to a divergence-free coarse one."""
    gf = periodic_grid(16, 3)
    gc = periodic_grid(4, 3)
    u, _ = poisson.project(gf, random_u(gf, 31))
    uc = diagnostics.face_average_filter(u, 3, 4)
    assert np.max(np.abs(op.divergence(gc, uc))) < 1e-12 * np.max(np.abs(u)) * 16


def test_spectrum_of_single_mode():
    """A single Fourier mode cos(3x) in u^y: E(3) = 1/4 * 1/2 * 2 ... = its energy, rest 0."""
    N = 16
    x = (np.arange(N) + 0.5) * 2 * np.pi / N
    u = np.zeros((3, N, N, N))
    u[1] = np.cos(3 * x)[None, None, :]
    E = diagnostics.shell_spectrum(u)
    # mean of 1/2 cos^2 = 1/4, carried by the two wavevectors (+-3, 0, 0)
    assert abs(E[3] - 0.25) < 1e-14 and abs(E.sum() - 0.25) < 1e-14


def test_kinetic_energy_uniform_is_mean_square():
    g = periodic_grid(8, 3)
    u = random_u(g, 5)
    assert abs(diagnostics.kinetic_energy(g, u) - 0.5 * np.sum(np.mean(u ** 2, axis=(1, 2, 3)))) < 1e-14
