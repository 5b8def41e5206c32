"""Pins of the oracle's operators against closed forms and exact identities.

Each test fixes a property the paper or the mathematics states, chosen so a
plausible slip (a dropped term, a wrong sign or index, a transposed operand,
wrong interpolation weights) fails at least one of them.
"""

import numpy as np
import pytest

import oracle
from oracle import operators as op, poisson
from oracle.grid import Grid, uniform_faces, tanh_faces
from paper_2604_18536_b300 import inputs


def periodic_grid(n, dim, nu=0.01, length=2 * np.pi):
    return Grid([uniform_faces(n, 0.0, length)] * dim, ["periodic"] * dim, nu)


def stretched_periodic_grid(n, dim, nu=0.01, seed=3):
    """Periodic directions with random (smooth-ish) non-uniform spacing."""
    rng = np.random.default_rng(seed)
    faces = []
    for _ in range(dim):
        w = 1.0 + 0.6 * rng.random(n)
        f = np.concatenate([[0.0], np.cumsum(w)])
        faces.append(f * (2 * np.pi / f[-1]))
    return Grid(faces, ["periodic"] * dim, nu)


def channel_grid(nx, ny, nz, nu=1.0 / 180, gamma=1.5):
    faces = [uniform_faces(nx, 0, 4 * np.pi), tanh_faces(ny, 0, 2, gamma), uniform_faces(nz, 0, 4 * np.pi / 3)]
    return Grid(faces, ["periodic", "wall", "periodic"], nu, force=[1.0, 0.0, 0.0])


def random_u(g, seed):
    u = inputs.random_field((g.dim,) + g.shape, seed)
    for a in range(g.dim):
        u[a] *= g.face_mask(a)
    return u


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("m", [1, 3, 7])
def test_diffusion_symbol(dim, m):
    """Diffusion of sin(m x) is -(4/D^2) sin^2(m D/2) sin(m x) exactly, in every direction."""
    n = 24
    g = periodic_grid(n, dim)
    D = 2 * np.pi / n
    lam = -(4.0 / D ** 2) * np.sin(m * D / 2) ** 2
    for a in range(dim):
        for b in range(dim):
            u = g.zeros_u()
            pos = g.face_coords(a)[b]
            u[a] = np.sin(m * pos) * np.ones(g.shape)
            out = op.diffusion(g, u)
            np.testing.assert_allclose(out[a], lam * u[a], atol=1e-12 * abs(lam))
            for c in range(dim):
                if c != a:
                    assert np.max(np.abs(out[c])) == 0.0


@pytest.mark.parametrize("m", [1, 2, 5])
def test_convection_cross_term_closed_form(m):
    """u^x = c, u^y = sin(m x): C^y = -c cos(m x) sin(m D)/D exactly, C^x = 0."""
    n, c = 20, 0.7
    g = periodic_grid(n, 2)
    D = 2 * np.pi / n
    u = g.zeros_u()
    u[0] = c
    x = g.face_coords(1)[0]
    u[1] = np.sin(m * x) * np.ones(g.shape)
    C = op.convection(g, u)
    expect = -c * np.cos(m * x) * np.sin(m * D) / D * np.ones(g.shape)
    np.testing.assert_allclose(C[1], expect, atol=1e-13)
    np.testing.assert_allclose(C[0], 0.0, atol=1e-13)


@pytest.mark.parametrize("m", [1, 3])
def test_convection_self_term_closed_form(m):
    """u^x = sin(m x_f), u^y = 0: C^x = -cos^2(mD/2) sin(2 m x_f) sin(m D)/D."""
    n = 16
    g = periodic_grid(n, 2)
    D = 2 * np.pi / n
    u = g.zeros_u()
    xf = g.face_coords(0)[0]
    u[0] = np.sin(m * xf) * np.ones(g.shape)
    C = op.convection(g, u)
    expect = -np.cos(m * D / 2) ** 2 * np.sin(2 * m * xf) * np.sin(m * D) / D * np.ones(g.shape)
    np.testing.assert_allclose(C[0], expect, atol=1e-13)
    np.testing.assert_allclose(C[1], 0.0, atol=1e-13)


def test_convection_3d_cross_terms_closed_form():
    """3-D: u^x = c, u^z = sin(m x), u^y = b: C^z = -c cos(m x) sin(mD)/D (y-flux carries a constant)."""
    n, c, bconst, m = 12, 0.4, -0.9, 2
    g = periodic_grid(n, 3)
    D = 2 * np.pi / n
    u = g.zeros_u()
    u[0] = c
    u[1] = bconst
    x = g.face_coords(2)[0]
    u[2] = np.sin(m * x) * np.ones(g.shape)
    C = op.convection(g, u)
    np.testing.assert_allclose(C[2], -c * np.cos(m * x) * np.sin(m * D) / D * np.ones(g.shape), atol=1e-13)
    np.testing.assert_allclose(C[0], 0.0, atol=1e-13)
    np.testing.assert_allclose(C[1], 0.0, atol=1e-13)


# --------------------------------------------------- conservation, duality
def _ke_rate(g, u):
    C = op.convection(g, u)
    num = sum(np.sum(g.face_volume(a) * u[a] * C[a]) for a in range(g.dim))
    scale = sum(np.sum(g.face_volume(a) * np.abs(u[a] * C[a])) for a in range(g.dim))
    return num, scale


@pytest.mark.parametrize("kind", ["uniform2", "uniform3", "stretched3", "channel"])
def test_convection_conserves_energy(kind):
    """sum_a sum_I |Omega^a_I| u^a_I C^a(u)_I = 0 for divergence-free u (Sec. 5.8, App. A)."""
    if kind == "uniform2":
        g = periodic_grid(16, 2)
    elif kind == "uniform3":
        g = periodic_grid(10, 3)
    elif kind == "stretched3":
        g = stretched_periodic_grid(8, 3)
    else:
        g = channel_grid(8, 10, 6)
    u = random_u(g, 11)
    if kind == "stretched3":
        # the spectral solver needs uniform spacing: make u divergence free with a dense solve
        u = dense_project(g, u)
    else:
        u, _ = poisson.project(g, u)
    assert np.max(np.abs(op.divergence(g, u))) < 1e-11
    num, scale = _ke_rate(g, u)
    assert abs(num) < 1e-13 * scale


def test_energy_pin_rejects_linear_interpolation(monkeypatch):
    """Planted mistake: the literal linear-interpolation weights break exact energy
    conservation on a stretched grid, so the energy pin really tests the weights."""
    g = channel_grid(6, 12, 4)
    u = random_u(g, 5)
    u, _ = poisson.project(g, u)
    num, scale = _ke_rate(g, u)
    assert abs(num) < 1e-13 * scale

    def linear(g_, a):
        d = g_.d[a]
        dn = op.d_next(g_, a)
        return dn / (d + dn), d / (d + dn)     # weight on the left value ~ the other cell's width

    monkeypatch.setattr(op, "interp_weights", linear)
    num, scale = _ke_rate(g, u)
    assert abs(num) > 1e-6 * scale


@pytest.mark.parametrize("kind", ["uniform3", "stretched2", "channel"])
def test_divergence_gradient_duality(kind):
    """sum_I |Omega_I| (D u)_I p_I = - sum_a sum_I |Omega^a_I| u^a_I (G p)^a_I (Sec. 2.3)."""
    if kind == "uniform3":
        g = periodic_grid(6, 3)
    elif kind == "stretched2":
        g = stretched_periodic_grid(9, 2)
    else:
        g = channel_grid(6, 7, 5)
    u = random_u(g, 1)
    p = inputs.random_field(g.shape, 2)
    lhs = np.sum(g.cell_volume() * op.divergence(g, u) * p)
    Gp = op.gradient(g, p)
    rhs = -sum(np.sum(g.face_volume(a) * u[a] * Gp[a]) for a in range(g.dim))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1.0)


def test_translation_equivariance_bitexact():
    """Shifting the input by whole cells shifts F(u) by the same cells, bit for bit."""
    g = periodic_grid(8, 3, nu=0.05)
    u = random_u(g, 4)
    F = op.rhs_F(g, u)
    for ax, s in [(0, 1), (1, 3), (2, -2)]:
        us = np.roll(u, s, axis=ax + 1)
        Fs = op.rhs_F(g, us)
        assert np.array_equal(Fs, np.roll(F, s, axis=ax + 1))


def test_axis_permutation_equivariance():
    """Swapping x and y (positions and components) commutes with F on a cubic grid."""
    g = periodic_grid(6, 3, nu=0.03)
    u = random_u(g, 8)
    F = op.rhs_F(g, u)
    # numpy axes (z, y, x): swap the y and x axes and the x, y components
    us = np.stack([np.swapaxes(u[1], 1, 2), np.swapaxes(u[0], 1, 2), np.swapaxes(u[2], 1, 2)])
    Fs = op.rhs_F(g, us)
    back = np.stack([np.swapaxes(Fs[1], 1, 2), np.swapaxes(Fs[0], 1, 2), np.swapaxes(Fs[2], 1, 2)])
    np.testing.assert_allclose(back, F, atol=1e-13)


def test_wall_faces_stay_zero():
    """F, G p and the projection never touch the stored top-wall u^y."""
    g = channel_grid(6, 8, 4)
    u = random_u(g, 3)
    F = op.rhs_F(g, u)
    assert np.all(F[1][:, -1, :] == 0.0)
    Pu, _ = poisson.project(g, u)
    assert np.all(Pu[1][:, -1, :] == 0.0)


# ------------------------------------------------------------ helpers
def dense_matrix(g, fn, nin, nout):
    M = np.zeros((nout, nin))
    for j in range(nin):
        e = np.zeros(nin)
        e[j] = 1.0
        M[:, j] = fn(e).ravel()
    return M


def dense_project(g, u):
    """Projection with a dense least-squares Poisson solve (brute force, tiny grids)."""
    npts = int(np.prod(g.shape))
    L = dense_matrix(g, lambda e: poisson.laplacian(g, e.reshape(g.shape)), npts, npts)
    r = op.divergence(g, u).ravel()
    p = np.linalg.lstsq(L, r, rcond=None)[0].reshape(g.shape)
    return u - op.gradient(g, p)
