"""Pins of the oracle's eddy-viscosity models (App. "Eddy-viscosity models").

Each pin is fixed by the mathematics, not by the oracle itself:
* a constant eddy viscosity c turns sum_b delta_b(2 c S_ab) into c (diffusion + G D), the
  already pinned diffusion and gradient-of-divergence operators (exact algebraic identity);
* every model formula against its closed form on pure shear, solid-body rotation,
  axisymmetric strain and two-component strain;
* summation by parts: sum_faces u . e = - sum 2 nu_t S:S over the staggered strain points;
* second-order convergence of the interpolated velocity gradient to the exact one.
"""

import numpy as np
import pytest

from oracle import eddy, operators as op
from oracle.grid import Grid, uniform_faces
from test_oracle_operators import periodic_grid, stretched_periodic_grid, random_u


@pytest.mark.parametrize("kind", ["uniform2", "uniform3", "stretched3"])
def test_constant_viscosity_is_diffusion_plus_grad_div(kind):
    g = {"uniform2": lambda: periodic_grid(10, 2), "uniform3": lambda: periodic_grid(6, 3),
         "stretched3": lambda: stretched_periodic_grid(7, 3)}[kind]()
    u = random_u(g, 3)
    c = 0.37
    e = eddy.stress_divergence(g, u, c * np.ones(g.shape))
    ref = c * (op.diffusion(g, u) + op.gradient(g, op.divergence(g, u)))
    np.testing.assert_allclose(e, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def _shear(s):
    A = np.zeros((3, 3))
    A[0, 1] = s            # du/dy = s
    return A


def test_smagorinsky_closed_forms():
    C, D = 0.1, 0.3
    # pure shear: sqrt(2 S:S) = |s|
    assert np.isclose(eddy.nu_t_pointwise(eddy.SMAGORINSKY, _shear(2.0), D, C), (C * D) ** 2 * 2.0, rtol=1e-14)
    # solid rotation: S = 0
    R = np.array([[0.0, -1.5, 0.0], [1.5, 0.0, 0.0], [0.0, 0.0, 0.0]])
    assert eddy.nu_t_pointwise(eddy.SMAGORINSKY, R, D, C) == 0.0
    # axisymmetric strain diag(-s, -s, 2s): 2 S:S = 12 s^2
    s = 0.7
    assert np.isclose(eddy.nu_t_pointwise(eddy.SMAGORINSKY, np.diag([-s, -s, 2 * s]), D, C),
                      (C * D) ** 2 * np.sqrt(12.0) * s, rtol=1e-14)


def test_wale_closed_forms():
    C, D = 0.5, 0.2
    # pure shear: A A = 0, so S^d = 0 and nu_t = 0 (WALE vanishes in pure shear)
    assert eddy.nu_t_pointwise(eddy.WALE, _shear(3.0), D, C) == 0.0
    # solid rotation w: S = 0, S^d = diag(-1, -1, 2) w^2 / 3, nu_t = (C D)^2 (2/3)^(1/4) |w|
    w = 1.3
    R = np.array([[0.0, -w, 0.0], [w, 0.0, 0.0], [0.0, 0.0, 0.0]])
    assert np.isclose(eddy.nu_t_pointwise(eddy.WALE, R, D, C), (C * D) ** 2 * (2.0 / 3.0) ** 0.25 * w, rtol=1e-13)
    # pure strain A = S = diag(s, -s, 0): S^d = diag(1, 1, -2) s^2 / 3, S^d:S^d = 2 s^4 / 3, S:S = 2 s^2
    s = 0.8
    sd, ss = 2.0 * s ** 4 / 3.0, 2.0 * s ** 2
    want = (C * D) ** 2 * sd ** 1.5 / (ss ** 2.5 + sd ** 1.25)
    assert np.isclose(eddy.nu_t_pointwise(eddy.WALE, np.diag([s, -s, 0.0]), D, C), want, rtol=1e-13)


def test_qr_closed_forms():
    C, D = np.sqrt(1.5) / np.pi, 0.25
    s = 0.9
    # axisymmetric strain diag(-s, -s, 2s): R_S = 2 s^3, Q_S = -3 s^2, nu_t = (C D)^2 (2/3) s
    assert np.isclose(eddy.nu_t_pointwise(eddy.QR, np.diag([-s, -s, 2 * s]), D, C), (C * D) ** 2 * 2.0 / 3.0 * s,
                      rtol=1e-13)
    # two-component strain: R_S = 0
    assert abs(eddy.nu_t_pointwise(eddy.QR, np.diag([s, -s, 0.0]), D, C)) < 1e-18
    # no strain at all
    assert eddy.nu_t_pointwise(eddy.QR, np.zeros((3, 3)), D, C) == 0.0


def test_vreman_closed_forms():
    C = np.sqrt(2.5 * 0.1 ** 2)
    w = [0.2, 0.2, 0.2]
    # pure shear du/dy = s: beta has a single nonzero entry, B_beta = 0
    assert eddy.nu_t_pointwise(eddy.VREMAN, _shear(2.0), 0.2, C, w) == 0.0
    # A = diag(s, -s, 0), equal widths D: B_beta = D^4 s^4, tr(A A^T)/2 = s^2: nu_t = C^2 D^2 |s|
    s = 1.1
    assert np.isclose(eddy.nu_t_pointwise(eddy.VREMAN, np.diag([s, -s, 0.0]), 0.2, C, w), C ** 2 * 0.04 * s,
                      rtol=1e-13)
    assert eddy.nu_t_pointwise(eddy.VREMAN, np.zeros((3, 3)), 0.2, C, w) == 0.0


@pytest.mark.parametrize("model", [eddy.SMAGORINSKY, eddy.WALE, eddy.QR, eddy.VREMAN])
def test_dissipation_identity(model):
    """sum_a sum_I u^a e^a = -sum_I [sum_a 2 nu_t S_aa^2 + sum_{a != b} 2 nu_edge S_ab^2] (uniform grid)."""
    g = periodic_grid(6, 3)
    u = random_u(g, 11)
    nu = eddy.eddy_viscosity(g, u, model)
    assert np.all(nu >= 0.0)
    e = eddy.stress_divergence(g, u, nu)
    lhs = float(np.sum(u * e))
    rhs = 0.0
    for a in range(3):
        rhs -= np.sum(2.0 * nu * eddy.diag_strain(g, u, a) ** 2)
        for b in range(3):
            if b == a:
                continue
            ax, bx = g.axis(a), g.axis(b)
            nu_e = 0.25 * (nu + np.roll(nu, -1, ax) + np.roll(nu, -1, bx) + np.roll(np.roll(nu, -1, ax), -1, bx))
            Sab = 0.5 * (eddy.edge_grad(g, u, a, b) + eddy.edge_grad(g, u, b, a))
            rhs -= np.sum(2.0 * nu_e * Sab ** 2)
    assert lhs <= 0.0
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_gradient_at_centres_second_order():
    """A from the staggered stencils converges to the exact gradient at second order."""
    errs = []
    for n in (16, 32):
        faces = [uniform_faces(n, 0, 2 * np.pi) for _ in range(3)]
        g = Grid(faces, ["periodic"] * 3, 0.0)
        u = g.zeros_u()
        # u^x = sin(y) cos(z) at the x-faces, u^y = sin(z) at the y-faces, u^z = sin(x) at the z-faces
        x, y, z = [f.reshape(s) for f, s in zip((g.xc[0], g.xc[1], g.xc[2]), ((1, 1, n), (1, n, 1), (n, 1, 1)))]
        u[0] = np.sin(y) * np.cos(z) * np.ones(g.shape)
        u[1] = np.sin(z) * np.ones(g.shape)
        u[2] = np.sin(x) * np.ones(g.shape)
        A = eddy.gradient_at_centres(g, u)
        exact = np.zeros_like(A)
        exact[0, 1] = np.cos(y) * np.cos(z) * np.ones(g.shape)
        exact[0, 2] = -np.sin(y) * np.sin(z) * np.ones(g.shape)
        exact[1, 2] = np.cos(z) * np.ones(g.shape)
        exact[2, 0] = np.cos(x) * np.ones(g.shape)
        errs.append(np.max(np.abs(A - exact)))
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_closure_enters_rhs():
    """operators.rhs_F adds the eddy term; a Smagorinsky LES field loses energy faster."""
    g = periodic_grid(8, 3, nu=0.0)
    u = random_u(g, 5)
    F0 = op.rhs_F(g, u)
    F1 = op.rhs_F(g, u, eddy.closure(g, eddy.SMAGORINSKY))
    np.testing.assert_allclose(F1 - F0, eddy.closure_term(g, u, eddy.SMAGORINSKY), rtol=0, atol=1e-13)
    assert float(np.sum(u * (F1 - F0))) < 0.0


def test_wall_constant_viscosity_identity():
    """On a tanh channel the constant-viscosity identity holds with the wall rules too."""
    from test_oracle_operators import channel_grid
    g = channel_grid(6, 7, 5)
    u = random_u(g, 3)
    c = 0.37
    e = eddy.stress_divergence(g, u, c * np.ones(g.shape))
    ref = c * (op.diffusion(g, u) + op.gradient(g, op.divergence(g, u)))
    np.testing.assert_allclose(e, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_wall_shear_with_row_viscosity_closed_form():
    """u^x = U(y), nu_t = f(y): e^x is the 1-D flux difference
    [nu_{j+1/2} (U_{j+1} - U_j) / h_j - nu_{j-1/2} (U_j - U_{j-1}) / h_{j-1}] / d_j with
    nu_{j+1/2} = (f_j + f_{j+1}) / 2, the odd velocity ghost at the walls (U_{-1} = -U_0,
    U_ny = -U_{ny-1}, h_{-1} = d_0, h_{ny-1} = d_{ny-1}) and the even viscosity ghost
    (f_{-1} = f_0, f_ny = f_{ny-1}); e^y = e^z = 0."""
    from test_oracle_operators import channel_grid
    g = channel_grid(4, 9, 3)
    ny = g.n[1]
    rng = np.random.default_rng(7)
    U = rng.standard_normal(ny)
    f = 0.1 + rng.random(ny)
    u = g.zeros_u()
    u[0] = U.reshape(1, ny, 1) * np.ones(g.shape)
    nu = f.reshape(1, ny, 1) * np.ones(g.shape)
    e = eddy.stress_divergence(g, u, nu)
    d, h = g.d[1], g.h[1]
    want = np.zeros(ny)
    for j in range(ny):
        Up = U[j + 1] if j + 1 < ny else -U[j]
        Um = U[j - 1] if j > 0 else -U[j]
        fp = 0.5 * (f[j] + (f[j + 1] if j + 1 < ny else f[j]))
        fm = 0.5 * (f[j] + (f[j - 1] if j > 0 else f[j]))
        hm = h[j - 1] if j > 0 else d[0]
        want[j] = (fp * (Up - U[j]) / h[j] - fm * (U[j] - Um) / hm) / d[j]
    np.testing.assert_allclose(e[0][0, :, 0], want, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(e[1:], 0.0, atol=1e-13)
