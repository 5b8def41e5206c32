"""Pins of the oracle's pullbacks on wall-bounded (channel) grids (Sec. 3.4, App. B pullbacks).

* dot-product identities <J v, w> = <v, J^T w> for D, G, the diffusion and both arguments of the
  convection bilinear form on tanh-stretched channel grids (exact transposes, any v and w);
* the projection pullback against the transpose of the assembled dense matrix of M P M
  (brute force on a tiny channel; M the mask of the unknown faces);
* the RK4 and Wray step pullbacks against central differences (eps = 1e-6) along seeded
  directions that vanish on the stored wall faces, in u0 and in nu.
"""

import numpy as np
import pytest

from oracle import adjoint, operators as op, poisson, timestep
from oracle.grid import Grid, uniform_faces, tanh_faces
from test_oracle_operators import channel_grid, random_u, dense_matrix


def _dot(a, b):
    return float(np.sum(a * b))


def full_random_u(g, seed):
    """Random values on every stored entry, wall faces included (exact-transpose checks)."""
    rng = np.random.default_rng(seed)
    return 2.0 * rng.random((g.dim,) + g.shape) - 1.0


@pytest.mark.parametrize("dims", [(6, 5, 4), (7, 6)])
def test_linear_adjoints_dot_product_wall(dims):
    g = channel_grid(*dims) if len(dims) == 3 else Grid(
        [uniform_faces(dims[0], 0, 3.0), tanh_faces(dims[1], 0, 2, 1.5)], ["periodic", "wall"], 0.1)
    v = full_random_u(g, 1)
    w = full_random_u(g, 2)
    q = np.random.default_rng(3).random(g.shape)
    s = max(1.0, abs(_dot(op.diffusion(g, v), w)))
    assert abs(_dot(op.divergence(g, v), q) - _dot(v, adjoint.divergence_T(g, q))) < 1e-12 * s
    assert abs(_dot(op.gradient(g, q), w) - _dot(q, adjoint.gradient_T(g, w))) < 1e-12 * s
    assert abs(_dot(op.diffusion(g, v), w) - _dot(v, adjoint.diffusion_T(g, w))) < 1e-12 * s


@pytest.mark.parametrize("dims", [(6, 5, 4), (7, 6)])
def test_convection_adjoint_dot_product_wall(dims):
    g = channel_grid(*dims) if len(dims) == 3 else Grid(
        [uniform_faces(dims[0], 0, 3.0), tanh_faces(dims[1], 0, 2, 1.5)], ["periodic", "wall"], 0.1)
    u = full_random_u(g, 4)
    v = full_random_u(g, 5)
    w = full_random_u(g, 6)
    ab, tb = adjoint.convection_bilinear_T(g, u, u, w)
    s = max(1.0, abs(_dot(op.convection_bilinear(g, v, u), w)))
    assert abs(_dot(op.convection_bilinear(g, v, u), w) - _dot(v, ab)) < 1e-11 * s
    assert abs(_dot(op.convection_bilinear(g, u, v), w) - _dot(v, tb)) < 1e-11 * s
    Jv = op.convection_bilinear(g, v, u) + op.convection_bilinear(g, u, v)
    assert abs(_dot(Jv, w) - _dot(v, adjoint.convection_vjp(g, u, w))) < 1e-11 * s


def test_projection_pullback_is_dense_transpose():
    """project_T equals (M P M)^T column by column (brute force, 4 x 5 x 3 channel)."""
    g = channel_grid(4, 5, 3)
    nin = g.dim * int(np.prod(g.shape))

    def P(x):
        return adjoint.mask_u(g, poisson.project(g, adjoint.mask_u(g, x.reshape((g.dim,) + g.shape)))[0])

    def PT(x):
        return adjoint.project_T(g, x.reshape((g.dim,) + g.shape))

    M = dense_matrix(g, P, nin, nin)
    MT = dense_matrix(g, PT, nin, nin)
    np.testing.assert_allclose(MT, M.T, rtol=0, atol=1e-11)


@pytest.mark.parametrize("scheme", ["rk4", "wray3"])
def test_step_vjp_fd_wall(scheme):
    g = channel_grid(6, 6, 4, nu=0.05)
    u0, _ = poisson.project(g, random_u(g, 21))
    dt = 0.5 * timestep.cfl_dt(g, u0, 0.3)
    c = random_u(g, 22)
    step = timestep.rk4_step if scheme == "rk4" else timestep.wray3_step

    def loss(u, nu):
        gg = channel_grid(6, 6, 4, nu=nu)
        return _dot(c, step(gg, u, dt))

    if scheme == "rk4":
        ubar, nubar = adjoint.rk4_step_vjp(g, u0, dt, c)
    else:
        ubar, nubar = adjoint.wray3_step_vjp(g, u0, dt, c)
    for a in range(g.dim):
        assert np.all(ubar[a][g.face_mask(a) == 0] == 0.0)
    eps = 1e-6
    for seed in range(3):
        du = random_u(g, 100 + seed)
        fd = (loss(u0 + eps * du, g.nu) - loss(u0 - eps * du, g.nu)) / (2 * eps)
        assert abs(fd - _dot(ubar, du)) < 1e-7 * max(1, abs(fd))
    fdn = (loss(u0, g.nu + eps) - loss(u0, g.nu - eps)) / (2 * eps)
    assert abs(fdn - nubar) < 1e-6 * max(1, abs(fdn))
