"""Closed-form pins of the oracle's channel statistics, face-average filter and CFL rule.

Each pin evaluates the oracle on a field whose answer is written out by hand, and
each is shown to reject a planted mistake (a shifted face, the wrong wall value,
a missing mean subtraction, a cell width in place of a centre distance), so the
pin really constrains the part of the function it is about.

Paper: Sec. 6.2 (channel statistics from velocities interpolated to the volume
centres), Sec. 4 (filtered DNS: face averaging to the coarse grid), Sec. 2.6.2
(adaptive time step from the convective and diffusive limits).
"""

import numpy as np
import pytest

from oracle import diagnostics, timestep, operators as op
from oracle.grid import Grid, uniform_faces, tanh_faces
from test_oracle_operators import stretched_periodic_grid


# ------------------------------------------------------------ channel statistics
LX, LY, LZ = 4 * np.pi, 2.0, 4 * np.pi / 3
NX, NY, NZ = 12, 10, 8
KX = 2 * np.pi * 2 / LX      # two periods in x
KZ = 2 * np.pi * 1 / LZ      # one period in z
A, B, C = 0.7, 1.3, 0.4


def _f(y):
    return 3.0 * y * (2.0 - y)


def _g(y):
    return y * (2.0 - y)       # vanishes on both walls


def _e(y):
    return 1.0 + y


def _channel():
    faces = [uniform_faces(NX, 0, LX), tanh_faces(NY, 0, LY, 1.5), uniform_faces(NZ, 0, LZ)]
    return Grid(faces, ["periodic", "wall", "periodic"], 1.0 / 180)


def _analytic_channel_field(g):
    """u^x = f(y) + A sin(kx x), u^y = B g(y) sin(kx x), u^z = C e(y) cos(kz z), each at its own face."""
    xf, yf, zf = (f[1:] for f in g.faces)
    xc, yc, zc = g.xc
    u = g.zeros_u()
    u[0] = _f(yc)[None, :, None] + A * np.sin(KX * xf)[None, None, :]
    u[1] = B * _g(yf)[None, :, None] * np.sin(KX * xc)[None, None, :]
    u[2] = C * _e(yc)[None, :, None] * np.cos(KZ * zf)[:, None, None]
    return u


def _expected_profiles(g):
    """Plane means and covariances of the centre velocities, by hand.

    Centre of cell i in x: the mean of the faces at xf[i] and xf[i+1], so
    (sin(k xf[i]) + sin(k xf[i+1]))/2 = cos(k dx/2) sin(k xc[i]). In y the face
    below row 0 is the bottom wall, where u^y = 0 = g(0). Over whole periods of
    uniform samples <sin> = <cos> = 0 and <sin^2> = <cos^2> = 1/2.
    """
    yf = g.faces[1]
    yc = g.xc[1]
    cx = np.cos(KX * (LX / NX) / 2)
    cz = np.cos(KZ * (LZ / NZ) / 2)
    gb = 0.5 * (_g(yf[:-1]) + _g(yf[1:]))
    zero = np.zeros(NY)
    mean = [_f(yc), zero, zero]
    cov = {(0, 0): 0.5 * (A * cx) ** 2 * np.ones(NY),
           (0, 1): 0.5 * A * cx * B * gb,
           (0, 2): zero,
           (1, 1): 0.5 * (B * gb) ** 2,
           (1, 2): zero,
           (2, 2): 0.5 * (C * _e(yc) * cz) ** 2}
    return mean, cov


def _profile_error(profiles_fn):
    g = _channel()
    u = _analytic_channel_field(g)
    mean, cov = profiles_fn(g, u)
    em, ec = _expected_profiles(g)
    err = max(float(np.max(np.abs(mean[a] - em[a]))) for a in range(3))
    err = max(err, max(float(np.max(np.abs(cov[k] - ec[k]))) for k in ec))
    return err


def test_wall_profiles_closed_form():
    """Plane means and covariances of an analytic channel field equal the hand-written values."""
    assert _profile_error(diagnostics.wall_profiles) < 1e-13


def test_centre_velocity_closed_form():
    """Centre velocities, cell by cell, including row 0 where the bottom-wall u^y = 0 enters."""
    g = _channel()
    uc = diagnostics.centre_velocity(g, _analytic_channel_field(g))
    xc, yc, zc = g.xc
    yf = g.faces[1]
    cx = np.cos(KX * (LX / NX) / 2)
    cz = np.cos(KZ * (LZ / NZ) / 2)
    ex = _f(yc)[None, :, None] + A * cx * np.sin(KX * xc)[None, None, :]
    ey = B * (0.5 * (_g(yf[:-1]) + _g(yf[1:])))[None, :, None] * np.sin(KX * xc)[None, None, :]
    ez = C * cz * _e(yc)[None, :, None] * np.cos(KZ * zc)[:, None, None]
    for got, want in zip(uc, (ex, ey, ez)):
        np.testing.assert_allclose(got, np.broadcast_to(want, got.shape), rtol=0, atol=1e-13)
    # row 0 of u^y by itself: half the first interior face value (the wall face below holds 0)
    np.testing.assert_allclose(uc[1][:, 0, :], 0.5 * _analytic_channel_field(g)[1][:, 0, :],
                               rtol=0, atol=1e-15)


def test_profile_pin_rejects_centre_from_wrong_neighbour(monkeypatch):
    """Planted mistake: the centre averaged with the face above instead of the face below."""
    def shifted(g, u):
        out = g.zeros_u()
        for a in range(g.dim):
            out[a] = 0.5 * (u[a] + op.shift(g, u[a], a, +1, op.NORMAL))
        return out

    monkeypatch.setattr(diagnostics, "centre_velocity", shifted)
    assert _profile_error(diagnostics.wall_profiles) > 1e-3


def test_profile_pin_rejects_mirrored_wall_value(monkeypatch):
    """Planted mistake: an even (mirrored) ghost below row 0 instead of the zero wall face."""
    real_shift = op.shift

    def mirrored(g, f, a, s, kind):
        return real_shift(g, f, a, s, op.EVEN if kind == op.NORMAL else kind)

    monkeypatch.setattr(op, "shift", mirrored)
    assert _profile_error(diagnostics.wall_profiles) > 1e-3


def test_profile_pin_rejects_missing_mean_subtraction():
    """Planted mistake: raw second moments reported as covariances."""
    def raw_moments(g, u):
        uc = diagnostics.centre_velocity(g, u)
        axes = (g.axis(0), g.axis(2))
        mean = [np.mean(uc[a], axis=axes) for a in range(3)]
        cov = {(a, b): np.mean(uc[a] * uc[b], axis=axes) for a in range(3) for b in range(a, 3)}
        return mean, cov

    assert _profile_error(raw_moments) > 1e-1


# ------------------------------------------------------------ face-average filter
def _linear_field(faces, coef):
    """u^a = coef[a][0] + sum_b coef[a][b+1] x_b at the u^a positions of the grid with these faces."""
    dim = len(faces)
    shape = tuple(len(f) - 1 for f in reversed(faces))
    u = np.zeros((dim,) + shape)
    for a in range(dim):
        val = np.full(shape, coef[a][0])
        for b in range(dim):
            f = faces[b]
            x = f[1:] if b == a else 0.5 * (f[:-1] + f[1:])
            shp = [1] * dim
            shp[dim - 1 - b] = -1
            val = val + coef[a][b + 1] * x.reshape(shp)
        u[a] = val
    return u


_COEF = [(0.3, 1.1, -0.7, 0.5), (-0.2, 0.4, 1.9, -0.6), (1.0, -0.8, 0.3, 1.4)]


def _filter_error(filter_fn, dim, nc, m):
    """Max deviation of the filtered linear field from the same field at the coarse face positions.

    A coarse face is tiled by fine faces at the same coordinate along its own
    direction; averaging a linear function over the m fine cell centres in each
    other direction gives its value at the coarse cell centre. So for a linear
    field the coarse value is the field evaluated at the coarse face position.
    """
    lengths = [2 * np.pi, 3.0, 1.5][:dim]
    fine = [uniform_faces(m * n, 0, L) for n, L in zip(nc, lengths)]
    coarse = [uniform_faces(n, 0, L) for n, L in zip(nc, lengths)]
    coef = [c[:dim + 1] for c in _COEF[:dim]]
    got = filter_fn(_linear_field(fine, coef), dim, m)
    want = _linear_field(coarse, coef)
    return float(np.max(np.abs(got - want)))


@pytest.mark.parametrize("dim,nc,m", [(2, (5, 3), 4), (3, (5, 4, 3), 4), (3, (3, 3, 3), 2)])
def test_face_average_filter_linear_field(dim, nc, m):
    assert _filter_error(diagnostics.face_average_filter, dim, nc, m) < 1e-12


@pytest.mark.parametrize("shift", [1, 2])
def test_filter_pin_rejects_shifted_fine_face(shift):
    """Planted mistake: each coarse face averages a fine face `shift` fine cells below the right one
    (also divergence free, so the divergence pin cannot see it)."""
    def shifted(u_fine, dim, m):
        v = u_fine.copy()
        for a in range(dim):
            v[a] = np.roll(u_fine[a], shift, axis=dim - 1 - a)
        return diagnostics.face_average_filter(v, dim, m)

    assert _filter_error(shifted, 3, (5, 4, 3), 4) > 0.1


# ------------------------------------------------------------ CFL rule
def _cfl_channel(nu, geometric=False):
    """A wall-bounded box: tanh-stretched y, or (geometric=True) cells growing by 1.2 from the bottom wall,
    so that no centre distance equals the smallest cell width (the tanh grid's top ghost mirrors it)."""
    if geometric:
        w = 1.2 ** np.arange(8)
        y = np.concatenate([[0.0], np.cumsum(w)]) * (2.0 / w.sum())
    else:
        y = tanh_faces(8, 0, 2, 1.5)
    faces = [uniform_faces(6, 0, 4 * np.pi), y, uniform_faces(4, 0, 4 * np.pi / 3)]
    return Grid(faces, ["periodic", "wall", "periodic"], nu)


def _single_value_u(g, a, idx, v):
    u = g.zeros_u()
    u[a][idx] = v
    return u


def test_cfl_convective_limit_stretched_wall_direction():
    """One nonzero u^y = -2.5 at row j = 1 of a tanh grid: dt = 0.3 (y[3] - y[1]) / 2 / 2.5."""
    g = _cfl_channel(1e-4)
    y = g.faces[1]
    u = _single_value_u(g, 1, (1, 1, 2), -2.5)
    want = 0.3 * ((y[3] - y[1]) / 2) / 2.5
    assert want < 0.3 * (y[1] - y[0]) ** 2 / 1e-4      # the convective limit is the active one
    assert timestep.cfl_dt(g, u, 0.3) == pytest.approx(want, rel=1e-15)


def test_cfl_convective_limit_wrapped_periodic_face():
    """Nonzero u^x on the last face of a non-uniform periodic direction: h = (d[n-1] + d[0]) / 2."""
    g = stretched_periodic_grid(6, 3, nu=1e-6)
    x = g.faces[0]
    u = _single_value_u(g, 0, (2, 1, 5), 1.7)
    want = 0.3 * (((x[6] - x[5]) + (x[1] - x[0])) / 2) / 1.7
    assert timestep.cfl_dt(g, u, 0.3) == pytest.approx(want, rel=1e-15)


@pytest.mark.parametrize("geometric", [False, True])
def test_cfl_diffusive_limit_is_smallest_cell_squared(geometric):
    """With nu = 1 the diffusive limit wins: dt = 0.3 (y[1] - y[0])^2 / nu (the bottom wall cell)."""
    g = _cfl_channel(1.0, geometric)
    y = g.faces[1]
    u = _single_value_u(g, 1, (1, 1, 2), -2.5)
    assert timestep.cfl_dt(g, u, 0.3) == pytest.approx(0.3 * (y[1] - y[0]) ** 2 / 1.0, rel=1e-15)


def test_cfl_zero_field_is_diffusive_limit():
    g = _cfl_channel(0.25)
    y = g.faces[1]
    assert timestep.cfl_dt(g, g.zeros_u(), 0.3) == pytest.approx(0.3 * (y[1] - y[0]) ** 2 / 0.25, rel=1e-15)


def test_cfl_pin_rejects_cell_width_for_centre_distance():
    """Planted mistake: the cell width d in place of the centre distance h in the convective limit."""
    g = _cfl_channel(1e-4)
    y = g.faces[1]
    u = _single_value_u(g, 1, (1, 1, 2), -2.5)
    g.h = [d.copy() for d in g.d]
    want = 0.3 * ((y[3] - y[1]) / 2) / 2.5
    assert abs(timestep.cfl_dt(g, u, 0.3) - want) > 1e-3 * want


def test_cfl_pin_rejects_centre_distance_in_diffusive_limit():
    """Planted mistake: min h^2 / nu in place of min d^2 / nu (h > d next to a stretched wall)."""
    g = _cfl_channel(1.0, geometric=True)
    y = g.faces[1]
    u = _single_value_u(g, 1, (1, 1, 2), -2.5)
    g.d = [h.copy() for h in g.h]
    want = 0.3 * (y[1] - y[0]) ** 2 / 1.0
    assert abs(timestep.cfl_dt(g, u, 0.3) - want) > 1e-3 * want
