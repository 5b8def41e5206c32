"""Pressure Poisson equation L p = D F(u) and the projection (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Sec. 2.6.1 (pressure Poisson equation; L = D G symmetric semi-definite;
spectral solver p = DFT^-1 Lhat^-1 DFT r with Lhat at the zero wavenumber set
to one), Sec. 2.3 (du/dt = F(u) - G p, D u = 0).

Two solvers, matching the grids the method runs on:

* ``solve_periodic``: every direction periodic and uniform. numpy's FFT is the
  DFT; Lhat is the exact symbol of D G,
  lambda_a(k) = -4 sin^2(pi k / n_a) / (d_a h_a).
* ``solve_wall``: one wall-normal direction (no-slip walls, possibly stretched),
  all other directions periodic and uniform. DFT in the periodic directions,
  then for every wavenumber the tridiagonal system of D G along the wall
  direction, solved by the Thomas algorithm in FP64. The wall rows have no
  neighbour outside the wall, because the normal velocity on the wall is fixed
  and no pressure gradient acts there (homogeneous Neumann). Reading taken for
  the mean mode (the paper's direct solver pins the mean with an augmented
  system instead): the row of the first cell is replaced by p_0 = 0, which is
  valid because the system is consistent.

Pressure is defined up to a constant (Sec. 2.6.1); compare it after removing
its volume mean.
"""

import numpy as np

from .grid import PERIODIC, WALL
from . import operators as op


def eigenvalues(g, a):
    """Symbol of the 1-D operator (d/dx)(d/dx) of D G along a periodic uniform direction."""
    n = g.n[a]
    d = g.d[a][0]
    h = g.h[a][0]
    k = np.arange(n)
    return -4.0 * np.sin(np.pi * k / n) ** 2 / (d * h)


def solve_periodic(g, r):
    """p = IDFT(Lhat^-1 DFT r), Lhat(0) := 1   (Sec. 2.6.1, spectral solver)."""
    for a in range(g.dim):
        assert g.bc[a] == PERIODIC and g.is_uniform(a), "spectral solver needs periodic uniform grids"
    rh = np.fft.fftn(r)
    Lh = np.zeros(g.shape)
    for a in range(g.dim):
        Lh = Lh + g.along(eigenvalues(g, a), a)
    Lh[(0,) * g.dim] = 1.0
    return np.real(np.fft.ifftn(rh / Lh))


def thomas(lo, diag, up, rhs):
    """Thomas algorithm for a tridiagonal system along axis 0 (textbook form).

    lo[j] p[j-1] + diag[j] p[j] + up[j] p[j+1] = rhs[j]; lo[0] and up[-1] unused.
    All arrays broadcast over the trailing (mode) axes.
    """
    n = rhs.shape[0]
    cp = np.zeros(np.broadcast(diag, rhs).shape, dtype=np.float64)
    dp = np.zeros(rhs.shape, dtype=rhs.dtype)
    m = diag[0] * np.ones_like(cp[0])
    cp[0] = up[0] / m
    dp[0] = rhs[0] / m
    for j in range(1, n):
        m = diag[j] - lo[j] * cp[j - 1]
        cp[j] = up[j] / m
        dp[j] = (rhs[j] - lo[j] * dp[j - 1]) / m
    x = np.zeros_like(dp)
    x[n - 1] = dp[n - 1]
    for j in range(n - 2, -1, -1):
        x[j] = dp[j] - cp[j] * x[j + 1]
    return x


def solve_wall(g, r):
    """FFT in the periodic directions + FP64 Thomas along the single wall direction."""
    walls = g.wall_dirs()
    assert len(walls) == 1, "exactly one wall-normal direction"
    w = walls[0]
    per = [a for a in range(g.dim) if a != w]
    for a in per:
        assert g.bc[a] == PERIODIC and g.is_uniform(a)
    axes = tuple(g.axis(a) for a in per)
    rh = np.fft.fftn(r, axes=axes)
    lam = np.zeros(g.shape)
    for a in per:
        lam = lam + g.along(eigenvalues(g, a), a)
    # move the wall axis to the front; modes on the remaining axes
    wax = g.axis(w)
    rh = np.moveaxis(rh, wax, 0)
    lam = np.moveaxis(lam, wax, 0)[0]          # lambda does not depend on the wall index
    n = g.n[w]
    d = g.d[w]
    h = g.h[w]
    lo = np.zeros(n)
    up = np.zeros(n)
    lo[1:] = 1.0 / (d[1:] * h[:-1])            # coupling to p[j-1] across face j-1
    up[:-1] = 1.0 / (d[:-1] * h[:-1])          # coupling to p[j+1] across face j
    shp = (n,) + (1,) * (g.dim - 1)
    diag = (-lo - up).reshape(shp) + lam[None]
    lo_b = lo.reshape(shp) * np.ones_like(diag)
    up_b = up.reshape(shp) * np.ones_like(diag)
    # mean mode: replace the first row by p_0 = 0
    mean_idx = (0,) + (0,) * (g.dim - 1)
    diag[mean_idx] = 1.0
    up_b[mean_idx] = 0.0
    rhs = rh.copy()
    rhs[mean_idx] = 0.0
    ph = thomas(lo_b, diag, up_b, rhs)
    ph = np.moveaxis(ph, 0, wax)
    return np.real(np.fft.ifftn(ph, axes=axes))


def solve(g, r):
    """Solve L p = r on the grid's boundary configuration."""
    if g.wall_dirs():
        return solve_wall(g, r)
    return solve_periodic(g, r)


def project(g, u):
    """Divergence-free projection: P u = u - G p with L p = D u. Returns (P u, p)."""
    p = solve(g, op.divergence(g, u))
    return u - op.gradient(g, p), p


def rhs(g, u, closure=None):
    """du/dt = F(u) - G p with L p = D F(u)   (Sec. 2.3 and 2.6.1). Returns (dudt, p)."""
    F = op.rhs_F(g, u, closure)
    p = solve(g, op.divergence(g, F))
    return F - op.gradient(g, p), p


def laplacian(g, p):
    """L p = D G p, the operator the solvers invert."""
    return op.divergence(g, op.gradient(g, p))
