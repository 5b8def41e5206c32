"""Diagnostics: kinetic energy, divergence, face-averaging filter, spectrum, profiles.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Sec. 2.3 (energy conservation, duality of D and G), Sec. 6.2
(channel statistics: mean velocity and Reynolds stresses from velocities
interpolated to the volume centres), Sec. 4 (filtered DNS as training data).

Readings taken where the paper is silent:
* kinetic energy is the volume average (1/|Omega|) * 1/2 sum_a sum_I |Omega^a_I| (u^a_I)^2;
* the filter from a fine grid to a coarse grid m times coarser takes, for each
  coarse face, the mean of the m^(d-1) fine face values of the same component
  that tile it (a face average, so the coarse divergence is the average of
  fine divergences and stays zero);
* the shell spectrum of a periodic cubic grid is
  E(k) = sum over |kvec| in [k - 1/2, k + 1/2) of 1/2 sum_a |uhat^a(kvec)|^2 / N^(2d)
  with uhat the unnormalised DFT and integer wavenumbers.
"""

import numpy as np

from . import operators as op


def kinetic_energy(g, u):
    """Volume-averaged kinetic energy."""
    tot = 0.0
    for a in range(g.dim):
        tot += 0.5 * float(np.sum(g.face_volume(a) * u[a] ** 2))
    return tot / float(np.prod(g.length))


def max_abs_div(g, u):
    return float(np.max(np.abs(op.divergence(g, u))))


def face_average_filter(u_fine, dim, m):
    """Coarse face values: mean of the m^(dim-1) fine faces of the same component tiling each coarse face.

    u_fine has shape (dim, *fine_shape) with x the last axis; the fine grid has
    m times as many cells as the coarse one in every direction.
    """
    fine_shape = u_fine.shape[1:]
    coarse_shape = tuple(s // m for s in fine_shape)
    out = np.zeros((dim,) + coarse_shape)
    for a in range(dim):
        ax = dim - 1 - a
        f = u_fine[a]
        # the right face of coarse cell I in direction a is fine face (I+1) m - 1
        sl = [slice(None)] * dim
        sl[ax] = slice(m - 1, None, m)
        f = f[tuple(sl)]
        # average over the m fine cells in each other direction
        for b in range(dim):
            if b == a:
                continue
            bx = dim - 1 - b
            shp = list(f.shape)
            shp[bx:bx + 1] = [shp[bx] // m, m]
            f = f.reshape(shp).mean(axis=bx + 1)
        out[a] = f
    return out


def shell_spectrum(u):
    """E(k) for k = 0..N/2 of a periodic cubic (or square) field u of shape (dim, N, ..., N)."""
    dim = u.shape[0]
    N = u.shape[1]
    e = np.zeros(u.shape[1:])
    for a in range(dim):
        uh = np.fft.fftn(u[a])
        e += 0.5 * np.abs(uh) ** 2
    e /= float(N) ** (2 * dim)
    k1 = np.fft.fftfreq(N, d=1.0 / N)
    grids = np.meshgrid(*([k1] * dim), indexing="ij")
    kmag = np.sqrt(sum(gk ** 2 for gk in grids))
    kmax = N // 2
    E = np.zeros(kmax + 1)
    shell = np.floor(kmag + 0.5).astype(np.int64)
    for k in range(kmax + 1):
        E[k] = float(np.sum(e[shell == k]))
    return E


def centre_velocity(g, u):
    """Velocity components interpolated to the cell centres (mean of the two faces)."""
    out = g.zeros_u()
    for a in range(g.dim):
        out[a] = 0.5 * (u[a] + op.shift(g, u[a], a, -1, op.NORMAL))
    return out


def wall_profiles(g, u):
    """Plane averages along the wall direction (y) of the centre velocities.

    Returns (mean[a], cov) with mean[a][j] = <u^a_c>(y_j) and
    cov[(a, b)][j] = <u^a_c u^b_c> - <u^a_c><u^b_c> for a <= b.
    """
    w = g.wall_dirs()[0]
    uc = centre_velocity(g, u)
    axes = tuple(g.axis(a) for a in range(g.dim) if a != w)
    mean = [np.mean(uc[a], axis=axes) for a in range(g.dim)]
    cov = {}
    for a in range(g.dim):
        for b in range(a, g.dim):
            cov[(a, b)] = np.mean(uc[a] * uc[b], axis=axes) - mean[a] * mean[b]
    return mean, cov
