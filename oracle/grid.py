"""Staggered Cartesian (MAC) grid, built from face coordinates.

Paper: Sec. 2.1 (staggered grid), App. A (staggered grid configuration),
Sec. 2.5 (non-uniform grids, tanh-grid equation).

Conventions (storage index, no ghost cells in the stored arrays):

* direction alpha = 0 (x), 1 (y), 2 (z); a field array has shape
  (nz, ny, nx) in 3-D and (ny, nx) in 2-D, so x is the fastest axis and
  direction alpha lives on numpy axis ``dim - 1 - alpha``;
* cell i of direction alpha spans [faces[i], faces[i+1]], width d[i];
* pressure p[I] sits at the cell centre; u^alpha[I] sits on the face to the
  right of cell I in direction alpha (the paper's "one velocity component to
  the right of the volume centre" convention, Sec. 3.1);
* h[i] is the distance between the centres of cells i and i+1 (the width of
  the alpha-velocity volume of face i). Periodic: the last one wraps,
  h[n-1] = (d[n-1] + d[0]) / 2. Wall: the ghost cell beyond each wall mirrors
  the first interior cell, so h[n-1] = d[n-1] and the spacing below cell 0 is
  h_lo = d[0].

A wall direction (no-slip, Sec. 2.4 Dirichlet u = 0) stores u^alpha on its
n faces 1..n; the last one is the top wall and holds 0. The bottom wall face
is not stored and is 0.
"""

import numpy as np

PERIODIC = "periodic"
WALL = "wall"


def uniform_faces(n, a, b):
    """n+1 equally spaced face coordinates on [a, b] (Sec. 2.5, uniform grid)."""
    return a + (b - a) * np.arange(n + 1, dtype=np.float64) / n


def tanh_faces(n, a, b, gamma):
    """Hyperbolic-tangent stretched faces (Sec. 2.5, tanh-grid equation).

    x_i = a + (b - a)/2 * (1 + tanh(gamma (2 i/n - 1)) / tanh(gamma)).
    """
    s = np.arange(n + 1, dtype=np.float64) / n
    return a + 0.5 * (b - a) * (1.0 + np.tanh(gamma * (2.0 * s - 1.0)) / np.tanh(gamma))


class Grid:
    """A staggered grid in 2 or 3 dimensions.

    faces: list of dim 1-D arrays (n_alpha + 1 face coordinates each)
    bc:    list of dim strings, "periodic" or "wall"
    nu:    kinematic viscosity
    force: constant body force f^alpha (App. A momentum equation); default 0
    """

    def __init__(self, faces, bc, nu, force=None):
        self.dim = len(faces)
        assert self.dim in (2, 3)
        assert len(bc) == self.dim
        self.faces = [np.asarray(f, dtype=np.float64) for f in faces]
        self.bc = list(bc)
        self.nu = float(nu)
        self.force = np.zeros(self.dim) if force is None else np.asarray(force, dtype=np.float64)
        self.n = tuple(len(f) - 1 for f in self.faces)
        # numpy shape: reversed direction order (x fastest)
        self.shape = tuple(reversed(self.n))
        self.d = [np.diff(f) for f in self.faces]            # cell widths
        self.xc = [0.5 * (f[:-1] + f[1:]) for f in self.faces]  # cell centres
        self.h = []
        self.h_lo = []
        for a in range(self.dim):
            d = self.d[a]
            if self.bc[a] == PERIODIC:
                d_next = np.roll(d, -1)
                self.h.append(0.5 * (d + d_next))
                self.h_lo.append(0.5 * (d[-1] + d[0]))
            else:
                d_next = np.concatenate([d[1:], d[-1:]])  # mirrored ghost above
                self.h.append(0.5 * (d + d_next))
                self.h_lo.append(d[0])                     # mirrored ghost below
        self.length = [f[-1] - f[0] for f in self.faces]

    # ------------------------------------------------------------------ helpers
    def axis(self, a):
        """numpy axis of direction a."""
        return self.dim - 1 - a

    def along(self, v, a):
        """Reshape a 1-D per-index array of direction a so that it broadcasts."""
        shp = [1] * self.dim
        shp[self.axis(a)] = -1
        return np.asarray(v).reshape(shp)

    def zeros_u(self):
        return np.zeros((self.dim,) + self.shape)

    def zeros_p(self):
        return np.zeros(self.shape)

    def wall_dirs(self):
        return [a for a in range(self.dim) if self.bc[a] == WALL]

    def face_mask(self, a):
        """1 where u^a is an unknown, 0 on a stored wall face (top of a wall direction).

        The momentum equation is only evaluated in the velocity unknowns
        (Sec. 2.3: boundary values are stored with the solution but the momentum
        equation is not defined there).
        """
        m = np.ones(self.shape)
        if self.bc[a] == WALL:
            idx = [slice(None)] * self.dim
            idx[self.axis(a)] = -1
            m[tuple(idx)] = 0.0
        return m

    def cell_volume(self):
        """|Omega_I| for every pressure cell."""
        v = np.ones(self.shape)
        for a in range(self.dim):
            v = v * self.along(self.d[a], a)
        return v

    def face_volume(self, a):
        """|Omega^a_I|: the volume of the a-velocity control volume of face I."""
        v = np.ones(self.shape) * self.along(self.h[a], a)
        for b in range(self.dim):
            if b != a:
                v = v * self.along(self.d[b], b)
        return v * self.face_mask(a)

    def face_coords(self, a):
        """Coordinates of the u^a unknowns: a list of dim broadcastable arrays."""
        out = []
        for b in range(self.dim):
            if b == a:
                out.append(self.along(self.faces[b][1:], b))
            else:
                out.append(self.along(self.xc[b], b))
        return out

    def cell_coords(self):
        return [self.along(self.xc[b], b) for b in range(self.dim)]

    def is_uniform(self, a, rtol=1e-12):
        d = self.d[a]
        return np.max(np.abs(d - d.mean())) <= rtol * d.mean()
