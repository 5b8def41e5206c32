"""Discrete operators of the staggered finite-volume scheme (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Sec. 2.2 (discrete derivative, the four operators), App. A (momentum
equation eq. P2:momentum_discrete: convection with weights 1/2 for the
transported alpha-component and interpolation of the beta-component,
diffusion, force, pressure gradient), App. B (divergence, pressure-gradient,
diffusion and convection kernels).

Every operator is written as whole-array numpy expressions over the storage
index (see ``oracle.grid`` for the index conventions) with one helper,
``shift``, that supplies neighbour values including the boundary rule:

* periodic: wrap-around (Sec. 2.4, periodic ghost volumes);
* wall (no-slip, Sec. 2.4 Dirichlet u = 0):
  - NORMAL kind (u^a along its own direction a): the wall faces hold 0;
  - TANGENT kind (u^a along another direction b): the ghost cell holds the
    odd reflection -u, so the value interpolated onto the wall is 0;
  - EVEN kind (pressure): even reflection. It never reaches a result because
    the pressure gradient is not applied on wall faces.

Reading taken where the appendix indices are ambiguous on stretched grids: the
transported component is averaged with weights 1/2 and the advecting component
is interpolated along alpha with volume weights d[i]/(d[i]+d[i+1]) on the left
value. With these weights the mass fluxes through the faces of each velocity
volume add up to half the sum of the divergences of the two pressure cells it
overlaps, which makes the convection operator exactly energy conserving on
divergence-free fields (the property claimed in App. A/B and tested in
Sec. 5.8). On uniform grids every reading gives weights 1/2.
"""

import numpy as np

from .grid import PERIODIC

NORMAL = "normal"
TANGENT = "tangent"
EVEN = "even"


def shift(g, f, a, s, kind):
    """Value of f at storage index I + s*e_a (s = +1 or -1), with the boundary rule."""
    ax = g.axis(a)
    out = np.roll(f, -s, axis=ax)
    if g.bc[a] == PERIODIC:
        return out
    n = g.n[a]
    idx = [slice(None)] * g.dim
    src = [slice(None)] * g.dim
    if s == +1:
        idx[ax] = n - 1          # wants f[n]: beyond the last stored index
        src[ax] = n - 1
        if kind == NORMAL:
            out[tuple(idx)] = 0.0              # never used (wall face is not an unknown)
        elif kind == TANGENT:
            out[tuple(idx)] = -f[tuple(src)]   # odd ghost above the top wall
        else:
            out[tuple(idx)] = f[tuple(src)]
    elif s == -1:
        idx[ax] = 0              # wants f[-1]
        src[ax] = 0
        if kind == NORMAL:
            out[tuple(idx)] = 0.0              # bottom wall face
        elif kind == TANGENT:
            out[tuple(idx)] = -f[tuple(src)]   # odd ghost below the bottom wall
        else:
            out[tuple(idx)] = f[tuple(src)]
    else:
        raise ValueError("shift by +1 or -1 only")
    return out


def d_next(g, a):
    """Width of the next cell, d[i+1] (wrapped, or the mirrored ghost at a wall)."""
    d = g.d[a]
    if g.bc[a] == PERIODIC:
        return np.roll(d, -1)
    return np.concatenate([d[1:], d[-1:]])


def h_prev(g, a):
    """h[i-1], the centre distance below cell i (h_lo for i = 0)."""
    return np.concatenate([[g.h_lo[a]], g.h[a][:-1]])


# --------------------------------------------------------------------- App. B
def divergence(g, u):
    """(D u)_I = sum_a (u^a_I - u^a_{I-e_a}) / d_a[i]   (App. B, divergence kernel)."""
    out = g.zeros_p()
    for a in range(g.dim):
        out += (u[a] - shift(g, u[a], a, -1, NORMAL)) / g.along(g.d[a], a)
    return out


def gradient(g, p):
    """(G p)^a_I = (p_{I+e_a} - p_I) / h_a[i]   (App. B, pressure-gradient kernel).

    Zero on stored wall faces, which are not unknowns.
    """
    out = g.zeros_u()
    for a in range(g.dim):
        out[a] = (shift(g, p, a, +1, EVEN) - p) / g.along(g.h[a], a) * g.face_mask(a)
    return out


def diffusion(g, u):
    """sum_b delta_b delta_b u^a, WITHOUT the factor nu   (App. B, diffusion kernel).

    b == a: the inner differences sit at the cell centres (widths d), the outer
            one divides by the velocity-volume width h.
    b != a: the inner differences sit at the b-faces (distances h), the outer
            one divides by the cell width d.
    """
    out = g.zeros_u()
    for a in range(g.dim):
        ua = u[a]
        for b in range(g.dim):
            if b == a:
                up = shift(g, ua, a, +1, NORMAL)
                um = shift(g, ua, a, -1, NORMAL)
                term = ((up - ua) / g.along(d_next(g, a), a)
                        - (ua - um) / g.along(g.d[a], a)) / g.along(g.h[a], a)
            else:
                up = shift(g, ua, b, +1, TANGENT)
                um = shift(g, ua, b, -1, TANGENT)
                term = ((up - ua) / g.along(g.h[b], b)
                        - (ua - um) / g.along(h_prev(g, b), b)) / g.along(g.d[b], b)
            out[a] += term
        out[a] *= g.face_mask(a)
    return out


def interp_weights(g, a):
    """Volume weights for interpolating a cell-located quantity along a onto face i.

    Returns (wl, wr) with wl = d[i]/(d[i]+d[i+1]), wr = d[i+1]/(d[i]+d[i+1]).
    Uniform grid: both 1/2.
    """
    d = g.d[a]
    dn = d_next(g, a)
    return d / (d + dn), dn / (d + dn)


def convection_bilinear(g, adv, tra):
    """B(adv, tra): the convective term of App. A with advecting field ``adv`` and
    transported field ``tra``; the convection of u is C(u) = B(u, u).

    For component a and direction b the a-velocity volume of face I loses the
    flux difference  (V_+ T_+ - V_- T_-) / width_b  where
      b == a: V_+, T_+ are adv^a, tra^a averaged (1/2, 1/2) onto the cell centre
              i+1 and V_-, T_- onto centre i; width = h_a[i];
      b != a: V_+ is adv^b interpolated along a (volume weights) onto the
              b-face above I, V_- the same one b-face below; T_+-, T_- are tra^a
              averaged (1/2, 1/2) onto those b-faces; width = d_b[j].
    """
    out = g.zeros_u()
    for a in range(g.dim):
        ta = tra[a]
        for b in range(g.dim):
            if b == a:
                aa = adv[a]
                vp = 0.5 * (aa + shift(g, aa, a, +1, NORMAL))
                vm = 0.5 * (shift(g, aa, a, -1, NORMAL) + aa)
                tp = 0.5 * (ta + shift(g, ta, a, +1, NORMAL))
                tm = 0.5 * (shift(g, ta, a, -1, NORMAL) + ta)
                out[a] -= (vp * tp - vm * tm) / g.along(g.h[a], a)
            else:
                ab = adv[b]
                wl, wr = interp_weights(g, a)
                vp = g.along(wl, a) * ab + g.along(wr, a) * shift(g, ab, a, +1, TANGENT)
                vm = shift(g, vp, b, -1, NORMAL)
                tp = 0.5 * (ta + shift(g, ta, b, +1, TANGENT))
                tm = 0.5 * (shift(g, ta, b, -1, TANGENT) + ta)
                out[a] -= (vp * tp - vm * tm) / g.along(g.d[b], b)
        out[a] *= g.face_mask(a)
    return out


def convection(g, u):
    """C(u) = B(u, u)   (App. B, convection kernel)."""
    return convection_bilinear(g, u, u)


def force(g):
    """Constant body force f^a on the velocity unknowns (App. A)."""
    out = g.zeros_u()
    for a in range(g.dim):
        out[a] = g.force[a] * g.face_mask(a)
    return out


def rhs_F(g, u, closure=None):
    """F(u) = C(u) + nu * diffusion(u) + f  (+ closure term m(u) when given)."""
    F = convection(g, u) + g.nu * diffusion(g, u) + force(g)
    if closure is not None:
        F = F + closure(u)
    return F
