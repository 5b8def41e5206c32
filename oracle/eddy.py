"""Eddy-viscosity closure models on the staggered grid (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: App. "Eddy-viscosity models" (general framework: m^a = -sum_b d_b(2 nu_t S_ab);
S_aa at the pressure points, S_ab (a != b) at the edge midpoints; nu_t at the pressure
points from the velocity gradient A interpolated there; nu_t back on the edges by a
four-point average; the invariants Q_S, R_S, ...; the Smagorinsky, Vreman, QR and WALE
formulas) and Sec. 6.3 (model constants C_S = 0.1, C_W = 0.5, C_Q = sqrt(3/2)/pi,
C_V = sqrt(2.5 C_S^2), filter width (dx dy dz)^(1/3)).

Readings taken where the paper is silent or its printed formula conflicts with its text:

* Sign: the closure term added to F is the eddy-viscous stress divergence
  e^a = + sum_b delta_b(2 nu_t S_ab), i.e. the paper's m enters the momentum equation
  with a minus sign, so the models dissipate energy.
* Staggered derivatives: A_ab = delta_b u^a. Diagonal at cell I: (u^a_I - u^a_{I-e_a}) / d_a.
  Off-diagonal at the (a, b) edge of cell I (face a of I, face b of I):
  E_ab(I) = (u^a_{I+e_b} - u^a_I) / h_b; S_ab = (E_ab + E_ba) / 2 there.
* A at the pressure point: the mean of the four E_ab around the cell (edges I, I - e_a,
  I - e_b, I - e_a - e_b); the cell centre is the midpoint of its faces, so this is the
  linear interpolation. nu_t on the (a, b) edge of I: the mean of nu_t at I, I + e_a,
  I + e_b, I + e_a + e_b (the paper's four-point average).
* WALE: S^d is taken as the traceless symmetric part of A A, as the text defines it:
  S^d = (A A + (A A)^T) / 2 - tr(A A) / 3 I (the printed "-(Q_A / 3) I" is not traceless).
* Vreman: as printed, nu_t = C^2 sqrt(B_beta / (tr(A A^T) / 2)) with
  beta_ij = sum_m D_m^2 A_im A_jm (D_m the cell widths); 0 where A = 0.
* QR: nu_t = -(C D)^2 |R_S| / Q_S, 0 where Q_S = 0.
* Walls (y): the velocity ghosts of ``operators`` (odd tangential, zero wall-normal); nu_t takes
  the even ghost (the mirrored cell's value) where an edge average reaches across a wall. The
  stored top wall face of u^y is not an unknown (no term there).
* Filter width D = (d_x d_y d_z)^(1/3) per cell (d_x d_y in 2-D: D = sqrt).

Parity: pinned by tests/test_oracle_eddy.py (a constant eddy viscosity reduces the
operator to nu (diffusion + G D) on periodic and channel grids, closed forms of every model
on pure shear, solid rotation, axisymmetric and two-component strain, the dissipation
identity, second-order convergence of the interpolated gradient, and on a channel the
closed-form flux difference of a wall shear flow with a row-dependent nu_t (the wall rules
of the velocity and of nu_t)).
"""

import numpy as np

from .grid import PERIODIC
from . import operators as op
from .operators import NORMAL, TANGENT, EVEN

SMAGORINSKY = "smagorinsky"
WALE = "wale"
QR = "qr"
VREMAN = "vreman"
CONSTANT = "constant"      # nu_t = C everywhere (test model for the operator pin)

DEFAULT_C = {
    SMAGORINSKY: 0.1,
    WALE: 0.5,
    QR: np.sqrt(1.5) / np.pi,
    VREMAN: np.sqrt(2.5 * 0.1 ** 2),
}


def _check(g):
    for a in range(g.dim):
        assert g.bc[a] == PERIODIC or a == 1, "walls are supported in y only"


def _sh(g, f, a, s, kind=TANGENT):
    """f at I + s e_a with the boundary rule of ``operators.shift`` (kind at a wall)."""
    return op.shift(g, f, a, s, kind)


def _along(g, v, a):
    return g.along(v, a)


def _h_prev(g, a):
    return op.h_prev(g, a)


def diag_strain(g, u, a):
    """S_aa = A_aa at the cell centres (u^a below a bottom wall is the wall value 0)."""
    return (u[a] - _sh(g, u[a], a, -1, NORMAL)) / _along(g, g.d[a], a)


def edge_grad(g, u, a, b):
    """E_ab(I) = delta_b u^a on the (a, b) edge of cell I: (u^a_{I+e_b} - u^a_I) / h_b
    (odd ghost of a tangential velocity above a top wall)."""
    return (_sh(g, u[a], b, +1, TANGENT) - u[a]) / _along(g, g.h[b], b)


def edge_grad_lower(g, u, a, b):
    """E_ab(I - e_b): (u^a_I - u^a_{I-e_b}) / h_b[i-1] (odd ghost below a bottom wall)."""
    return (u[a] - _sh(g, u[a], b, -1, TANGENT)) / _along(g, _h_prev(g, b), b)


def gradient_at_centres(g, u):
    """A_ab at the pressure points, array of shape (dim, dim) + grid shape."""
    _check(g)
    A = np.zeros((g.dim, g.dim) + g.shape)
    for a in range(g.dim):
        A[a, a] = diag_strain(g, u, a)
        for b in range(g.dim):
            if b == a:
                continue
            E = edge_grad(g, u, a, b)               # edge (I; a, b)
            El = edge_grad_lower(g, u, a, b)        # edge (I - e_b)
            # edges (I - e_a) and (I - e_a - e_b): shift along a; below a wall in a the
            # edge of u^a's lower neighbour carries the wall velocity 0 (NORMAL rule)
            A[a, b] = 0.25 * (E + El + _sh(g, E, a, -1, NORMAL) + _sh(g, El, a, -1, NORMAL))
    return A


def filter_width(g):
    """D = (prod_a d_a)^(1/dim) at every cell."""
    vol = np.ones(g.shape)
    for a in range(g.dim):
        vol = vol * _along(g, g.d[a], a)
    return vol ** (1.0 / g.dim)


def nu_t_pointwise(model, A, D, C, widths=None):
    """Eddy viscosity of one velocity gradient A (dim x dim) with filter width D.

    widths: the cell widths (d_1 .. d_dim) for Vreman's beta tensor.
    """
    A = np.asarray(A, dtype=np.float64)
    dim = A.shape[0]
    S = 0.5 * (A + A.T)
    if model == CONSTANT:
        return C
    if model == SMAGORINSKY:
        return (C * D) ** 2 * np.sqrt(2.0 * np.sum(S * S))
    if model == WALE:
        A2 = A @ A
        Sd = 0.5 * (A2 + A2.T) - np.trace(A2) / 3.0 * np.eye(dim)
        sd = np.sum(Sd * Sd)
        ss = np.sum(S * S)
        den = ss ** 2.5 + sd ** 1.25
        return 0.0 if den == 0.0 else (C * D) ** 2 * sd ** 1.5 / den
    if model == QR:
        QS = -0.5 * np.trace(S @ S)
        RS = np.trace(S @ S @ S) / 3.0
        return 0.0 if QS == 0.0 else -(C * D) ** 2 * abs(RS) / QS
    if model == VREMAN:
        w = np.asarray(widths, dtype=np.float64)
        beta = (A * w[None, :] ** 2) @ A.T        # beta_ij = sum_m w_m^2 A_im A_jm
        B = 0.0
        for i in range(dim):
            for j in range(i + 1, dim):
                B += beta[i, i] * beta[j, j] - beta[i, j] ** 2
        den = 0.5 * np.sum(A * A)
        return 0.0 if den == 0.0 else C ** 2 * np.sqrt(max(B, 0.0) / den)
    raise ValueError(model)


def eddy_viscosity(g, u, model, C=None):
    """nu_t at every pressure point (plain loop over cells of the pointwise formula)."""
    _check(g)
    C = DEFAULT_C.get(model, 0.0) if C is None else C
    A = gradient_at_centres(g, u)
    D = filter_width(g)
    out = np.zeros(g.shape)
    for idx in np.ndindex(*g.shape):
        Ai = A[(slice(None), slice(None)) + idx]
        widths = [g.d[a][idx[g.axis(a)]] for a in range(g.dim)]
        out[idx] = nu_t_pointwise(model, Ai, D[idx], C, widths)
    return out


def stress_divergence(g, u, nu_t):
    """e^a = sum_b delta_b (2 nu_t S_ab) on the a-faces, for a given nu_t at the cells.

    Across a wall nu_t takes the even ghost (the mirrored cell's value); the strain on a wall
    edge uses the odd ghost of the tangential velocity and the zero wall-normal velocity."""
    _check(g)
    e = g.zeros_u()

    def nsh(f, b, s):
        return op.shift(g, f, b, s, EVEN)

    for a in range(g.dim):
        Taa = 2.0 * nu_t * diag_strain(g, u, a)
        e[a] += (nsh(Taa, a, +1) - Taa) / _along(g, g.h[a], a)
        for b in range(g.dim):
            if b == a:
                continue
            nu_up = 0.25 * (nu_t + nsh(nu_t, a, +1) + nsh(nu_t, b, +1) + nsh(nsh(nu_t, a, +1), b, +1))
            nu_lo = 0.25 * (nsh(nu_t, b, -1) + nsh(nsh(nu_t, a, +1), b, -1) + nu_t + nsh(nu_t, a, +1))
            S_up = 0.5 * (edge_grad(g, u, a, b) + edge_grad(g, u, b, a))
            # lower edge (I - e_b): E_ab from the odd ghost, E_ba at I - e_b (zero below a wall in b)
            S_lo = 0.5 * (edge_grad_lower(g, u, a, b) + _sh(g, edge_grad(g, u, b, a), b, -1, NORMAL))
            e[a] += (2.0 * nu_up * S_up - 2.0 * nu_lo * S_lo) / _along(g, g.d[b], b)
        e[a] *= g.face_mask(a)
    return e


def closure_term(g, u, model, C=None):
    """The term added to F: stress_divergence with the model's nu_t."""
    return stress_divergence(g, u, eddy_viscosity(g, u, model, C))


def closure(g, model, C=None):
    """Callable u -> term, for operators.rhs_F / timestep.rk4_step."""
    return lambda u: closure_term(g, u, model, C)
