"""Pullbacks (vector-Jacobian products) of the operators and of one RK step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Sec. 3.4 (pullback definition, eq. S:pullback: ubar_J = <phibar, d phi / d u_J>;
linear operators pull back through their transpose; the Poisson solve is
self-adjoint so its pullback is again a Poisson solve), App. B (pullback
kernels of divergence, pressure gradient, diffusion, convection).

Scope: periodic directions (any spacing) for the operator transposes; the
step VJP additionally needs a uniform grid, where the projection P = I - G L^-1 D
is symmetric in the plain Euclidean inner product over the storage index.

Every transpose is written with the transpose of the shift, (S+)^T = S-,
so it reads as the term-by-term transpose of ``oracle.operators``. The
convection pullback is the transpose of the bilinear form B(adv, tra) in both
arguments; its sum over the two arguments at adv = tra = u is the pullback of
C(u) = B(u, u) (the eight contributions listed in App. B).
"""

import numpy as np

from .grid import PERIODIC
from . import operators as op
from . import poisson
from .timestep import RK4_A, RK4_B, WRAY3_A, WRAY3_B


def _check_periodic(g):
    for a in range(g.dim):
        assert g.bc[a] == PERIODIC, "adjoints are implemented for periodic directions"


def _sp(g, f, a):
    """S+ along a (periodic)."""
    return np.roll(f, -1, axis=g.axis(a))


def _sm(g, f, a):
    """S- along a (periodic)."""
    return np.roll(f, +1, axis=g.axis(a))


def divergence_T(g, phibar):
    """D^T: ubar^a = phibar/d_a[i] - phibar_{I+e_a}/d_a[i+1]   (App. B divergence pullback)."""
    _check_periodic(g)
    out = g.zeros_u()
    for a in range(g.dim):
        z = phibar / g.along(g.d[a], a)
        out[a] = z - _sp(g, z, a)
    return out


def gradient_T(g, phibar):
    """G^T: pbar = sum_a phibar^a_{I-e_a}/h_a[i-1] - phibar^a_I/h_a[i]   (App. B)."""
    _check_periodic(g)
    out = g.zeros_p()
    for a in range(g.dim):
        z = phibar[a] / g.along(g.h[a], a)
        out += _sm(g, z, a) - z
    return out


def _diff_coeffs(g, a, b):
    """(c+, c-) of the 1-D second difference of u^a along b: c+ S+u + c- S-u - (c+ + c-) u."""
    if a == b:
        cp = 1.0 / (op.d_next(g, a) * g.h[a])
        cm = 1.0 / (g.d[a] * g.h[a])
    else:
        cp = 1.0 / (g.h[b] * g.d[b])
        cm = 1.0 / (op.h_prev(g, b) * g.d[b])
    return g.along(cp, b), g.along(cm, b)


def diffusion_T(g, phibar):
    """Transpose of ``operators.diffusion`` (without nu)   (App. B diffusion pullback)."""
    _check_periodic(g)
    out = g.zeros_u()
    for a in range(g.dim):
        z = phibar[a]
        for b in range(g.dim):
            cp, cm = _diff_coeffs(g, a, b)
            out[a] += _sm(g, cp * z, b) + _sp(g, cm * z, b) - (cp + cm) * z
    return out


def convection_bilinear_T(g, adv, tra, w):
    """Gradients of <w, B(adv, tra)> with respect to adv and to tra.

    Returns (advbar, trabar). Mirrors ``operators.convection_bilinear`` term by term:
    a term -sum z * X(adv) * Y(tra) gives advbar += -X^T(z Y) and trabar += -Y^T(z X).
    """
    _check_periodic(g)
    advbar = g.zeros_u()
    trabar = g.zeros_u()
    for a in range(g.dim):
        ta = tra[a]
        for b in range(g.dim):
            if b == a:
                aa = adv[a]
                z = w[a] / g.along(g.h[a], a)
                vp = 0.5 * (aa + _sp(g, aa, a))
                vm = 0.5 * (_sm(g, aa, a) + aa)
                tp = 0.5 * (ta + _sp(g, ta, a))
                tm = 0.5 * (_sm(g, ta, a) + ta)
                # avg+ (x) = (x + S+x)/2  ->  avg+^T (y) = (y + S-y)/2 ; avg- likewise with S+
                advbar[a] += -0.5 * (z * tp + _sm(g, z * tp, a)) + 0.5 * (z * tm + _sp(g, z * tm, a))
                trabar[a] += -0.5 * (z * vp + _sm(g, z * vp, a)) + 0.5 * (z * vm + _sp(g, z * vm, a))
            else:
                ab = adv[b]
                wl, wr = op.interp_weights(g, a)
                wl = g.along(wl, a)
                wr = g.along(wr, a)
                z = w[a] / g.along(g.d[b], b)
                vp = wl * ab + wr * _sp(g, ab, a)
                vm = _sm(g, vp, b)
                tp = 0.5 * (ta + _sp(g, ta, b))
                tm = 0.5 * (_sm(g, ta, b) + ta)
                # vp = I(ab) with I(x) = wl x + wr S+_a x  ->  I^T(y) = wl y + S-_a(wr y)
                # vm = S-_b I(ab)                          ->  (S-_b I)^T(y) = I^T(S+_b y)
                y1 = z * tp
                y2 = _sp(g, z * tm, b)
                advbar[b] += -(wl * y1 + _sm(g, wr * y1, a)) + (wl * y2 + _sm(g, wr * y2, a))
                trabar[a] += -0.5 * (z * vp + _sm(g, z * vp, b)) + 0.5 * (z * vm + _sp(g, z * vm, b))
    return advbar, trabar


def convection_vjp(g, u, w):
    """Pullback of C(u) = B(u, u): ubar = (dC/du)^T w."""
    ab, tb = convection_bilinear_T(g, u, u, w)
    return ab + tb


def F_vjp(g, u, w, closure=None):
    """Pullback of F(u) = C(u) + nu diffusion(u) + f (+ m(u)), and d<w,F>/dnu = <w, diffusion(u)>.

    With a closure (``oracle.closure.Closure``) also returns its per-layer (dW, db)."""
    ubar = convection_vjp(g, u, w) + g.nu * diffusion_T(g, w)
    nubar = float(np.sum(w * op.diffusion(g, u)))
    if closure is None:
        return ubar, nubar
    from . import closure as cl
    cu, grads = cl.backward(closure.params, u, w, closure.quantize)
    return ubar + cu, nubar, grads


def project_T(g, kbar):
    """P^T = P on periodic uniform grids (the Poisson solve is self-adjoint, Sec. 2.6.1)."""
    for a in range(g.dim):
        assert g.is_uniform(a), "P is symmetric only on uniform periodic grids"
    w, _ = poisson.project(g, kbar)
    return w


def rk4_step_vjp(g, u0, dt, ybar, closure=None):
    """Pullback of one RK4 step u0 -> u1 (dt frozen): returns (u0bar, nubar), and with a
    closure also the closure's per-layer (dW, db) summed over the four stages.

    Forward (``timestep.rk4_step``): k_s = P F(u_s), u_s = u0 + dt a_{s,s-1} k_{s-1},
    u1 = u0 + dt sum_s b_s k_s. Reverse: kbar_s = dt b_s ybar + dt a_{s+1,s} ubar_{s+1},
    w_s = P^T kbar_s, ubar_s = J_F(u_s)^T w_s, u0bar = ybar + sum_s ubar_s,
    nubar = sum_s <w_s, diffusion(u_s)>.
    """
    _check_periodic(g)
    # recompute the stage states from the checkpoint u0
    us = [u0]
    for s in range(3):
        from .timestep import stage_derivative
        k = stage_derivative(g, us[s], closure)
        us.append(u0 + dt * RK4_A[s + 1] * k)
    u0bar = ybar.copy()
    nubar = 0.0
    wgrads = None
    kbar = [dt * RK4_B[s] * ybar for s in range(4)]
    for s in range(3, -1, -1):
        w = project_T(g, kbar[s])
        if closure is None:
            ubar_s, nb = F_vjp(g, us[s], w)
        else:
            ubar_s, nb, gr = F_vjp(g, us[s], w, closure)
            wgrads = gr if wgrads is None else [(a[0] + b[0], a[1] + b[1]) for a, b in zip(wgrads, gr)]
        nubar += nb
        u0bar = u0bar + ubar_s
        if s > 0:
            kbar[s - 1] = kbar[s - 1] + dt * RK4_A[s] * ubar_s
    if closure is not None:
        return u0bar, nubar, wgrads
    return u0bar, nubar


def erk_step_vjp(g, u0, dt, ybar, A, b):
    """Pullback of one explicit RK step in Butcher form (``timestep.erk_step``), dt frozen:
    returns (u0bar, nubar).

    Forward: u_s = u0 + dt sum_{t<s} a_{s,t} k_t, k_s = P F(u_s), u1 = u0 + dt sum_s b_s k_s.
    Reverse (s from the last stage down): kbar_s = dt b_s ybar + dt sum_{r>s} a_{r,s} ubar_r,
    w_s = P^T kbar_s, ubar_s = J_F(u_s)^T w_s, u0bar = ybar + sum_s ubar_s,
    nubar = sum_s <w_s, diffusion(u_s)>.
    """
    from .timestep import stage_derivative
    _check_periodic(g)
    ns = len(b)
    us, ks = [], []
    for s in range(ns):
        x = u0.copy()
        for t, a in enumerate(A[s]):
            x = x + dt * a * ks[t]
        us.append(x)
        ks.append(stage_derivative(g, x))
    kbar = [dt * b[s] * ybar for s in range(ns)]
    u0bar = ybar.copy()
    nubar = 0.0
    for s in range(ns - 1, -1, -1):
        w = project_T(g, kbar[s])
        ubar_s, nb = F_vjp(g, us[s], w)
        nubar += nb
        u0bar = u0bar + ubar_s
        for t, a in enumerate(A[s]):
            kbar[t] = kbar[t] + dt * a * ubar_s
    return u0bar, nubar


def wray3_step_vjp(g, u0, dt, ybar):
    """Pullback of one step of Wray's scheme (``timestep.wray3_step``)."""
    return erk_step_vjp(g, u0, dt, ybar, WRAY3_A, WRAY3_B)
