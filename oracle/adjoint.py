"""Pullbacks (vector-Jacobian products) of the operators and of one RK step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Sec. 3.4 (pullback definition, eq. S:pullback: ubar_J = <phibar, d phi / d u_J>;
linear operators pull back through their transpose; the Poisson solve is
self-adjoint so its pullback is again a Poisson solve), App. B (pullback
kernels of divergence, pressure gradient, diffusion, convection), Sec. 2.6.1
(with volume matrices, L^T = Omega_p L Omega_p^-1 on non-uniform grids).

Scope: periodic directions (any spacing) and no-slip wall directions.

Every transpose is written with the transpose of the boundary-aware shift of
``oracle.operators`` (``shift_T``): in a periodic direction (S+)^T = S-; at a wall
the ghost rule of the forward shift (0, odd or even reflection of the first or
last stored value) becomes an extra diagonal term at that stored index. So each
transpose reads as the term-by-term transpose of ``oracle.operators``. The
convection pullback is the transpose of the bilinear form B(adv, tra) in both
arguments; its sum over the two arguments at adv = tra = u is the pullback of
C(u) = B(u, u) (the eight contributions listed in App. B).

Wall faces that are stored but are not unknowns (the top face of a wall direction,
``Grid.face_mask``) are not degrees of freedom: the pullbacks take cotangents there as
zero and return zero there.

Reading for the projection pullback: with the face volumes Omega_u, D = Omega_p^-1 Dh and
G = -Omega_u^-1 Dh^T on the unknowns (Dh the face-area divergence), so P^T = Omega_u P
Omega_u^-1; on a uniform periodic grid this is P itself.
"""

import numpy as np

from .grid import PERIODIC
from . import operators as op
from .operators import NORMAL, TANGENT, EVEN
from . import poisson
from .timestep import RK4_A, RK4_B, WRAY3_A, WRAY3_B


def shift_T(g, y, a, s, kind):
    """Transpose of f -> operators.shift(g, f, a, s, kind)."""
    ax = g.axis(a)
    out = np.roll(y, s, axis=ax)
    if g.bc[a] == PERIODIC:
        return out
    n = g.n[a]
    idx = [slice(None)] * g.dim
    if s == +1:
        # shift(+1)[i] = f[i+1] for i < n-1; row n-1 holds the ghost rule in f[n-1]
        idx[ax] = 0
        out[tuple(idx)] = 0.0                     # nothing maps onto f[0]
        last = [slice(None)] * g.dim
        last[ax] = n - 1
        if kind == TANGENT:
            out[tuple(last)] -= y[tuple(last)]
        elif kind == EVEN:
            out[tuple(last)] += y[tuple(last)]
    elif s == -1:
        idx[ax] = n - 1
        out[tuple(idx)] = 0.0                     # nothing maps onto f[n-1]
        first = [slice(None)] * g.dim
        first[ax] = 0
        if kind == TANGENT:
            out[tuple(first)] -= y[tuple(first)]
        elif kind == EVEN:
            out[tuple(first)] += y[tuple(first)]
    else:
        raise ValueError("shift by +1 or -1 only")
    return out


def mask_u(g, v):
    """Zero the stored wall faces that are not unknowns."""
    out = np.array(v, dtype=np.float64, copy=True)
    for a in range(g.dim):
        out[a] = out[a] * g.face_mask(a)
    return out


def divergence_T(g, phibar):
    """D^T: ubar^a = z - S-^T z with z = phibar / d_a   (App. B divergence pullback)."""
    out = g.zeros_u()
    for a in range(g.dim):
        z = phibar / g.along(g.d[a], a)
        out[a] = z - shift_T(g, z, a, -1, NORMAL)
    return out


def gradient_T(g, phibar):
    """G^T: pbar = sum_a S+^T z - z with z = mask phibar^a / h_a   (App. B)."""
    out = g.zeros_p()
    for a in range(g.dim):
        z = phibar[a] * g.face_mask(a) / g.along(g.h[a], a)
        out += shift_T(g, z, a, +1, EVEN) - z
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
    out = g.zeros_u()
    for a in range(g.dim):
        z = phibar[a] * g.face_mask(a)
        for b in range(g.dim):
            kind = NORMAL if b == a else TANGENT
            cp, cm = _diff_coeffs(g, a, b)
            out[a] += shift_T(g, cp * z, b, +1, kind) + shift_T(g, cm * z, b, -1, kind) - (cp + cm) * z
    return out


def convection_bilinear_T(g, adv, tra, w):
    """Gradients of <w, B(adv, tra)> with respect to adv and to tra.

    Returns (advbar, trabar). Mirrors ``operators.convection_bilinear`` term by term:
    a term -sum z * X(adv) * Y(tra) gives advbar += -X^T(z Y) and trabar += -Y^T(z X).
    """
    advbar = g.zeros_u()
    trabar = g.zeros_u()

    def sh(f, a, s, kind):
        return op.shift(g, f, a, s, kind)

    def shT(y, a, s, kind):
        return shift_T(g, y, a, s, kind)

    for a in range(g.dim):
        ta = tra[a]
        wa = w[a] * g.face_mask(a)
        for b in range(g.dim):
            if b == a:
                aa = adv[a]
                z = wa / g.along(g.h[a], a)
                vp = 0.5 * (aa + sh(aa, a, +1, NORMAL))
                vm = 0.5 * (sh(aa, a, -1, NORMAL) + aa)
                tp = 0.5 * (ta + sh(ta, a, +1, NORMAL))
                tm = 0.5 * (sh(ta, a, -1, NORMAL) + ta)
                # avg+ (x) = (x + S+x)/2  ->  avg+^T (y) = (y + S+^T y)/2 ; avg- likewise with S-^T
                advbar[a] += -0.5 * (z * tp + shT(z * tp, a, +1, NORMAL)) + 0.5 * (z * tm + shT(z * tm, a, -1, NORMAL))
                trabar[a] += -0.5 * (z * vp + shT(z * vp, a, +1, NORMAL)) + 0.5 * (z * vm + shT(z * vm, a, -1, NORMAL))
            else:
                ab = adv[b]
                wl, wr = op.interp_weights(g, a)
                wl = g.along(wl, a)
                wr = g.along(wr, a)
                z = wa / g.along(g.d[b], b)
                vp = wl * ab + wr * sh(ab, a, +1, TANGENT)
                vm = sh(vp, b, -1, NORMAL)
                tp = 0.5 * (ta + sh(ta, b, +1, TANGENT))
                tm = 0.5 * (sh(ta, b, -1, TANGENT) + ta)
                # vp = I(ab) with I(x) = wl x + wr S+_a x  ->  I^T(y) = wl y + S+_a^T(wr y)
                # vm = S-_b I(ab)                          ->  (S-_b I)^T(y) = I^T(S-_b^T y)
                y1 = z * tp
                y2 = shT(z * tm, b, -1, NORMAL)
                advbar[b] += -(wl * y1 + shT(wr * y1, a, +1, TANGENT)) + (wl * y2 + shT(wr * y2, a, +1, TANGENT))
                trabar[a] += (-0.5 * (z * vp + shT(z * vp, b, +1, TANGENT))
                              + 0.5 * (z * vm + shT(z * vm, b, -1, TANGENT)))
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


def _face_volumes(g):
    """Omega_u^a without the wall mask (positive everywhere)."""
    out = g.zeros_u()
    for a in range(g.dim):
        v = np.ones(g.shape) * g.along(g.h[a], a)
        for b in range(g.dim):
            if b != a:
                v = v * g.along(g.d[b], b)
        out[a] = v
    return out


def project_T(g, kbar):
    """P^T = M Omega_u P Omega_u^-1 M (M the mask of the unknowns; reading in the module docstring).
    On a uniform periodic grid Omega_u is constant and P^T = P (Sec. 2.6.1)."""
    vol = _face_volumes(g)
    w, _ = poisson.project(g, mask_u(g, kbar) / vol)
    return mask_u(g, vol * w)


def rk4_step_vjp(g, u0, dt, ybar, closure=None):
    """Pullback of one RK4 step u0 -> u1 (dt frozen): returns (u0bar, nubar), and with a
    closure also the closure's per-layer (dW, db) summed over the four stages.

    Forward (``timestep.rk4_step``): k_s = P F(u_s), u_s = u0 + dt a_{s,s-1} k_{s-1},
    u1 = u0 + dt sum_s b_s k_s. Reverse: kbar_s = dt b_s ybar + dt a_{s+1,s} ubar_{s+1},
    w_s = P^T kbar_s, ubar_s = J_F(u_s)^T w_s, u0bar = ybar + sum_s ubar_s,
    nubar = sum_s <w_s, diffusion(u_s)>. ybar and u0bar are masked to the unknowns.
    """
    ybar = mask_u(g, ybar)
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
    u0bar = mask_u(g, u0bar)
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
    ybar = mask_u(g, ybar)
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
    return mask_u(g, u0bar), nubar


def wray3_step_vjp(g, u0, dt, ybar):
    """Pullback of one step of Wray's scheme (``timestep.wray3_step``)."""
    return erk_step_vjp(g, u0, dt, ybar, WRAY3_A, WRAY3_B)
