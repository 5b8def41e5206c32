"""Explicit Runge-Kutta time step with a projection at every stage (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Sec. 2.6.2 (explicit RK, the pressure Poisson equation solved at every
sub-step so every stage is divergence free and the RK order is kept; adaptive
time step from convective and diffusive limits).

Readings taken where the paper is silent:

* Scheme: the classic 4-stage RK (tableau a21 = a32 = 1/2, a43 = 1,
  b = (1/6, 1/3, 1/3, 1/6)). Each stage derivative is the projected right-hand
  side k_s = F(u_s) - G p_s with L p_s = D F(u_s); the stage states are
  u_s = u_0 + dt a_{s,s-1} k_{s-1}. Because u_0 and every k_s are divergence
  free, this equals projecting the stage velocities.
* Low-storage scheme: the paper lists Wray3 among its explicit RK methods and as its
  low-storage method (Sec. 2.6.2, Sec. 3.3) without printing it. Reading: Wray's
  third-order three-stage scheme, Butcher tableau a21 = 8/15, a31 = 1/4, a32 = 5/12,
  b = (1/4, 0, 3/4), c = (0, 8/15, 2/3), with the same projected stage derivatives.
  The oracle evaluates it in plain Butcher form (``erk_step``), not in the two-register
  form a low-storage implementation uses.
* CFL rule (the paper gives no formula):
  dt = cfl * min( 1 / max_{a,I} |u^a_I| / h_a[i],  min_{a,i} d_a[i]^2 / nu ).
  Every operation is one IEEE-rounded FP64 operation (abs, divide, max, min,
  multiply), so an implementation that performs the same operations gets the
  same bits regardless of the order of the max reduction.
"""

import numpy as np

from . import operators as op
from . import poisson

RK4_A = (None, 0.5, 0.5, 1.0)      # a_{s+1,s} for s = 1, 2, 3 (index s)
RK4_B = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)


def stage_derivative(g, u, closure=None):
    """k = F(u) - G p, L p = D F(u)."""
    k, _ = poisson.rhs(g, u, closure)
    return k


def rk4_step(g, u0, dt, closure=None, return_stages=False):
    """One classic RK4 step with per-stage projection."""
    us = u0
    acc = np.zeros_like(u0)
    stages = []
    for s in range(4):
        k = stage_derivative(g, us, closure)
        stages.append((us, k))
        acc = acc + RK4_B[s] * k
        if s < 3:
            us = u0 + dt * RK4_A[s + 1] * k
    u1 = u0 + dt * acc
    if return_stages:
        return u1, stages
    return u1


WRAY3_A = ((), (8.0 / 15.0,), (1.0 / 4.0, 5.0 / 12.0))   # row s: a_{s,t}, t < s
WRAY3_B = (1.0 / 4.0, 0.0, 3.0 / 4.0)


def erk_step(g, u0, dt, A, b, closure=None):
    """One explicit RK step in Butcher form with projected stage derivatives:
    u_s = u0 + dt sum_{t<s} a_{s,t} k_t, k_s = P F(u_s), u1 = u0 + dt sum_s b_s k_s."""
    ks = []
    for s in range(len(b)):
        us = u0.copy()
        for t, a in enumerate(A[s]):
            us = us + dt * a * ks[t]
        ks.append(stage_derivative(g, us, closure))
    u1 = u0.copy()
    for s, bs in enumerate(b):
        u1 = u1 + dt * bs * ks[s]
    return u1


def wray3_step(g, u0, dt, closure=None):
    """One step of Wray's low-storage third-order scheme (tableau in the module docstring)."""
    return erk_step(g, u0, dt, WRAY3_A, WRAY3_B, closure)


def max_u_over_h(g, u):
    """max_{a,I} |u^a_I| / h_a[i] in FP64 (wall faces hold 0 and do not contribute)."""
    m = 0.0
    for a in range(g.dim):
        q = np.abs(np.asarray(u[a], dtype=np.float64)) / g.along(g.h[a], a)
        m = max(m, float(np.max(q)))
    return m


def cfl_dt(g, u, cfl):
    """Adaptive time step (reading stated in the module docstring)."""
    m = max_u_over_h(g, u)
    conv = np.inf if m == 0.0 else 1.0 / m
    dmin = min(float(np.min(g.d[a])) for a in range(g.dim))
    diff = np.inf if g.nu == 0.0 else (dmin * dmin) / g.nu
    return cfl * min(conv, diff)


def integrate(g, u0, dt, nsteps, closure=None, scheme="rk4"):
    """nsteps fixed-dt steps of the classic RK4 ("rk4") or Wray's scheme ("wray3")."""
    step = {"rk4": rk4_step, "wray3": wray3_step}[scheme]
    u = u0
    for _ in range(nsteps):
        u = step(g, u, dt, closure)
    return u
