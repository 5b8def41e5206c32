"""torch.autograd over ins_step: differentiable steps with per-step checkpointing.

The step is the grid's scheme (classic RK4 or Wray's low-storage RK3). Each step saves only
its input u_n; the backward pass (ins_step_vjp) recomputes the stage states from it and runs
the hand-written pullback kernels, so an unroll of T steps keeps T velocity fields plus one
step's stage states. The time step dt is
treated as a constant. The viscosity enters as a tensor so that dL/dnu is returned;
its value must equal the grid's nu (the grid's coefficients are built from it).
"""

import torch


class _SolverStep(torch.autograd.Function):
    """One ins_step of the grid's scheme; backward is ins_step_vjp."""

    @staticmethod
    def forward(ctx, u, nu, grid, dt):
        ctx.grid = grid
        ctx.dt = dt
        ctx.save_for_backward(u)
        out = u.detach().clone()
        grid.step(out, dt=dt)
        return out

    @staticmethod
    def backward(ctx, gout):
        (u,) = ctx.saved_tensors
        ubar, nubar = ctx.grid.step_vjp(u.detach(), gout.contiguous(), dt=ctx.dt)
        return ubar, nubar.reshape(()), None, None


def _nu_tensor(u, grid, nu):
    """nu as a float64 tensor, checked against the grid's viscosity (one host read)."""
    if nu is None:
        return torch.tensor(grid.nu, dtype=torch.float64, device=u.device)
    if abs(float(nu.detach()) - grid.nu) > 1e-15 * max(1.0, abs(grid.nu)):
        raise ValueError("nu must equal the grid's viscosity (create a new grid to change it)")
    return nu


def step(u, grid, dt, nu=None):
    """One differentiable step of the grid's scheme: u_{n+1} = step(u_n); gradients flow to u and nu."""
    return _SolverStep.apply(u, _nu_tensor(u, grid, nu), grid, float(dt))


def rollout(u0, grid, dt, nsteps, nu=None):
    """nsteps differentiable steps; returns the list of states u_1 .. u_nsteps. nu is checked
    once (its host read waits for the device), not at every step."""
    nu = _nu_tensor(u0, grid, nu)
    out = []
    u = u0
    for _ in range(nsteps):
        u = _SolverStep.apply(u, nu, grid, float(dt))
        out.append(u)
    return out
