"""A-posteriori training of the CNN closure on filtered DNS (the learned LES closure).

Pipeline (every solver operation runs in libins; torch only holds tensors, forms the
trajectory loss and applies Adam to the parameter tensors):

1. DNS data: for each seed, a decaying-turbulence DNS on an n_dns^3 periodic grid
   (random Fourier initial field with E(k) ~ k^4 exp(-2 (k/k0)^2), projected, unit
   energy), a spin-up, then snapshots every LES time step, each reduced to the LES grid
   with the face-averaging filter. The LES step dt is fixed by the CFL rule on the
   filtered initial field; the DNS takes m equal sub-steps per LES step (m from the DNS
   CFL), landing exactly on the snapshots.
2. Training: batches of trajectories; each runs `nsteps` LES steps with the closure in F
   from the filtered initial field; loss = (1/nsteps) sum_n |u_n - ubar_n|^2 / |ubar_n|^2;
   the gradient flows back through every step with ins_step_vjp (which recomputes the
   stages from the step input and accumulates the closure's weight gradients).
3. Evaluation: spectrum error at the last snapshot, relative L2 distance of log E(k) over
   k = 1 .. n_les/2 - 1, against the filtered DNS, with and without the closure. If the
   closure produces a non-finite field the no-closure LES is used (fallback).
4. Paired evaluation (evaluate_paired): the same errors per held-out trajectory at several
   horizons, for the closure, the no-closure LES and the eddy-viscosity models, with the
   mean paired difference (no closure minus closure) and its standard error, so that a gain
   can be told apart from the spread between trajectories.

The trajectories can be longer than the training unroll: training then draws windows of
`nsteps` LES steps that start at every `stride`-th snapshot (training_windows), and the
final evaluation time is the end of the filtered DNS trajectory.
"""

import math

import torch

from . import inputs
from .closure import Closure, init_params
from .solver import Grid, filter_face_average
from ._lib import InsError


def _box(n, nu, dtype=torch.float32):
    return Grid(inputs.periodic_box(n, 3), ["periodic"] * 3, nu, dtype=dtype)


def dns_dataset(seeds, n_dns=256, n_les=64, nu=1.0 / 2000, k0=4.0, nsnap=10, spinup=100, cfl=0.3):
    """Filtered DNS trajectories: list of (snapshots (nsnap+1, 3, n, n, n) float32, dt_les)."""
    ratio = n_dns // n_les
    gd = _box(n_dns, nu)
    gl = _box(n_les, nu)
    out = []
    for seed in seeds:
        # the spectrum is below 1e-24 of its peak beyond 8 k0; only wavevectors up to there draw numbers
        u = torch.tensor(inputs.spectrum_velocity_raw(n_dns, 3, seed=int(seed), k0=k0, kmax=int(8 * k0)),
                         dtype=torch.float32, device="cuda")
        gd.project(u, out=u)
        u.mul_(1.0 / math.sqrt(gd.diag(u)["ke"]))
        dt = gd.cfl_dt(u, cfl)
        for _ in range(spinup):
            gd.step(u, dt_dev=dt, next_dt_dev=dt, cfl=cfl)
        ub = filter_face_average(u, ratio)
        dt_les = gl.cfl_dt(ub, cfl).item()
        m = max(1, math.ceil(dt_les / gd.cfl_dt(u, cfl).item()))
        dt_dns = dt_les / m
        snaps = [ub]
        for _ in range(nsnap):
            for _ in range(m):
                gd.step(u, dt=dt_dns)
            snaps.append(filter_face_average(u, ratio))
        gd.check_finite()
        out.append((torch.stack(snaps), dt_les))
    gd.close()
    gl.close()
    return out


class Adam:
    """Adam on a list of tensors (torch elementwise ops on the parameters)."""

    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.p = params
        self.m = [torch.zeros_like(t) for t in params]
        self.v = [torch.zeros_like(t) for t in params]
        self.lr, self.b1, self.b2, self.eps, self.t = lr, b1, b2, eps, 0

    def step(self, grads):
        self.t += 1
        for p, g, m, v in zip(self.p, grads, self.m, self.v):
            m.mul_(self.b1).add_(g, alpha=1 - self.b1)
            v.mul_(self.b2).addcmul_(g, g, value=1 - self.b2)
            mh = m / (1 - self.b1 ** self.t)
            vh = v / (1 - self.b2 ** self.t)
            p.sub_(self.lr * mh / (vh.sqrt() + self.eps))


def trajectory_loss_and_grad(grid, snaps, dt, nsteps):
    """Unrolled LES with the attached closure; returns the loss (closure gradients accumulate)."""
    u = snaps[0].clone()
    states = [u.clone()]
    for _ in range(nsteps):
        grid.step(u, dt=dt)
        states.append(u.clone())
    loss = 0.0
    ybar = torch.zeros_like(u)
    for n in range(nsteps, 0, -1):
        diff = states[n] - snaps[n]
        den = float((snaps[n] * snaps[n]).sum())
        loss += float((diff * diff).sum()) / den / nsteps
        ybar.add_(diff, alpha=2.0 / den / nsteps)
        ybar, _ = grid.step_vjp(states[n - 1], ybar, dt=dt)
    return loss


def train(data, n_les, nu, iters=100, batch=8, lr=1e-3, nsteps=10, seed=0, init_scale=0.1, log=None):
    """Train the closure on `data`; returns (W, b, loss history)."""
    g = _box(n_les, nu)
    W, b = init_params(seed, init_scale)
    c = Closure(g)
    c.set_params(W, b)
    g.set_closure(c)
    dW = [torch.zeros_like(w) for w in W]
    db = [torch.zeros_like(x) for x in b]
    c.set_grads(dW, db)
    opt = Adam(W + b, lr=lr)
    gen = torch.Generator().manual_seed(seed)
    hist = []
    for it in range(iters):
        for t in dW + db:
            t.zero_()
        idx = torch.randperm(len(data), generator=gen)[:batch].tolist()
        loss = 0.0
        for i in idx:
            snaps, dt = data[i]
            loss += trajectory_loss_and_grad(g, snaps, dt, nsteps) / len(idx)
        for t in dW + db:
            t.div_(len(idx))
        opt.step(dW + db)
        c.set_params(W, b)
        hist.append(loss)
        if log:
            log(it, loss)
    c.check()
    g.set_closure(None)
    c.close()
    g.close()
    return W, b, hist


def spectrum_error(grid, u, ref):
    """Relative L2 distance of log E(k), k = 1 .. N/2 - 1."""
    kmax = grid.n[0] // 2 - 1
    E = grid.spectrum(u, kmax)[1:]
    Er = grid.spectrum(ref, kmax)[1:]
    la, lb = torch.log(E), torch.log(Er)
    return float(torch.linalg.norm(la - lb) / torch.linalg.norm(lb))


def evaluate(data, n_les, nu, W=None, b=None, nsteps=10, eddy=None):
    """Mean spectrum error at step nsteps against the filtered DNS: with the CNN closure if W is
    given, with an eddy-viscosity model if eddy names one (paper constants), else without closure."""
    g = _box(n_les, nu)
    c = None
    if W is not None:
        c = Closure(g)
        c.set_params(W, b)
        g.set_closure(c)
    elif eddy is not None:
        g.set_eddy_viscosity(eddy)
    errs = []
    fallbacks = 0
    for snaps, dt in data:
        u = snaps[0].clone()
        for _ in range(nsteps):
            g.step(u, dt=dt)
        try:
            g.check_finite()
        except InsError:
            # no-closure fallback for this trajectory
            fallbacks += 1
            g.set_closure(None)
            g.set_eddy_viscosity(None)
            u = snaps[0].clone()
            for _ in range(nsteps):
                g.step(u, dt=dt)
            g.set_closure(c)
            if eddy is not None and c is None:
                g.set_eddy_viscosity(eddy)
        errs.append(spectrum_error(g, u, snaps[nsteps]))
    g.set_closure(None)
    if c is not None:
        c.close()
    g.close()
    return sum(errs) / len(errs), fallbacks


def training_windows(data, nsteps, stride):
    """Windows of nsteps + 1 snapshots starting at every stride-th snapshot of each trajectory."""
    out = []
    for snaps, dt in data:
        for k in range(0, snaps.shape[0] - nsteps, stride):
            out.append((snaps[k:k + nsteps + 1], dt))
    return out


def _errors(data, n_les, nu, horizon, W=None, b=None, eddy=None):
    """Spectrum error of each trajectory after `horizon` LES steps (closure W, b, an eddy model, or none)."""
    g = _box(n_les, nu)
    c = None
    if W is not None:
        c = Closure(g)
        c.set_params(W, b)
        g.set_closure(c)
    elif eddy is not None:
        g.set_eddy_viscosity(eddy)
    errs = []
    for snaps, dt in data:
        u = snaps[0].clone()
        for _ in range(horizon):
            g.step(u, dt=dt)
        g.check_finite()
        errs.append(spectrum_error(g, u, snaps[horizon]))
    g.set_closure(None)
    if c is not None:
        c.close()
    g.close()
    return errs


def paired(base, other):
    """Mean of base - other over trajectories, its standard error, and the count with base > other."""
    d = [x - y for x, y in zip(base, other)]
    n = len(d)
    m = sum(d) / n
    sd = math.sqrt(sum((x - m) ** 2 for x in d) / (n - 1)) if n > 1 else float("nan")
    return {"mean_diff": m, "se": sd / math.sqrt(n), "wins": sum(1 for x in d if x > 0), "n": n}


def evaluate_paired(data, n_les, nu, W, b, horizons, eddy=("smagorinsky", "wale")):
    """Per-trajectory spectrum errors at each horizon and paired comparisons against no closure."""
    out = {}
    for h in horizons:
        base = _errors(data, n_les, nu, h)
        cl = _errors(data, n_les, nu, h, W, b)
        rec = {"no_closure": base, "closure": cl, "no_closure_mean": sum(base) / len(base),
               "closure_mean": sum(cl) / len(cl), "closure_vs_no_closure": paired(base, cl)}
        for m in eddy:
            e = _errors(data, n_les, nu, h, eddy=m)
            rec[m + "_mean"] = sum(e) / len(e)
        out[h] = rec
    return out


def main():
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description="a-posteriori CNN closure training on filtered DNS")
    ap.add_argument("--n-dns", type=int, default=256)
    ap.add_argument("--n-les", type=int, default=64)
    ap.add_argument("--seeds", type=int, default=64)
    ap.add_argument("--test", type=int, default=16)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--nsteps", type=int, default=10)
    ap.add_argument("--spinup", type=int, default=100)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--nsnap", type=int, default=40, help="LES steps of each filtered DNS trajectory")
    ap.add_argument("--stride", type=int, default=5, help="start spacing of the training windows")
    a = ap.parse_args()
    nu = 1.0 / 2000
    t0 = time.time()
    data = dns_dataset(range(a.seeds), a.n_dns, a.n_les, nu, nsnap=a.nsnap, spinup=a.spinup)
    t1 = time.time()
    train_set, test_set = data[: a.seeds - a.test], data[a.seeds - a.test:]
    import sys

    def log(it, loss):
        if it % 10 == 0 or it == a.iters - 1:
            print(f"iter {it} loss {loss:.6e} t {time.time() - t1:.1f}s", file=sys.stderr, flush=True)

    windows = training_windows(train_set, a.nsteps, a.stride)
    W, b, hist = train(windows, a.n_les, nu, a.iters, a.batch, a.lr, a.nsteps, log=log)
    t2 = time.time()
    horizons = sorted({a.nsteps, a.nsnap // 2, a.nsnap})
    ev = evaluate_paired(test_set, a.n_les, nu, W, b, horizons)
    print(json.dumps({"final_horizon": a.nsnap, "evaluation": ev, "loss_first": hist[0], "loss_last": hist[-1],
                      "windows": len(windows), "dns_s": t1 - t0, "train_s": t2 - t1}))


if __name__ == "__main__":
    main()
