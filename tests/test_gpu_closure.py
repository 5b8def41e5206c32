"""CNN closure on the tensor cores against the oracle.

Per layer (tight): the oracle's convolution applied to the GPU's own BF16 layer input must
match the GPU's FP32 pre-activation (the only difference is FP32 vs FP64 summation order),
and the GPU's next BF16 activation must equal bf16(gelu(z)) of its own z except where FP32
and FP64 GELU straddle a rounding boundary (rare, one BF16 ulp).
End to end (loose): independent BF16 roundings on both sides let single activations differ by
one BF16 ulp, so whole-network outputs and gradients are compared in relative L2 norm.
"""

import numpy as np
import pytest
import torch

from oracle import closure as oc, poisson, timestep, adjoint
from oracle.grid import Grid as OGrid
from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300.closure import Closure, init_params, SHAPES
from paper_2604_18536_b300.solver import Grid

pytestmark = pytest.mark.gpu


def make(n=(16, 16, 8), dtype=torch.float64, seed=0, scale=1.0, nu=0.01):
    faces = [inputs.uniform_faces(k, 0, 2 * np.pi) for k in n]
    g = Grid(faces, ["periodic"] * 3, nu, dtype=dtype)
    og = OGrid(faces, ["periodic"] * 3, nu)
    W, b = init_params(seed, scale)
    for bb in b:
        bb.copy_(torch.linspace(-0.1, 0.1, bb.numel()))
    c = Closure(g)
    c.set_params(W, b)
    params = [(oc.bf16(w.double().cpu().numpy()), bb.double().cpu().numpy()) for w, bb in zip(W, b)]
    return g, og, c, W, b, params


def to_cfirst(t, C, og):
    """(nvox, C) channels-last -> (C, nz, ny, nx) float64."""
    return t.float().double().cpu().numpy()[:, :C].T.reshape((C,) + og.shape)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("n", [(16, 16, 8), (32, 32, 16)])
def test_layers_match_oracle(n):
    g, og, c, W, b, params = make(n)
    u = inputs.random_field((3,) + og.shape, 3)
    m = c.forward(torch.tensor(u, device="cuda"), save=True)
    c.check()
    x0, _ = c.saved(0)
    assert np.array_equal(to_cfirst(x0, 3, og), oc.bf16(u))
    for l in range(4):
        cin, cout = SHAPES[l]
        x, _ = c.saved(l)
        X = to_cfirst(x, cin, og)
        z_or = oc.conv(X, params[l][0], params[l][1])
        if l < 3:
            _, z = c.saved(l)
            Z = to_cfirst(z, cout, og)
            assert rel(Z, z_or) <= 1e-5, (l, rel(Z, z_or))
            xn, _ = c.saved(l + 1)
            XN = to_cfirst(xn, cout, og)
            ref = oc.bf16(oc.gelu(Z))
            diff = XN != ref
            assert diff.mean() <= 2e-3, (l, diff.mean())
            if diff.any():
                assert np.max(np.abs(XN - ref)[diff] / np.maximum(np.abs(ref[diff]), 1e-30)) <= 2.0 ** -7 + 1e-12
        else:
            assert rel(m.cpu().numpy(), z_or) <= 1e-5


def test_forward_and_backward_match_oracle():
    g, og, c, W, b, params = make((32, 32, 16))
    rng = np.random.default_rng(4)
    u = rng.standard_normal((3,) + og.shape)
    mbar = rng.standard_normal((3,) + og.shape)
    m = c.forward(torch.tensor(u, device="cuda"), save=True)
    m_or = oc.forward(params, u)
    assert rel(m.cpu().numpy(), m_or) <= 5e-3
    dW = [torch.zeros_like(w) for w in W]
    db = [torch.zeros_like(bb) for bb in b]
    ub = c.backward(torch.tensor(mbar, device="cuda"), dW=dW, db=db)
    c.check()
    ub_or, grads = oc.backward(params, u, mbar)
    assert rel(ub.cpu().numpy(), ub_or) <= 2e-2
    for l in range(4):
        assert rel(dW[l].double().cpu().numpy(), grads[l][0]) <= 2e-2, l
        assert rel(db[l].double().cpu().numpy(), grads[l][1]) <= 2e-2, l


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_step_and_step_vjp_with_closure(dtype):
    g, og, c, W, b, params = make((16, 16, 8), dtype=dtype, scale=0.5, nu=0.05)
    g.set_closure(c)
    clo = oc.Closure(params)
    u0, _ = poisson.project(og, inputs.random_field((3,) + og.shape, 5))
    if dtype == torch.float32:
        u0 = u0.astype(np.float32).astype(np.float64)
    dt = 0.5 * timestep.cfl_dt(og, u0, 0.3)
    ut = torch.tensor(u0, dtype=dtype, device="cuda")
    g.step(ut, dt=dt)
    ref = timestep.rk4_step(og, u0, dt, clo)
    assert rel(ut.double().cpu().numpy(), ref) <= 1e-4
    # pullback with the closure: input gradient and accumulated weight gradients
    ybar = inputs.random_field((3,) + og.shape, 6)
    dW = [torch.zeros_like(w) for w in W]
    db = [torch.zeros_like(bb) for bb in b]
    c.set_grads(dW, db)
    ub, nb = g.step_vjp(torch.tensor(u0, dtype=dtype, device="cuda"), torch.tensor(ybar, dtype=dtype, device="cuda"),
                        dt=dt)
    c.check()
    ub_or, nb_or, wg = adjoint.rk4_step_vjp(og, u0, dt, ybar, clo)
    assert rel(ub.double().cpu().numpy(), ub_or) <= 1e-3
    for l in range(4):
        assert rel(dW[l].double().cpu().numpy(), wg[l][0]) <= 3e-2, l
    g.set_closure(None)


@pytest.mark.parametrize("n", [(16, 16, 8), (24, 32, 6), (48, 32, 5)])
def test_last_layer_weight_gradient_tight(n):
    """Tensor-core weight gradient of the output layer on the GPU's own BF16 operands: the saved
    layer input x_3 and the BF16-rounded output cotangent (sizes with nx % 16 = ny % 8 = 0 take the
    staged-plane kernel, (24, 32, 6) the gathering one; nz = 5 splits z raggedly). Only the FP32 summation order differs
    from the FP64 oracle (conv_wgrad), so the relative error is at FP32 level; the bias gradient
    is the sum of the rounded cotangent."""
    g, og, c, W, b, params = make(n)
    rng = np.random.default_rng(9)
    u = rng.standard_normal((3,) + og.shape)
    mbar = rng.standard_normal((3,) + og.shape)
    c.forward(torch.tensor(u, device="cuda"), save=True)
    x3, _ = c.saved(3)
    dW = [torch.zeros_like(w) for w in W]
    db = [torch.zeros_like(bb) for bb in b]
    c.backward(torch.tensor(mbar, device="cuda"), dW=dW, db=db)
    c.check()
    gq = oc.bf16(mbar)
    ref = oc.conv_wgrad(to_cfirst(x3, 32, og), gq)
    assert rel(dW[3].double().cpu().numpy(), ref) <= 1e-5
    assert rel(db[3].double().cpu().numpy(), gq.reshape(3, -1).sum(axis=1)) <= 1e-5
