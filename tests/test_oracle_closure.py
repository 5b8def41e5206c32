"""Pins of the oracle's CNN closure (library routines, brute force, exact transposes, FD)."""

import numpy as np
import pytest
import torch
from scipy.stats import norm

from oracle import closure as cl


def test_bf16_round_to_nearest_even():
    one = 1.0
    assert cl.bf16(one) == one
    assert cl.bf16(1 + 2.0 ** -8) == 1.0                      # tie -> even mantissa
    assert cl.bf16(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6        # tie -> even (odd neighbour below)
    assert cl.bf16(1 + 2.0 ** -8 + 2.0 ** -12) == 1 + 2.0 ** -7
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).integers(-6, 6, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cl.bf16(x), ref)


def test_gelu_is_x_times_normal_cdf():
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(cl.gelu(z), z * norm.cdf(z), atol=1e-15)
    eps = 1e-6
    np.testing.assert_allclose(cl.gelu_grad(z), (cl.gelu(z + eps) - cl.gelu(z - eps)) / (2 * eps), atol=1e-8)


def test_conv_matches_torch_circular_conv3d():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((5, 6, 4, 7))
    W = rng.standard_normal((27, 5, 3))
    b = rng.standard_normal(3)
    y = cl.conv(x, W, b)
    wt = torch.tensor(W.reshape(3, 3, 3, 5, 3)).permute(4, 3, 0, 1, 2).contiguous()   # (co, ci, kz, ky, kx)
    xt = torch.nn.functional.pad(torch.tensor(x)[None], (1, 1, 1, 1, 1, 1), mode="circular")
    ref = torch.nn.functional.conv3d(xt, wt, torch.tensor(b))[0].numpy()
    np.testing.assert_allclose(y, ref, atol=1e-12)


def test_conv_brute_force_loop():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 3, 4, 5))
    W = rng.standard_normal((27, 2, 2))
    y = cl.conv(x, W)
    Z, Y, X = x.shape[1:]
    ref = np.zeros((2, Z, Y, X))
    for co in range(2):
        for k in range(Z):
            for j in range(Y):
                for i in range(X):
                    s = 0.0
                    for t, (dz, dy, dx) in enumerate(cl.taps()):
                        for ci in range(2):
                            s += W[t, ci, co] * x[ci, (k + dz) % Z, (j + dy) % Y, (i + dx) % X]
                    ref[co, k, j, i] = s
    np.testing.assert_allclose(y, ref, atol=1e-13)


def test_centre_one_hot_kernel_is_identity():
    x = np.random.default_rng(4).standard_normal((3, 4, 4, 4))
    W = np.zeros((27, 3, 3))
    W[13] = np.eye(3)
    assert np.array_equal(cl.conv(x, W), x)


def test_conv_transpose_and_weight_gradient_are_exact():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((4, 5, 6, 3))
    dy = rng.standard_normal((3, 5, 6, 3))
    W = rng.standard_normal((27, 4, 3))
    V = rng.standard_normal((27, 4, 3))
    assert abs(np.sum(cl.conv(x, W) * dy) - np.sum(x * cl.conv_T(dy, W))) < 1e-10
    # conv is linear in W: <conv(x; V), dy> = <V, wgrad(x, dy)>
    assert abs(np.sum(cl.conv(x, V) * dy) - np.sum(V * cl.conv_wgrad(x, dy))) < 1e-10


def test_translation_equivariance_bitexact():
    params = cl.init_params(0)
    u = np.random.default_rng(6).standard_normal((3, 6, 6, 6))
    m = cl.forward(params, u)
    us = np.roll(u, (1, -2, 3), axis=(1, 2, 3))
    assert np.array_equal(cl.forward(params, us), np.roll(m, (1, -2, 3), axis=(1, 2, 3)))


def test_backward_central_differences_unquantised():
    params = cl.init_params(1, scale=2.0)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((3, 4, 5, 6))
    mbar = rng.standard_normal((3, 4, 5, 6))
    ub, grads = cl.backward(params, u, mbar, quantize=False)
    eps = 1e-6
    for s in range(3):
        v = rng.standard_normal(u.shape)
        fd = (np.sum(mbar * cl.forward(params, u + eps * v, quantize=False))
              - np.sum(mbar * cl.forward(params, u - eps * v, quantize=False))) / (2 * eps)
        assert abs(fd - np.sum(ub * v)) < 1e-7 * max(1, abs(fd))
    for l in (0, 3):
        W, b = params[l]
        V = rng.standard_normal(W.shape)
        pp = [list(p) for p in params]
        pm = [list(p) for p in params]
        pp[l][0] = W + eps * V
        pm[l][0] = W - eps * V
        fd = (np.sum(mbar * cl.forward(pp, u, quantize=False)) - np.sum(mbar * cl.forward(pm, u, quantize=False))) / (2 * eps)
        assert abs(fd - np.sum(grads[l][0] * V)) < 1e-7 * max(1, abs(fd))
        db = rng.standard_normal(b.shape)
        pp = [list(p) for p in params]
        pm = [list(p) for p in params]
        pp[l][1] = b + eps * db
        pm[l][1] = b - eps * db
        fd = (np.sum(mbar * cl.forward(pp, u, quantize=False)) - np.sum(mbar * cl.forward(pm, u, quantize=False))) / (2 * eps)
        assert abs(fd - np.sum(grads[l][1] * db)) < 1e-7 * max(1, abs(fd))


def test_quantised_forward_is_close_to_unquantised():
    params = cl.init_params(2)
    u = np.random.default_rng(8).standard_normal((3, 6, 6, 6))
    mq = cl.forward(params, u)
    m = cl.forward(params, u, quantize=False)
    assert np.linalg.norm(mq - m) < 2e-2 * np.linalg.norm(m)


def test_step_vjp_with_closure_central_differences():
    """RK4 step with the (unquantised) closure in F: pullback in u0 and in a weight, against FD."""
    from oracle import adjoint, poisson, timestep
    from test_oracle_operators import periodic_grid, random_u
    g = periodic_grid(6, 3, nu=0.05)
    params = cl.init_params(3, scale=0.5)
    clo = cl.Closure(params, quantize=False)
    u0, _ = poisson.project(g, random_u(g, 31))
    c = random_u(g, 32)
    dt = 0.02
    ub, nb, wg = adjoint.rk4_step_vjp(g, u0, dt, c, clo)
    eps = 1e-6
    L = lambda u, cc=clo: float(np.sum(c * timestep.rk4_step(g, u, dt, cc)))
    v = random_u(g, 33)
    fd = (L(u0 + eps * v) - L(u0 - eps * v)) / (2 * eps)
    assert abs(fd - np.sum(ub * v)) < 1e-7 * max(1, abs(fd))
    V = np.random.default_rng(34).standard_normal(params[1][0].shape)
    pp = [list(p) for p in params]
    pm = [list(p) for p in params]
    pp[1][0] = params[1][0] + eps * V
    pm[1][0] = params[1][0] - eps * V
    fd = (L(u0, cl.Closure(pp, False)) - L(u0, cl.Closure(pm, False))) / (2 * eps)
    assert abs(fd - np.sum(wg[1][0] * V)) < 1e-7 * max(1, abs(fd))
