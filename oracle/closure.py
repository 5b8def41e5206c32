"""CNN closure model m(u) added to the right-hand side F (FP64 numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Sec. 4 (neural-network closure models inside the right-hand side of the
LES solver, trained a posteriori through the unrolled solver; gradients by
reverse-mode AD with hand-written pullbacks, Sec. 3.4). The paper names no
architecture. Reading taken (a choice, not the paper's):

* input channels: u^x, u^y, u^z at the same storage index; output channel a is
  added to F^a at that index;
* 4 convolution layers with 3x3x3 kernels and circular (periodic) padding,
  channels 3 -> 32 -> 32 -> 32 -> 3, GELU (erf form) after the first three;
* y[co, v] = b[co] + sum_t sum_ci W[t, ci, co] x[ci, v + o_t], with the 27 taps
  o_t = (dz, dy, dx), t = 9 (dz+1) + 3 (dy+1) + (dx+1) (a correlation);
* BF16 (round to nearest even) weights, layer inputs and activations; FP32
  biases; products of BF16 values are exact here and sums are FP64 (the GPU
  accumulates in FP32);
* the backward pass treats the BF16 roundings as identity and rounds each
  layer's incoming gradient to BF16; that rounded gradient feeds the transposed
  convolution, the weight gradient and the bias gradient alike.

``quantize=False`` switches every rounding off (a smooth FP64 network for
finite-difference pins).
"""

import numpy as np
from scipy.special import erf

SHAPES = [(3, 32), (32, 32), (32, 32), (32, 3)]


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) through float32; returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def taps():
    """The 27 offsets (dz, dy, dx) in tap order."""
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x, o):
    """x[..., v + o] with circular wrap; x has trailing axes (Z, Y, X)."""
    dz, dy, dx = o
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))


def conv(x, W, b=None):
    """y[co] = b[co] + sum_t sum_ci W[t, ci, co] x[ci](v + o_t); x: (C_in, Z, Y, X)."""
    cout = W.shape[2]
    y = np.zeros((cout,) + x.shape[1:])
    for t, o in enumerate(taps()):
        y += np.einsum("io,i...->o...", W[t], shift(x, o))
    if b is not None:
        y += np.asarray(b).reshape((-1, 1, 1, 1))
    return y


def conv_T(dy, W):
    """Transpose of ``conv`` in its input: dx[ci](v) = sum_t sum_co W[t, ci, co] dy[co](v - o_t)."""
    cin = W.shape[1]
    dx = np.zeros((cin,) + dy.shape[1:])
    for t, o in enumerate(taps()):
        dx += np.einsum("io,o...->i...", W[t], shift(dy, (-o[0], -o[1], -o[2])))
    return dx


def conv_wgrad(x, dy):
    """dW[t, ci, co] = sum_v x[ci](v + o_t) dy[co](v)."""
    cin, cout = x.shape[0], dy.shape[0]
    dW = np.zeros((27, cin, cout))
    for t, o in enumerate(taps()):
        dW[t] = shift(x, o).reshape(cin, -1) @ dy.reshape(cout, -1).T
    return dW


def init_params(seed, scale=1.0):
    """Seeded weights (BF16 values) and biases: uniform(+-scale sqrt(3/fan_in)), biases 0."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in SHAPES:
        lim = scale * np.sqrt(3.0 / (27 * cin))
        W = bf16(rng.uniform(-lim, lim, size=(27, cin, cout)))
        params.append((W, np.zeros(cout)))
    return params


def forward(params, u, quantize=True, keep=False):
    """m(u) for one sample u of shape (3, Z, Y, X). Returns m (and the per-layer record)."""
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    x = q(u)
    rec = []
    for l, (W, b) in enumerate(params):
        z = conv(x, q(W), b)
        rec.append((x, z))
        if l < len(params) - 1:
            x = q(gelu(z))
        else:
            m = np.asarray(z, dtype=np.float32).astype(np.float64) if quantize else z
    if keep:
        return m, rec
    return m


def backward(params, u, mbar, quantize=True):
    """Pullback of ``forward``: (ubar, [(dW, db) per layer]) for the cotangent mbar of m."""
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    _, rec = forward(params, u, quantize, keep=True)
    grads = [None] * len(params)
    g = np.asarray(mbar, dtype=np.float64)
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        x, z = rec[l]
        if l < len(params) - 1:
            g = g * gelu_grad(z)
        gq = q(g)
        grads[l] = (conv_wgrad(x, gq), np.sum(gq, axis=(1, 2, 3)))
        g = conv_T(gq, q(W))
    return g, grads


class Closure:
    """m(u) as the closure term of F for a (3, Z, Y, X) velocity (``operators.rhs_F`` hook)."""

    def __init__(self, params, quantize=True):
        self.params = params
        self.quantize = quantize

    def __call__(self, u):
        return forward(self.params, u, self.quantize)

    def vjp(self, u, mbar):
        ub, _ = backward(self.params, u, mbar, self.quantize)
        return ub
