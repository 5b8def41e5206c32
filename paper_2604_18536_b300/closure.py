"""CNN closure m(u) (libins ins_closure_*): torch tensors in, pointers out. Marshalling only.

Weights W[l] are float32 CUDA tensors of shape (27, cin, cout) (tap t = 9(dz+1) + 3(dy+1) + (dx+1)),
biases b[l] float32 (cout,); layer shapes 3->32->32->32->3. The library rounds the weights
to BF16 when set_params is called, so call it again after every weight update.
"""

import ctypes

import torch

from . import _lib
from ._lib import check, lib

SHAPES = [(3, 32), (32, 32), (32, 32), (32, 3)]


def _ptrs(ts):
    arr = (ctypes.c_void_p * 4)()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr() if t is not None else None
    return arr


def init_params(seed, scale=1.0, device="cuda"):
    """Seeded float32 weights uniform(+-scale sqrt(3/fan_in)) and zero biases (leaf tensors)."""
    gen = torch.Generator().manual_seed(seed)
    W, b = [], []
    for cin, cout in SHAPES:
        lim = scale * (3.0 / (27 * cin)) ** 0.5
        W.append(((torch.rand((27, cin, cout), generator=gen, dtype=torch.float64) * 2 - 1) * lim)
                 .float().to(device))
        b.append(torch.zeros(cout, dtype=torch.float32, device=device))
    return W, b


class Closure:
    def __init__(self, grid):
        self.grid = grid
        h = ctypes.c_void_p()
        check(lib().ins_closure_create(grid._h, ctypes.byref(h)), "ins_closure_create")
        self._h = h
        self.W = None
        self.b = None

    def close(self):
        if getattr(self, "_h", None):
            lib().ins_closure_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, W, b):
        for (cin, cout), w, bb in zip(SHAPES, W, b):
            if tuple(w.shape) != (27, cin, cout) or w.dtype != torch.float32 or not w.is_contiguous():
                raise ValueError("weights must be contiguous float32 (27, cin, cout)")
            if tuple(bb.shape) != (cout,) or bb.dtype != torch.float32:
                raise ValueError("biases must be float32 (cout,)")
        self.W, self.b = list(W), list(b)
        self.grid._sync_stream()
        check(lib().ins_closure_set_params(self._h, _ptrs(self.W), _ptrs(self.b)), "ins_closure_set_params")

    def set_grads(self, dW, db):
        """Accumulators that ins_step_vjp adds the closure's weight/bias gradients to."""
        self._gW, self._gB = list(dW), list(db)
        check(lib().ins_closure_set_grads(self._h, _ptrs(self._gW), _ptrs(self._gB)), "ins_closure_set_grads")

    def forward(self, u, m=None, save=False):
        self.grid._check_u(u)
        m = self.grid.new_velocity() if m is None else m
        self.grid._sync_stream()
        check(lib().ins_closure_fwd(self.grid._h, self._h, ctypes.c_void_p(u.data_ptr()),
                                    ctypes.c_void_p(m.data_ptr()), int(save)), "ins_closure_fwd")
        return m

    def backward(self, mbar, ubar=None, dW=None, db=None):
        """ubar += (dm/du)^T mbar (a new zero field if None); dW, db lists are accumulated into."""
        self.grid._check_u(mbar, "mbar")
        ubar = self.grid.new_velocity() if ubar is None else ubar
        self.grid._sync_stream()
        check(lib().ins_closure_bwd(self.grid._h, self._h, ctypes.c_void_p(mbar.data_ptr()),
                                    ctypes.c_void_p(ubar.data_ptr()),
                                    _ptrs(dW) if dW is not None else None,
                                    _ptrs(db) if db is not None else None), "ins_closure_bwd")
        return ubar

    def saved(self, layer):
        """(x_l as bf16 (nvox, C), z_l float32 (nvox, 32) or None) from the last saving forward."""
        nv = self.grid.N
        C = 8 if layer == 0 else 32
        x = torch.empty((nv, C), dtype=torch.bfloat16, device=self.grid.device)
        z = torch.empty((nv, 32), dtype=torch.float32, device=self.grid.device) if layer < 3 else None
        check(lib().ins_closure_saved(self._h, layer, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(z.data_ptr()) if z is not None else None), "ins_closure_saved")
        return x, z

    def check(self):
        check(lib().ins_closure_check(self._h), "ins_closure_check")
