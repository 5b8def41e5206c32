"""The learned closure gains over the method without it (reduced configuration).

Filtered DNS (128^3 -> 32^3, nu = 1/2000, k0 = 4) generated by the solver itself;
a-posteriori training through 5 unrolled FP32 LES steps with the tensor-core closure;
on held-out trajectories the trained closure must have a lower energy-spectrum error
against the filtered DNS than the LES without a closure, and the training loss must fall.
"""

import pytest

from paper_2604_18536_b300 import les

pytestmark = pytest.mark.gpu


def test_trained_closure_beats_no_closure_les():
    nu = 1.0 / 2000
    data = les.dns_dataset(range(16), n_dns=128, n_les=32, nu=nu, nsnap=5, spinup=50)
    train, test = data[:12], data[12:]
    base, _ = les.evaluate(test, 32, nu, nsteps=5)
    W, b, hist = les.train(train, 32, nu, iters=40, batch=4, lr=1e-3, nsteps=5)
    err, fallbacks = les.evaluate(test, 32, nu, W, b, nsteps=5)
    assert fallbacks == 0
    assert hist[-1] < hist[0]
    assert err < base, (err, base)
