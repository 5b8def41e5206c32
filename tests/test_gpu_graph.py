"""ins_step_n: the steps after the first replay a CUDA graph of one step.

k steps through ins_step_n equal k ins_step calls bit for bit (FP64 and FP32, periodic and channel,
fixed dt and the device-side adaptive dt that reads and writes the same scalar); the graph is
captured again when the velocity buffer or a setting changes; nsteps = 0 is a no-op, nsteps < 0
an argument error; the launch counter counts the replayed kernels.
"""

import pytest
import torch

from paper_2604_18536_b300 import inputs
from paper_2604_18536_b300.solver import Grid
from paper_2604_18536_b300._lib import InsError
from test_gpu_parity import case, rand_u, rounded, dev
from oracle.grid import Grid as OGrid

pytestmark = pytest.mark.gpu


def setup(name, dtype):
    c = case(name)
    og = OGrid(c["faces"], c["bc"], c["nu"], c["force"])
    g = Grid(c["faces"], c["bc"], c["nu"], c["force"], dtype=dtype)
    u0 = dev(rounded(rand_u(og, 7, project=True), dtype), dtype)
    return g, u0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("name", ["p3", "c3", "p3reg2"])
def test_step_n_equals_repeated_steps(name, dtype):
    g, u0 = setup(name, dtype)
    # adaptive dt on the device: every step reads dt and writes the next one into the same scalar
    dt_a = g.cfl_dt(u0, 0.3)
    dt_b = dt_a.clone()
    a, b = u0.clone(), u0.clone()
    for _ in range(5):
        g.step(a, dt_dev=dt_a, next_dt_dev=dt_a, cfl=0.3)
    g.step_n(b, 5, dt_dev=dt_b, next_dt_dev=dt_b, cfl=0.3)
    assert torch.equal(a, b) and torch.equal(dt_a, dt_b)
    # fixed host dt, and a second run that replays the already captured graph
    for _ in range(3):
        g.step(a, dt=1e-3)
    g.step_n(b, 3, dt=1e-3)
    assert torch.equal(a, b)
    for _ in range(4):
        g.step(a, dt=1e-3)
    g.step_n(b, 4, dt=1e-3)
    assert torch.equal(a, b)


def test_step_n_recaptures_on_new_buffer_and_setting():
    g, u0 = setup("p3", torch.float32)
    a, b, c = u0.clone(), u0.clone(), u0.clone()
    g.step_n(b, 3, dt=1e-3)
    g.step_n(c, 3, dt=1e-3)          # another buffer: a new graph
    for _ in range(3):
        g.step(a, dt=1e-3)
    assert torch.equal(a, b) and torch.equal(a, c)
    g.set_step_fusion(1)             # another kernel set
    d, e = u0.clone(), u0.clone()
    g.step_n(d, 3, dt=1e-3)
    for _ in range(3):
        g.step(e, dt=1e-3)
    assert torch.equal(d, e)


def test_step_n_arguments_and_launch_count():
    g, u0 = setup("p3", torch.float64)
    u = u0.clone()
    g.step_n(u, 0, dt=1e-3)
    assert torch.equal(u, u0)
    with pytest.raises(InsError):
        g.step_n(u, -1, dt=1e-3)
    n0 = g.launch_count()
    g.step(u, dt=1e-3)
    per_step = g.launch_count() - n0
    n1 = g.launch_count()
    g.step_n(u, 4, dt=1e-3)
    assert g.launch_count() - n1 == 4 * per_step


def test_step_n_with_eddy_viscosity_model():
    g, u0 = setup("c3", torch.float64)
    g.set_eddy_viscosity("wale")
    a, b = u0.clone(), u0.clone()
    for _ in range(3):
        g.step(a, dt=1e-3)
    g.step_n(b, 3, dt=1e-3)
    assert torch.equal(a, b)
