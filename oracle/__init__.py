"""Plain FP64 CPU oracle for the staggered-grid incompressible Navier-Stokes step.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library never
links, imports or calls it, and it shares no code with the CUDA library.

What it computes is the discrete scheme of the paper (arXiv 2604.18536,
"A differentiable software suite for accelerated simulation of turbulent
flows"), written as slowly and plainly as possible with numpy:

* ``grid``         -- staggered (MAC) grid from face coordinates (Sec. 2.1, App. A),
                      uniform and tanh-stretched faces (Sec. 2.5, tanh-grid equation).
* ``operators``    -- divergence, pressure gradient, diffusion, convection, F(u)
                      (Sec. 2.2, App. A momentum equation, App. B kernels).
* ``poisson``      -- pressure Poisson L p = D F (Sec. 2.6.1): spectral solver for
                      fully periodic uniform grids, FFT + tridiagonal solve for a
                      wall-normal direction; projection.
* ``timestep``     -- explicit RK4 with a projection at every stage (Sec. 2.6.2) and
                      the CFL time step.
* ``adjoint``      -- pullbacks (Sec. 3.4, App. B pullback equations) and the
                      vector-Jacobian product of one RK4 step.
* ``diagnostics``  -- kinetic energy, divergence norms, face-averaging filter,
                      shell energy spectrum, wall-normal profiles.

Parity status of every function is stated in its own docstring; where nothing
external pins it the docstring says "parity unpinned".
"""

from . import grid, operators, poisson, timestep, adjoint, diagnostics  # noqa: F401
from .grid import Grid, uniform_faces, tanh_faces  # noqa: F401
