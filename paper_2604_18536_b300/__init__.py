"""B300-native staggered-grid incompressible Navier-Stokes RK step (libins + thin binding).

Submodules:
  solver  -- Grid: torch tensors -> libins C ABI (ins_rhs, ins_project, ins_step, ...)
  inputs  -- seeded synthetic inputs (faces, initial fields); no method arithmetic
  build   -- nvcc build of libins.so (sm_103a)
The shared library is loaded on first use; there is no CPU fallback.
"""

__all__ = ["Grid"]


def __getattr__(name):
    if name == "Grid":
        from .solver import Grid
        return Grid
    raise AttributeError(name)
