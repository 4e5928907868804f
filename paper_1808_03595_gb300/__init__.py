"""semmg: GB300-native p-multigrid for the statically condensed spectral-element Helmholtz problem.

The solver (condensed operator, star smoother, transfers, coarse solve,
V-cycle and outer iteration) lives in the CUDA library libsemmg.so behind the
C ABI of include/semmg.h.  ``solver.Context`` is a thin binding for torch CUDA
tensors.  Nothing is imported eagerly so that the build step can run without
a GPU.
"""

__all__ = ["Context", "Batch", "build"]


def __getattr__(name):
    if name == "Context":
        from .solver import Context
        return Context
    if name == "Batch":
        from .solver import Batch
        return Batch
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
