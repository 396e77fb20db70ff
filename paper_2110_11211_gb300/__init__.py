"""sfcdd: GB300 (sm_103a) two-level overlapping Schwarz solver on
space-filling-curve subdomains (Griebel, Schweitzer, Troska, arXiv 2110.11211).

The compute path is the CUDA library libsfcdd.so (C-ABI in include/sfcdd.h);
this package only marshals arguments (ctypes) and provides a
torch.autograd.Function around the solve and its adjoint.
"""
from . import inputs  # noqa: F401


def build(force: bool = False) -> str:
    from .build import build as _b
    return _b(force=force)


def __getattr__(name):
    if name in ("Solver",):
        from .solver import Solver
        return Solver
    if name in ("SfcddSolve", "solve"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
