"""GB300 (sm_103a) Schur-complement PCG solve path for trajectory-optimisation
KKT systems (MPCGPU, arXiv 2309.08079).

The compute runs in libmpcg.so (C ABI: include/mpcg.h); this package holds
the ctypes/PyTorch binding, the autograd wrapper, the batched launch-plan
autotuner and the build script.
Importing the package does not load the library; the first Solver() does,
and fails loudly if it has not been built.
"""
__all__ = ["Solver", "LQTensors", "SchurTensors", "make_opts", "read_stats", "MPCGSolve",
           "Autotuner", "PlanRunner"]


def __getattr__(name):
    if name in ("Solver", "LQTensors", "SchurTensors", "make_opts", "read_stats"):
        from . import solver
        return getattr(solver, name)
    if name in ("Autotuner", "PlanRunner"):
        from . import autotune
        return getattr(autotune, name)
    if name == "MPCGSolve":
        from .autograd import MPCGSolve
        return MPCGSolve
    raise AttributeError(name)
