"""Batched AC power flow (Newton-Raphson + implicit adjoint) on GB300 (sm_103a).

Importing the package is cheap; the CUDA library ``libpf.so`` is loaded on first
use by ``PowerFlow`` (and fails loudly if it has not been built).
"""
__all__ = ["PowerFlow", "PFLayer", "PFLayerQlim", "build_ybus", "analyze", "SolveResult",
           "Gradients"]


def __getattr__(name):
    if name in __all__:
        from . import powerflow
        return getattr(powerflow, name)
    raise AttributeError(name)
