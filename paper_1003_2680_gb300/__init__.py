"""GB300 stochastic multigrid library for the Stochastic Eulerian-Lagrangian Method.

The compute path is ``libselm_mg.so`` (hand-written sm_103a CUDA behind the C
ABI of ``include/selm_mg.h``); ``selm`` is its ctypes binding.
"""

from . import _build  # noqa: F401

__all__ = ["selm", "build"]


def build(force=False, verbose=False):
    """Compile libselm_mg.so in-tree for sm_103a and return its path."""
    return _build.build(force=force, verbose=verbose)
