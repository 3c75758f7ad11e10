"""B300-native batched trajectory optimizer (alternating minimization over a
batch of Bernstein-polynomial trajectories with polar/spherical constraint
reformulation), built on a C-ABI CUDA library for sm_103a.

The CUDA binding (``paper_2408_10731_b300.trajbatch``) is imported lazily so
that ``paper_2408_10731_b300.scenes`` can be used without loading it.
"""
import importlib

__all__ = ["scenes", "trajbatch"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
