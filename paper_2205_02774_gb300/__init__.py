"""GB300 (sm_103a) implementation of the STG-LBM hot path.

The per-step computation (synthetic turbulence inlet, regularized LES-LBM
stream/collide with walls, periodic span and pressure outlet, FP64 statistics
and mass check) runs in hand-written CUDA kernels inside ``libstglbm.so``,
reached through the C ABI declared in ``include/stg_lbm.h``.  ``capi`` binds
that ABI one function per entry point; ``Channel`` is a convenience handle
that lets PyTorch provide the device memory and the stream.
"""
from . import capi  # noqa: F401
from .capi import lib, StgError  # noqa: F401


def build(force=False):
    from .compile_lib import build as _b
    return _b(force=force)


def __getattr__(name):
    if name == "Channel":
        from .channel import Channel
        return Channel
    raise AttributeError(name)
