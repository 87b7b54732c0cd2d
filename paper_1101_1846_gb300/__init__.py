"""GB300 (sm_103a) library for the parallel Marsaglia generators of
arXiv:1101.1846 (MWC, XorShift, KISS): CUDA kernels behind a C-ABI
(include/rng.h), with PyTorch used only for device memory and streams."""
from . import capi
from .capi import (RNG_F32, RNG_KISS, RNG_MWC32, RNG_U32, RNG_XOR128, RngError)

__all__ = ["capi", "RNG_MWC32", "RNG_XOR128", "RNG_KISS", "RNG_U32", "RNG_F32",
           "RngError", "Generator", "Plan", "BatchItem", "generate_batch",
           "multipliers"]


def __getattr__(name):
    # the torch-facing helpers import torch lazily
    if name in ("Generator", "Plan", "BatchItem", "generate_batch", "multipliers"):
        from . import generator
        return getattr(generator, name)
    raise AttributeError(name)
