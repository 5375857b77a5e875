"""GB300-native volume potentials with truncated free-space Green's functions.

Implements the method of Vico, Greengard & Ferrando, "Fast convolution with
free-space Green's functions" (arXiv:1604.03155): a one-off FP64 precompute of
the regularised kernel spectrum and a per-density zero-padded (2N)^d FFT
convolution, both as hand-written sm_103a CUDA kernels behind the C ABI of
``include/vp.h``.  ``vp`` is the thin Python binding of that ABI; ``inputs``
holds the seeded synthetic densities.
"""
from . import inputs  # noqa: F401
from .vp import Plan, VPError  # noqa: F401
