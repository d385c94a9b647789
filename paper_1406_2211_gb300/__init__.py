"""GB300 (sm_103a) coupled lattice-Boltzmann library.

The CUDA library (csrc/, built to _build/liblbc.so by builder.build()) runs
one time step of the D3Q19 lattice-Boltzmann fluid with the operator-split
particle coupling of arXiv:1406.2211; `lbc` is its ctypes binding.
"""
from . import builder  # noqa: F401
from . import lbc  # noqa: F401
