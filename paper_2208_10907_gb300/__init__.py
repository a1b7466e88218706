"""GB300 (sm_103a) dependency-free H^2-ULV solver (arXiv 2208.10907).

The compute path is the CUDA library libh2ulv.so (csrc/), reached through
the C ABI of include/h2ulv.h; ``h2ulv`` is its thin ctypes binding.
"""
from . import h2ulv  # noqa: F401
