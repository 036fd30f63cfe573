"""GB300-native hot path of the hybrid immersed-boundary / phase-field method
(arXiv 2104.00350): a CUDA C-ABI library (``csrc/``, ``include/ib_pf.h``) and its ctypes
binding (``ibpf``)."""
from . import ibpf  # noqa: F401
