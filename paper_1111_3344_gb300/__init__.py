"""GB300-native BSSN moving-puncture evolution (RK4 method of lines).

The compute path is the CUDA C-ABI library libbssn.so (include/bssn.h);
``paper_1111_3344_gb300.bssn`` is its ctypes binding.
"""
from . import bssn  # noqa: F401
from .bssn import Evolution, Params  # noqa: F401
