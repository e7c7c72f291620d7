"""GB300 (sm_103a) far-field compression by sampled-row interpolative decomposition.

The compute path is libffc.so (CUDA kernels behind the C ABI in include/ffc.h);
``paper_1409_2802_gb300.ffc`` is its ctypes binding.
"""
from . import ffc  # noqa: F401

__all__ = ["ffc"]
