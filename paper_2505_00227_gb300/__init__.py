"""GB300 (sm_103a) implementation of HP-MDR progressive data refactoring.

The compute path lives in ``libhpmdr.so`` (hand-written CUDA kernels behind the
C ABI of ``include/hpmdr.h``); ``binding`` marshals PyTorch tensors into it.
"""
from . import binding  # noqa: F401
from .binding import Context, Handle, HpmdrError, RetrieveInfo  # noqa: F401
