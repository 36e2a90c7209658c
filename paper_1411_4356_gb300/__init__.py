"""omss: GB300-native steady states of driven, damped optomechanical systems.

CUDA library libomss.so (C ABI in include/omss.h) with a thin Python
binding.  See ``api`` for the entry points and ``workloads`` for the
parameter sets.
"""
from .workloads import ADJOINT, CCPT, LARGE, MID, TINY, SystemParams, Workload  # noqa: F401

__all__ = ["SystemParams", "Workload", "TINY", "MID", "LARGE", "ADJOINT", "CCPT"]
