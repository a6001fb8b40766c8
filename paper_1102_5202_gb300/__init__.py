"""GB300-native GRMHD finite-volume hot path (HORIZON, arXiv:1102.5202).

The compute path is the CUDA library ``libhzn.so`` (sm_103a) behind the C-ABI declared in
``include/hzn.h``; ``paper_1102_5202_gb300.hzn`` is the thin ctypes binding with the same
names.  ``workloads`` writes the seeded synthetic inputs.  The library is loaded on first
use and a missing or unloadable library raises: there is no CPU fallback.
"""
__all__ = ["hzn", "workloads"]
