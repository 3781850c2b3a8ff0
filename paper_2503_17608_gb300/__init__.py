"""Step-based EM Monte Carlo transport with track sorting on one GB300.

A GB300-native (sm_103a) implementation of the step-based ("per-action")
transport loop of Lund et al., arXiv:2503.17608 (Sec. 2), with the
action-based reordering of track slots of Sec. 3.1. The compute path is the
CUDA library libceler_gb.so behind the C ABI of include/celer_gb.h;
``binding`` is its thin Python wrapper and ``workloads`` the seeded input
generators.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "binding", "build"]
