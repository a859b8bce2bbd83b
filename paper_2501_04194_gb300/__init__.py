"""GB300-native STL robustness (after STLCG++, arXiv 2501.04194).

PyTorch supplies device memory and streams; every step of the robustness trace and of its
gradient runs in the hand-written CUDA kernels of ``libstl.so`` (sm_103a), reached through
the C ABI in ``include/stl.h``.
"""
from .binding import STL_HARD, STL_SMOOTH, STL_SOFTMAX, Formula, FormulaSet, StlError, flatten, load, params  # noqa: F401
from .torch_api import (HostPipeline, RaggedBatch, STLRobustness, autotune, robustness,  # noqa: F401
                        robustness_and_grad, robustness_backward)

__all__ = ["Formula", "FormulaSet", "HostPipeline", "RaggedBatch", "STLRobustness", "robustness", "robustness_backward", "robustness_and_grad", "autotune", "params", "load", "StlError",
           "STL_HARD", "STL_SMOOTH", "STL_SOFTMAX", "flatten"]
