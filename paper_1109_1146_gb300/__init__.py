"""GB300-native exact grid max-flow / min-cut by the parallel sweep of
Augmented-path Region Discharge (P-ARD).

The compute path is libmf.so (hand-written sm_103a CUDA behind the C ABI of
include/mf.h); ``paper_1109_1146_gb300.mf`` is its thin Python binding.
"""
from . import mf  # noqa: F401
from .mf import Grid, MFError, default_opts, load  # noqa: F401
