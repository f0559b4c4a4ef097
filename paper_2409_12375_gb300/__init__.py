"""GB300 (sm_103a) library for FMM-accelerated SIE resistance/inductance
extraction after Wang et al., "XRL" (arXiv 2409.12375).

The compute path is the C-ABI shared library built from csrc/ (see
include/xrl.h); this package only marshals arguments to it.
"""
from .xrl import MLP, XRL, Options, Stats, XRLError, lib, library_path  # noqa: F401
