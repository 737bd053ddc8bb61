"""GSIS / source iteration for the steady gray RTE on one GB300 (sm_103a).

The compute path is the CUDA library libgsis.so (C ABI in include/gsis.h);
`paper_2507_03975_gb300.gsis` is its thin Python binding.  The library is
loaded lazily on first use and never replaced by a CPU path.
"""
from . import gsis  # noqa: F401
from .gsis import GsisError, default_options, solve, synthetic_step, transport_sweep  # noqa: F401
