"""GB300-native particle <-> fixed-mesh projection round trip (Duque & Espanol,
arXiv 1610.05266): hand-written sm_103a CUDA kernels behind the C ABI of include/pfem.h,
with a thin ctypes binding.

The CUDA library is required: importing the binding never falls back to a CPU path.
"""
from ._lib import LibraryMissing, PfemError, load  # noqa: F401
from .api import *  # noqa: F401,F403
from .api import Projector, Cells  # noqa: F401
from . import autograd  # noqa: F401
