"""GB300-native V-filtration cubical persistence (H0 + top dimension).

The computation runs in libcp_gb300.so (hand-written sm_103a kernels behind
the C-ABI of include/cubical_persistence.h); this package is its binding.
"""
from ._lib import PAIR_DTYPE, CpError, load  # noqa: F401
from .api import Diagram, diagram, pairs_backward, persistence, persistence_batched  # noqa: F401
from .batched import BatchedPersistence  # noqa: F401
