"""GB300-native cubical persistence (H0, the top dimension, and H1 of volumes).

The computation runs in libcp_gb300.so (hand-written sm_103a kernels behind
the C-ABI of include/cubical_persistence.h); this package is its binding.
"""
from ._lib import PAIR_DTYPE, CpError, load  # noqa: F401
from .api import (  # noqa: F401
    Diagram,
    diagram,
    pairs_backward,
    persistence,
    persistence_batched,
    persistence_full,
    persistence_full_batched,
    persistence_slabs,
)
from .batched import BatchedPersistence  # noqa: F401
