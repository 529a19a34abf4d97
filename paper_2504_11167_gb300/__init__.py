"""GB300-native LR-SPIKE: the data-parallel hot path of the Low-Rank SPIKE solver
for banded systems A x = f (Spring, Polizzi, Sameh, arXiv 2504.11167).

Every step of the path runs in hand-written CUDA kernels for sm_103a inside
``liblrspike.so``, behind the C ABI declared in ``include/lrspike.h``.  This
package is the thin Python binding (argument marshalling only).  Importing the
package is cheap; the shared library is loaded on first use and a missing
library raises instead of falling back to anything else.
"""

__all__ = ["LRSpike", "Options", "LRSpikeError", "load_library"]


def __getattr__(name):
    if name in ("LRSpike", "Options", "LRSpikeError", "load_library"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
