"""B300 (sm_103a) hot path of parallel Continuous Local Search (arXiv
2606.06656): batched Walsh-Fourier expansion + gradient of weighted symmetric
pseudo-Boolean constraints, projected gradient steps, rounding and exact
satisfaction counts, behind the C ABI of include/cls.h.

The compute lives in libcls_b300.so (built in-tree by csrc/build.py); this
package only marshals arguments.  Importing it does not require a GPU; the
first call that needs the library loads it and raises if it is missing.
"""
from . import _lib  # noqa: F401
from . import binding  # noqa: F401
from .api import Problem  # noqa: F401

__all__ = ["Problem", "binding"]
