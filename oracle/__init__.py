"""CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library does not, and this
package imports nothing from the library.
"""
from . import tpmg  # noqa: F401
from .tpmg import MGParams  # noqa: F401
