"""FP64 CPU oracle of the MUFFIN primal-dual method (test infrastructure only).

Imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py``; never by the library.
"""
from . import muffin_oracle  # noqa: F401
