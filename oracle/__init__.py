"""FP64 CPU oracle (test infrastructure only; see ``oracle.acq``).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
"""
from . import acq  # noqa: F401
