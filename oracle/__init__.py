"""FP64 CPU oracle for CLAMP.  Test infrastructure: imported only by tests/,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``."""
from . import clamp_oracle  # noqa: F401
