"""Single-GPU (B300, sm_103a) subgraph enumeration after HUGE (SIGMOD 2021): PULL-EXTEND and
PUSH-JOIN under a bounded-memory DFS/BFS-adaptive persistent scheduler, behind the C ABI of
include/huge.h. ``huge`` is the Python binding of that ABI."""
from . import huge  # noqa: F401
