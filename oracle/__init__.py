"""FP64 CPU oracle of the cascaded central-moment two-phase LB step (arXiv:1909.04166).

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it.
"""
from .oracle import *  # noqa: F401,F403
