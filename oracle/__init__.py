"""FP64 CPU oracle of the multilevel U(1) hot path.

Test infrastructure only: imported by ``tests/``, the package smoke check and
the benchmark's CPU-baseline leg, never by the product path.
"""

from .oracle import *  # noqa: F401,F403
from .oracle import build, lib  # noqa: F401
