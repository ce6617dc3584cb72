"""FP64 CPU oracle of continuous-component normal integration (arXiv 2510.11508).

This package is TEST INFRASTRUCTURE.  Only the test-suite, the smoke check in
``__graft_entry__`` and the CPU-baseline / reference legs of ``bench.py`` may
import it.  The CUDA library never calls it and shares no code with it.
"""
from .ni_oracle import *  # noqa: F401,F403
