"""FP64 CPU oracle of the ISAAC ray caster -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the C source, its structures and the op-code table here are its own.
"""
from .oracle import (INF, build, render, invert4, max_threads, chain_eval, classify,  # noqa: F401
                     quantize, lowp_copy, opacity_grid, range_grid, render_iso, OP_CODES)
