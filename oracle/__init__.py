"""FP64 CPU oracle for the LapH block contraction (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library does not.
"""
from .oracle import (baryon_blocks, baryon_dense, baryon_triples, build, diquarks,  # noqa: F401
                     meson_blocks, num_threads, phase_table)
