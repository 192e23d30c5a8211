"""Write the oracle regression fixtures in this folder.

The paper prints no block values, so these fixtures are not the paper's:
they are the FP64 oracle's output on small seeded inputs, written by this
script, which calls only ``oracle/`` and the seeded input generator.  They
guard the oracle against unintended changes; the oracle itself is pinned by
``tests/test_oracle_pins.py``.

Usage: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2510_26313_gb300 import synth  # noqa: E402

CASES = [("L2_N4_P7", 2, 4, 1), ("L3_N5_P19", 3, 5, 2)]


def write(name, L, N, n2):
    mom = synth.momentum_shell(n2)
    phi = synth.random_phi(L, N, T=1, instance=900)[0]
    B = O.baryon_blocks(phi, L, mom)
    M = O.meson_blocks(phi, L, mom)
    path = os.path.join(HERE, f"oracle_{name}.txt")
    with open(path, "w") as f:
        f.write(f"# oracle regression fixture: L={L} N={N} momenta |n|^2<={n2} (P={mom.shape[0]}),\n")
        f.write("# phi = synth.random_phi(L, N, T=1, instance=900)[0]; written by make_golden.py\n")
        for p in range(B.shape[0]):
            for idx in range(B.shape[1]):
                f.write(f"B {p} {idx} {float(B[p, idx].real)!r} {float(B[p, idx].imag)!r}\n")
        for p in range(M.shape[0]):
            for i in range(N):
                for j in range(N):
                    f.write(f"M {p} {i * N + j} {float(M[p, i, j].real)!r} {float(M[p, i, j].imag)!r}\n")


if __name__ == "__main__":
    for c in CASES:
        write(*c)
