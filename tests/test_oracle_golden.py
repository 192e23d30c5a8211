"""The oracle reproduces its committed regression fixtures (tests/golden/)."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_26313_gb300 import synth

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name,L,N,n2", [("L2_N4_P7", 2, 4, 1), ("L3_N5_P19", 3, 5, 2)])
def test_oracle_matches_fixture(name, L, N, n2):
    mom = synth.momentum_shell(n2)
    phi = synth.random_phi(L, N, T=1, instance=900)[0]
    B = O.baryon_blocks(phi, L, mom)
    M = O.meson_blocks(phi, L, mom).reshape(mom.shape[0], -1)
    nB = nM = 0
    with open(os.path.join(HERE, f"oracle_{name}.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            kind, p, idx, re, im = line.split()
            ref = complex(float(re), float(im))
            got = B[int(p), int(idx)] if kind == "B" else M[int(p), int(idx)]
            assert abs(got - ref) <= 1e-14 * max(1.0, abs(ref))
            nB += kind == "B"
            nM += kind == "M"
    assert nB == B.size and nM == M.size
