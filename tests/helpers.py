"""Shared helpers for the tests: error metrics and lazy builds."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Relative Frobenius bound for the FP32 and split-precision paths.
TOL_SPLIT = 1e-5
# Single-term FP16 / BF16 products: stated separately (one rounding of each
# operand to 11 / 8 significant bits).
TOL_PLAIN = {"f16": 2e-3, "bf16": 1.5e-2}


def rel_frob(got, ref) -> float:
    got = np.asarray(got)
    ref = np.asarray(ref)
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((got - ref).ravel()) / (den if den > 0 else 1.0))


def worst_slice(got, ref, axes=1) -> float:
    """Largest relative Frobenius error over the leading `axes` indices (e.g. per (t) or per (t,p))."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    lead = got.shape[:axes]
    g = got.reshape(int(np.prod(lead)), -1)
    r = ref.reshape(int(np.prod(lead)), -1)
    return max(rel_frob(g[n], r[n]) for n in range(g.shape[0]))


def tol_for(mode: str) -> float:
    return TOL_PLAIN.get(mode, TOL_SPLIT)


def ensure_built():
    from paper_2510_26313_gb300 import build
    return build.build()
