"""The oracle's FP64 Lanczos (oracle.lanczos_eigenpairs, no GPU): Lanczos with two classical Gram-Schmidt passes per
step, on -Delta or on the Chebyshev filter T_d((-Delta - c) / e) that maps [lo, 12] onto [-1, 1], Ritz pairs of the
tridiagonal matrix at the wanted end (smallest for -Delta; for the filter the largest when d is even and the most
negative when d is odd), eigenvalues as Rayleigh quotients with -Delta.  Pinned against numpy's dense Hermitian
eigensolver on the oracle's dense Laplacian: it fixes the conventions the CUDA solver follows (paper, section
"Innovations", subsection "Scalable Lanczos Eigensolver", which names a batched Lanczos eigensolver and leaves these
choices open).  The negative controls apply the wrong conventions to the same problem.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_26313_gb300 import synth


def chebyshev(A, v, d, lo):
    c, e = 0.5 * (12.0 + lo), 0.5 * (12.0 - lo)
    B = lambda x: (A @ x - c * x) / e
    y0, y1 = v, B(v)
    for _ in range(2, d + 1):
        y0, y1 = y1, 2.0 * B(y1) - y0
    return y1


L6 = 6


@pytest.fixture(scope="module")
def problem():
    U = synth.random_links(L6, 1, instance=66, eps=0.6)[0]
    A = O.laplacian_matrix(U, L6)
    return A, np.linalg.eigvalsh(A), U


@pytest.mark.parametrize("d,m", [(0, 300), (7, 60), (8, 60)])
def test_oracle_lanczos_finds_the_lowest_eigenpairs(problem, d, m):
    A, w, U = problem
    n_ev = 20
    lo = 0.5 * (w[n_ev + 2] + w[n_ev + 3])          # a bound in the gap above the wanted eigenvalues
    lam, res = O.lanczos_eigenpairs(U, L6, n_ev, m, d, lo)
    np.testing.assert_allclose(lam, w[:n_ev], atol=1e-9)
    assert res.max() < 1e-6


def test_model_with_the_wrong_sign_convention_misses_them(problem):
    """For an odd degree the filter is large and negative below lo: taking the largest Ritz values, as for an even
    degree, returns pairs from the damped part of the spectrum."""
    A, w, _ = problem
    n_ev, d, m = 20, 7, 60
    lo = 0.5 * (w[n_ev + 2] + w[n_ev + 3])
    n = A.shape[0]
    rng = np.random.default_rng(0)
    Q = np.zeros((m + 1, n), dtype=np.complex128)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Q[0] = v / np.linalg.norm(v)
    alpha, beta = np.zeros(m), np.zeros(m)
    for j in range(m):
        wv = chebyshev(A, Q[j], d, lo)
        c1 = Q[: j + 1].conj() @ wv
        wv = wv - Q[: j + 1].T @ c1
        wv = wv - Q[: j + 1].T @ (Q[: j + 1].conj() @ wv)
        alpha[j], beta[j] = c1[j].real, np.linalg.norm(wv)
        Q[j + 1] = wv / beta[j]
    Tm = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    theta, S = np.linalg.eigh(Tm)
    X = S[:, m - n_ev:].T @ Q[:m]                     # the largest, wrong for odd d
    lam = np.einsum("ij,ij->i", X.conj(), X @ A.T).real / np.einsum("ij,ij->i", X.conj(), X).real
    assert np.sort(lam)[0] > w[n_ev]                   # none of them is among the wanted eigenvalues


def test_model_with_the_bound_below_the_wanted_eigenvalues_does_not_converge(problem):
    """lo must lie above the wanted eigenvalues: with lo below the 20th eigenvalue, the pairs between lo and the
    20th eigenvalue are damped like the rest of the spectrum and are not resolved."""
    _, w, U = problem
    n_ev, d, m = 20, 8, 60
    lo = 0.5 * (w[9] + w[10])
    lam, res = O.lanczos_eigenpairs(U, L6, n_ev, m, d, lo)
    assert res.max() > 1e-3 or np.abs(lam - w[:n_ev]).max() > 1e-3
