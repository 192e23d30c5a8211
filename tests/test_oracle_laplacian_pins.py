"""Pins for the oracle's 3-d gauge-covariant Laplacian (LapH eigenvectors are its lowest modes; paper, section
"Innovations", subsection "Scalable Lanczos Eigensolver"):

    (-Delta f)(x) = sum_mu [ 2 f(x) - U_mu(x) f(x + mu) - U_mu(x - mu)^dagger f(x - mu) ]

Each test targets a plausible mistake: a dropped dagger, the backward link taken at the wrong site, a wrong
diagonal, a wrong periodic wrap, transposed colour indices.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_26313_gb300 import synth


def coords(L):
    x = np.arange(L ** 3)
    return np.stack([x % L, (x // L) % L, x // (L * L)], axis=1)


def unit_links(L):
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (3, L ** 3, 3, 3)).copy()


def gaussian(L, n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, L ** 3, 3)) + 1j * rng.standard_normal((n, L ** 3, 3))


@pytest.mark.parametrize("L", [3, 4, 5])
def test_free_field_plane_waves_are_eigenvectors_with_the_closed_form_eigenvalue(L):
    """U = 1: -Delta e^{2 pi i k.x/L} u = sum_mu 4 sin^2(pi k_mu / L) e^{2 pi i k.x/L} u."""
    rng = np.random.default_rng(L)
    for k in [(0, 0, 0), (1, 0, 0), (0, 2, 1), (L - 1, 1, 3 % L)]:
        u = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        f = np.exp(2j * np.pi * (coords(L) @ np.array(k)) / L)[:, None] * u[None, :]
        lam = sum(4 * np.sin(np.pi * kk / L) ** 2 for kk in k)
        np.testing.assert_allclose(O.laplacian(unit_links(L), f, L), lam * f, atol=1e-12)


def test_free_field_spectrum_closed_form():
    L = 4
    w = np.linalg.eigvalsh(O.laplacian_matrix(unit_links(L), L))
    ks = [(a, b, c) for a in range(L) for b in range(L) for c in range(L)]
    ref = np.sort(np.repeat([sum(4 * np.sin(np.pi * k / L) ** 2 for k in kk) for kk in ks], 3))
    np.testing.assert_allclose(w, ref, atol=1e-12)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_hermitian_and_positive_on_rough_links(L):
    U = synth.random_links(L, instance=L)[0]
    f, g = gaussian(L, 2, 7 + L)
    lhs = np.vdot(f, O.laplacian(U, g, L))
    rhs = np.vdot(O.laplacian(U, f, L), g)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    w = np.linalg.eigvalsh(O.laplacian_matrix(U, L))
    assert w.min() > -1e-12 and w.max() < 12 + 1e-12


def test_gauge_covariance():
    """U'_mu(x) = g(x) U_mu(x) g(x + mu)^dagger, f'(x) = g(x) f(x)  =>  -Delta' f' = g (-Delta f)."""
    L = 4
    V = L ** 3
    rng = np.random.default_rng(3)
    U = synth.random_links(L, instance=9)[0].astype(np.complex128)
    g = synth.random_su3(V, rng)
    c = coords(L)
    Up = np.empty_like(U)
    for mu in range(3):
        step = np.zeros(3, dtype=int)
        step[mu] = 1
        up = ((c + step) % L) @ np.array([1, L, L * L])
        Up[mu] = g @ U[mu] @ np.conj(np.transpose(g[up], (0, 2, 1)))
    f = gaussian(L, 1, 11)[0]
    fp = np.einsum("xab,xb->xa", g, f)
    np.testing.assert_allclose(O.laplacian(Up, fp, L), np.einsum("xab,xb->xa", g, O.laplacian(U, f, L)),
                               atol=1e-11 * np.abs(f).max())


def test_translation_covariance():
    L = 4
    U = synth.random_links(L, instance=4)[0]
    f = gaussian(L, 1, 5)[0]
    a = np.array([1, 3, 2])
    src = ((coords(L) + a) % L) @ np.array([1, L, L * L])
    np.testing.assert_allclose(O.laplacian(U[:, src], f[src], L), O.laplacian(U, f, L)[src], atol=1e-11)


def test_lowest_eigenpairs_satisfy_the_eigen_equation_and_free_field_zero_modes():
    L = 3
    U = synth.random_links(L, instance=2, eps=0.3)[0]
    w, v = O.lowest_eigenpairs(U, L, 6)
    assert np.all(np.diff(w) >= -1e-12)
    for lam, x in zip(w, v):
        np.testing.assert_allclose(O.laplacian(U, x, L), lam * x, atol=1e-10)
    w0, v0 = O.lowest_eigenpairs(unit_links(L), L, 4)
    np.testing.assert_allclose(w0[:3], 0.0, atol=1e-12)           # constant colour vectors
    assert w0[3] > 1.0                                             # then 4 sin^2(pi / 3) = 3
