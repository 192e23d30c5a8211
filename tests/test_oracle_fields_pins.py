"""Pins for the oracle's three-field triplets, two-field doublets and projection.

    B3[p][i][j][k] = sum_x ph_p(x) eps_abc phi_i^a(x) psi_j^b(x) chi_k^c(x)   (dense, no symmetry)
    M2[p][i][j]    = sum_x ph_p(x) sum_a conj(phi_i^a(x)) psi_j^a(x)
    Pr[p][i][j]    = the same with Nv vectors v and Ns vectors s (subsection
                     "Eigenvector Projection": at n = 0 the inner products <v_i, s_j>)

The same contractions as the LapH baryon/meson blocks, of different sets of
colour vectors (e.g. stochastic-LapH quark sinks; paper, section
"Innovations", subsection "QUDA").  Each test targets a plausible mistake: a
field bound to the wrong index, a conjugation on the wrong field, a wrong
epsilon sign, a transposed or misindexed dense output.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_26313_gb300 import synth

MOMS = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [-1, 0, 2], [1, -1, 1]], dtype=np.int32)


def coords(L):
    x = np.arange(L ** 3)
    return np.stack([x % L, (x // L) % L, x // (L * L)], axis=1)


def np_phase(L, mom):
    return np.exp(-2j * np.pi * (np.asarray(mom).reshape(-1, 3) @ coords(L).T) / L)


def fields(L, N, seed, n=3):
    rng = np.random.default_rng(seed)
    V = L ** 3
    return [rng.standard_normal((N, V, 3)) + 1j * rng.standard_normal((N, V, 3)) for _ in range(n)]


@pytest.mark.parametrize("L,N", [(2, 4), (3, 3)])
def test_triplet_matches_numpy_determinant_on_every_index_triple(L, N):
    """eps_abc u^a v^b w^c = det[u v w] (library routine), for all (i, j, k) including repeats."""
    phi, psi, chi = fields(L, N, 40 + L)
    ph = np_phase(L, MOMS)
    B = O.triplet_blocks(phi, psi, chi, L, MOMS)
    for i, j, k in itertools.product(range(N), repeat=3):
        d = np.linalg.det(np.stack([phi[i], psi[j], chi[k]], axis=2))
        np.testing.assert_allclose(B[:, i, j, k], ph @ d, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("L,N", [(2, 5), (3, 4)])
def test_doublet_matches_numpy_einsum(L, N):
    phi, psi = fields(L, N, 50 + L, n=2)
    ph = np_phase(L, MOMS)
    M = O.doublet_blocks(phi, psi, L, MOMS)
    ref = np.einsum("px,ixa,jxa->pij", ph, phi.conj(), psi)
    np.testing.assert_allclose(M, ref, rtol=1e-12, atol=1e-12)


def test_one_field_reduces_to_the_baryon_and_meson_blocks():
    L, N = 2, 6
    (phi,) = fields(L, N, 3, n=1)
    B3 = O.triplet_blocks(phi, phi, phi, L, MOMS)
    dense = O.baryon_dense(O.baryon_blocks(phi, L, MOMS), N)
    np.testing.assert_allclose(B3, dense, rtol=1e-12, atol=1e-12 * np.abs(dense).max())
    np.testing.assert_allclose(O.doublet_blocks(phi, phi, L, MOMS), O.meson_blocks(phi, L, MOMS), rtol=1e-13,
                               atol=1e-13)


def test_triplet_changes_sign_when_two_fields_swap_with_their_indices():
    L, N = 3, 4
    phi, psi, chi = fields(L, N, 61)
    B = O.triplet_blocks(phi, psi, chi, L, MOMS)
    scale = np.abs(B).max()
    # (phi, psi) swapped: [p][j][i][k] of the swapped call
    B12 = O.triplet_blocks(psi, phi, chi, L, MOMS)
    np.testing.assert_allclose(B12.transpose(0, 2, 1, 3), -B, rtol=1e-12, atol=1e-12 * scale)
    # (phi, chi) swapped
    B13 = O.triplet_blocks(chi, psi, phi, L, MOMS)
    np.testing.assert_allclose(B13.transpose(0, 3, 2, 1), -B, rtol=1e-12, atol=1e-12 * scale)
    # cyclic shift keeps the sign
    Bc = O.triplet_blocks(psi, chi, phi, L, MOMS)
    np.testing.assert_allclose(Bc.transpose(0, 3, 1, 2), B, rtol=1e-12, atol=1e-12 * scale)


def test_linear_in_every_field():
    """A conjugated field would make the blocks antilinear in it."""
    L, N = 2, 3
    phi, psi, chi = fields(L, N, 71)
    phi2, psi2, chi2 = fields(L, N, 72)
    a, b = 0.7 - 1.3j, -0.4 + 0.9j
    for pos in range(3):
        f1, f2 = [phi, psi, chi], [phi, psi, chi]
        f1[pos] = [phi2, psi2, chi2][pos]
        mix = list(f1)
        mix[pos] = a * [phi, psi, chi][pos] + b * f1[pos]
        lhs = O.triplet_blocks(*mix, L, MOMS)
        rhs = a * O.triplet_blocks(*f2, L, MOMS) + b * O.triplet_blocks(*f1, L, MOMS)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-11, atol=1e-11 * np.abs(rhs).max())
    # doublet: antilinear in phi, linear in psi
    lhs = O.doublet_blocks(a * phi + b * phi2, psi, L, MOMS)
    rhs = np.conj(a) * O.doublet_blocks(phi, psi, L, MOMS) + np.conj(b) * O.doublet_blocks(phi2, psi, L, MOMS)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())
    lhs = O.doublet_blocks(phi, a * psi + b * psi2, L, MOMS)
    rhs = a * O.doublet_blocks(phi, psi, L, MOMS) + b * O.doublet_blocks(phi, psi2, L, MOMS)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())


def test_doublet_swapped_fields_give_the_conjugate_transpose_at_opposite_momentum():
    L, N = 4, 4
    phi, psi = fields(L, N, 81, n=2)
    mom = np.array([[1, 0, 0], [-1, 0, 0], [1, -1, 2], [-1, 1, -2]], dtype=np.int32)
    M = O.doublet_blocks(phi, psi, L, mom)
    Ms = O.doublet_blocks(psi, phi, L, mom)
    np.testing.assert_allclose(Ms[1], M[0].conj().T, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Ms[3], M[2].conj().T, rtol=1e-12, atol=1e-12)
    # and the doublet of two different fields is not Hermitian (negative control)
    assert np.abs(M[0] - M[1].conj().T).max() > 1e-3 * np.abs(M).max()


def test_plane_waves_closed_form():
    """phi_i = e^{2 pi i q_i.x/L} u_i / sqrt(V), psi_j, chi_k likewise with their own momenta:
    B3[p]_ijk = V^-1/2 delta(q_i + r_j + s_k = n_p mod L) det[u_i v_j w_k],
    M2[p]_ij = delta(r_j - q_i = n_p mod L) <u_i, v_j>."""
    L = 4
    V = L ** 3
    rng = np.random.default_rng(15)
    q = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 1], [3, 0, 0]])
    r = np.array([[0, 0, 0], [0, 1, 0], [1, 0, 0], [0, 0, 3]])
    s = np.array([[0, 0, 1], [0, 0, 0], [1, 1, 0], [0, 3, 0]])
    N = 4
    u, v, w = (rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3)) for _ in range(3))
    phi, psi, chi = synth.plane_wave_phi(L, q, u), synth.plane_wave_phi(L, r, v), synth.plane_wave_phi(L, s, w)
    mom = synth.momentum_shell(2)
    B = O.triplet_blocks(phi, psi, chi, L, mom)
    M = O.doublet_blocks(phi, psi, L, mom)
    hits_B = hits_M = 0
    for p, n in enumerate(mom):
        for i, j, k in itertools.product(range(N), repeat=3):
            hit = np.all((q[i] + r[j] + s[k] - n) % L == 0)
            ref = np.linalg.det(np.stack([u[i], v[j], w[k]], axis=1)) / np.sqrt(V) if hit else 0.0
            hits_B += hit
            assert abs(B[p, i, j, k] - ref) < 1e-12
        for i, j in itertools.product(range(N), repeat=2):
            hit = np.all((r[j] - q[i] - n) % L == 0)
            ref = np.vdot(u[i], v[j]) if hit else 0.0
            hits_M += hit
            assert abs(M[p, i, j] - ref) < 1e-12
    assert hits_B >= 8 and hits_M >= 6          # the closed form is not vacuous


def test_translation_multiplies_blocks_by_phase():
    L, N = 4, 3
    phi, psi, chi = fields(L, N, 91)
    a = np.array([2, 1, 3])
    src = ((coords(L) + a) % L) @ np.array([1, L, L * L])
    fac = np.exp(2j * np.pi * (MOMS @ a) / L)
    B0 = O.triplet_blocks(phi, psi, chi, L, MOMS)
    B1 = O.triplet_blocks(phi[:, src], psi[:, src], chi[:, src], L, MOMS)
    np.testing.assert_allclose(B1, fac[:, None, None, None] * B0, rtol=1e-11, atol=1e-11 * np.abs(B0).max())
    M0 = O.doublet_blocks(phi, psi, L, MOMS)
    M1 = O.doublet_blocks(phi[:, src], psi[:, src], L, MOMS)
    np.testing.assert_allclose(M1, fac[:, None, None] * M0, rtol=1e-11, atol=1e-11 * np.abs(M0).max())


def test_triples_form_matches_dense_form():
    L, N = 2, 4
    phi, psi, chi = fields(L, N, 101)
    B = O.triplet_blocks(phi, psi, chi, L, MOMS)
    ijk = [(3, 0, 2), (1, 1, 1), (0, 3, 3), (2, 1, 0)]
    got = O.triplet_triples(phi, psi, chi, L, MOMS, ijk)
    for n, (i, j, k) in enumerate(ijk):
        np.testing.assert_allclose(got[n], B[:, i, j, k], rtol=0, atol=0)


# ----------------------------------------------------------------- projection

@pytest.mark.parametrize("L,Nv,Ns", [(2, 3, 7), (3, 6, 2)])
def test_projection_matches_numpy_einsum(L, Nv, Ns):
    rng = np.random.default_rng(110 + L)
    V = L ** 3
    v = rng.standard_normal((Nv, V, 3)) + 1j * rng.standard_normal((Nv, V, 3))
    s = rng.standard_normal((Ns, V, 3)) + 1j * rng.standard_normal((Ns, V, 3))
    ph = np_phase(L, MOMS)
    got = O.projection(v, s, L, MOMS)
    np.testing.assert_allclose(got, np.einsum("px,ixa,jxa->pij", ph, v.conj(), s), rtol=1e-12, atol=1e-12)
    # the plain inner products at n = 0
    np.testing.assert_allclose(O.projection(v, s, L)[0], np.einsum("ixa,jxa->ij", v.conj(), s), rtol=1e-12,
                               atol=1e-12)


def test_projection_recovers_the_coefficients_of_an_orthonormal_expansion():
    """s_j = sum_i C_ij v_i with orthonormal v  =>  <v_i, s_j> = C_ij (closed form)."""
    L, Nv, Ns = 4, 10, 6
    v = synth.random_phi(L, Nv, T=1, instance=3)[0].astype(np.complex128)
    rng = np.random.default_rng(7)
    C = rng.standard_normal((Nv, Ns)) + 1j * rng.standard_normal((Nv, Ns))
    s = np.einsum("ij,ixa->jxa", C, v)
    got = O.projection(v, s, L)[0]
    np.testing.assert_allclose(got, C, atol=1e-5 * np.abs(C).max())   # v is orthonormal to the complex64 cast
    # and a vector orthogonal to every v_i projects to zero
    w = rng.standard_normal((1, L ** 3, 3)) + 1j * rng.standard_normal((1, L ** 3, 3))
    w -= np.einsum("i,ixa->xa", np.einsum("ixa,xa->i", v.conj(), w[0]), v)[None]
    assert np.abs(O.projection(v, w, L)).max() < 1e-5 * np.linalg.norm(w)
