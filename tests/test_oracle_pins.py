"""Pins for the FP64 oracle: results fixed by mathematics, not by the oracle itself.

Each test targets a plausible mistake: a wrong epsilon sign or dropped term,
a conjugation on the wrong index, a wrong phase sign or site ordering, a
packing error, a normalisation factor.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_26313_gb300 import synth


def coords(L):
    x = np.arange(L ** 3)
    return np.stack([x % L, (x // L) % L, x // (L * L)], axis=1)


def np_phase(L, mom):
    """exp(-2 pi i n.x / L) with numpy, no reduction mod L."""
    return np.exp(-2j * np.pi * (np.asarray(mom).reshape(-1, 3) @ coords(L).T) / L)


def gaussian_phi(L, N, seed):
    rng = np.random.default_rng(seed)
    V = L ** 3
    return rng.standard_normal((N, V, 3)) + 1j * rng.standard_normal((N, V, 3))


def sorted_triples(N):
    return [(i, j, k) for k in range(N) for j in range(k) for i in range(j)]


def colex(i, j, k):
    return math.comb(k, 3) + math.comb(j, 2) + i


MOMS = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [-1, 0, 2], [1, -1, 1]], dtype=np.int32)


# ---------------------------------------------------------------- phase table

def test_phase_table_closed_form_values():
    L = 4
    mom = np.array([[1, 0, 0], [0, 1, 0], [1, 1, 1], [-1, 0, 0]], dtype=np.int32)
    ph = O.phase_table(L, mom)
    x100 = 1            # (1,0,0)
    x010 = L            # (0,1,0)
    x111 = 1 + L + L * L
    assert abs(ph[0, x100] - (-1j)) < 1e-15
    assert abs(ph[1, x010] - (-1j)) < 1e-15
    assert abs(ph[2, x111] - (1j)) < 1e-15       # r = 3: exp(-3 pi i / 2) = +i
    assert abs(ph[3, x100] - (1j)) < 1e-15       # r = -1 mod 4 = 3
    assert abs(ph[0, 0] - 1) < 1e-15


@pytest.mark.parametrize("L", [2, 3, 5, 8])
def test_phase_table_matches_unreduced_exponential(L):
    ph = O.phase_table(L, MOMS)
    np.testing.assert_allclose(ph, np_phase(L, MOMS), atol=1e-13)


# ---------------------------------------------------- brute force, tiny lattices

@pytest.mark.parametrize("L,N", [(2, 6), (3, 5)])
def test_baryon_matches_numpy_determinant(L, N):
    """eps_abc u^a v^b w^c is the 3x3 determinant det[u v w] (library routine)."""
    phi = gaussian_phi(L, N, 11 + L)
    ph = np_phase(L, MOMS)
    B = O.baryon_blocks(phi, L, MOMS)
    for (i, j, k) in sorted_triples(N):
        mats = np.stack([phi[i], phi[j], phi[k]], axis=2)  # [V][colour][vector]
        d = np.linalg.det(mats)                           # [V]
        ref = ph @ d
        np.testing.assert_allclose(B[:, colex(i, j, k)], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("L,N", [(2, 5), (3, 4)])
def test_meson_matches_numpy_einsum(L, N):
    phi = gaussian_phi(L, N, 7 + L)
    ph = np_phase(L, MOMS)
    M = O.meson_blocks(phi, L, MOMS)
    ref = np.einsum("px,ixa,jxa->pij", ph, phi.conj(), phi)
    np.testing.assert_allclose(M, ref, rtol=1e-12, atol=1e-12)


def test_packed_equals_triple_form_and_dense_fill():
    L, N = 2, 6
    phi = gaussian_phi(L, N, 3)
    B = O.baryon_blocks(phi, L, MOMS)
    allijk = list(itertools.product(range(N), repeat=3))
    Bt = O.baryon_triples(phi, L, MOMS, allijk)          # [N^3][P]
    dense = O.baryon_dense(B, N)                         # [P][N][N][N]
    for n, (a, b, c) in enumerate(allijk):
        np.testing.assert_allclose(dense[:, a, b, c], Bt[n], rtol=1e-12, atol=1e-12)
    for (i, j, k) in sorted_triples(N):
        np.testing.assert_allclose(B[:, colex(i, j, k)], Bt[(i * N + j) * N + k], rtol=0, atol=0)


def test_diquarks_match_numpy_cross_product():
    L, N = 3, 5
    phi = gaussian_phi(L, N, 13)
    D = O.diquarks(phi, L)
    for j in range(N):
        for i in range(j):
            q = j * (j - 1) // 2 + i
            np.testing.assert_allclose(D[q], np.cross(phi[i], phi[j]), rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------------- symmetries

def test_baryon_antisymmetric_under_every_swap_and_zero_on_repeats():
    L, N = 3, 5
    phi = gaussian_phi(L, N, 5)
    base = O.baryon_triples(phi, L, MOMS, [(0, 2, 4)])[0]
    scale = np.abs(base).max()
    for perm, sign in [((0, 2, 4), 1), ((2, 0, 4), -1), ((0, 4, 2), -1), ((4, 2, 0), -1),
                       ((2, 4, 0), 1), ((4, 0, 2), 1)]:
        got = O.baryon_triples(phi, L, MOMS, [perm])[0]
        np.testing.assert_allclose(got, sign * base, rtol=1e-13, atol=1e-13 * scale)
    rep = O.baryon_triples(phi, L, MOMS, [(1, 1, 3), (3, 1, 3), (2, 2, 2)])
    assert np.abs(rep).max() < 1e-13 * scale


def test_vector_permutation_maps_packed_blocks_with_sign():
    """Relabelling the vectors permutes B with the sign of the sort permutation."""
    L, N = 2, 6
    phi = gaussian_phi(L, N, 21)
    perm = np.array([3, 0, 5, 1, 4, 2])                  # new vector n = old vector perm[n]
    B = O.baryon_blocks(phi, L, MOMS)
    Bp = O.baryon_blocks(phi[perm], L, MOMS)
    for (i, j, k) in sorted_triples(N):
        old = [perm[i], perm[j], perm[k]]
        s = np.argsort(old)
        sign = np.linalg.det(np.eye(3)[s])               # sign of the sorting permutation
        o = sorted(old)
        np.testing.assert_allclose(Bp[:, colex(i, j, k)], sign * B[:, colex(*o)], rtol=1e-12, atol=1e-12)


def test_meson_hermitian_relation_between_opposite_momenta():
    L, N = 4, 5
    phi = gaussian_phi(L, N, 9)
    mom = np.array([[1, 0, 0], [-1, 0, 0], [1, -1, 2], [-1, 1, -2], [0, 0, 0]], dtype=np.int32)
    M = O.meson_blocks(phi, L, mom)
    np.testing.assert_allclose(M[1], M[0].conj().T, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(M[3], M[2].conj().T, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(M[4], M[4].conj().T, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------- orthonormal inputs

def test_orthonormal_vectors_give_identity_meson_block_at_zero_momentum():
    L, N = 4, 12
    phi = synth.random_phi(L, N, T=1)[0].astype(np.complex128)
    M = O.meson_blocks(phi, L, MOMS[:2])
    np.testing.assert_allclose(M[0], np.eye(N), atol=1e-6)   # c64 cast limits this to ~1e-7
    assert np.abs(M[1]).max() < 0.5                          # p != 0 is not the identity


def test_complete_basis_norms():
    """N = 3V orthonormal vectors form a unitary Phi; Parseval fixes these sums."""
    L = 2
    V = L ** 3
    rng = np.random.default_rng(77)
    z = rng.standard_normal((3 * V, 3 * V)) + 1j * rng.standard_normal((3 * V, 3 * V))
    q = synth.orthonormal_columns(z)                      # FP64 unitary
    phi = np.ascontiguousarray(q.T.reshape(3 * V, V, 3))
    mom = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 1], [0, 1, 1]], dtype=np.int32)
    B = O.baryon_blocks(phi, L, mom)
    M = O.meson_blocks(phi, L, mom)
    for p in range(mom.shape[0]):
        assert abs(np.sum(np.abs(B[p]) ** 2) - V) < 1e-10
        assert abs(np.sum(np.abs(M[p]) ** 2) - 3 * V) < 1e-10
        tr = np.trace(M[p])
        assert abs(tr - (3 * V if p == 0 else 0)) < 1e-10


# ---------------------------------------------------------------- closed forms

def test_plane_waves_closed_form():
    """phi_i = exp(2 pi i q_i.x/L) u_i / sqrt(V):
    M[p]_ij = delta(q_j - q_i = n_p mod L) <u_i,u_j>,
    B[p]_ijk = V^-1/2 delta(q_i + q_j + q_k = n_p mod L) det[u_i u_j u_k]."""
    L = 4
    V = L ** 3
    rng = np.random.default_rng(5)
    qs = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 1], [0, 0, 1], [1, 1, 0], [3, 0, 0]])
    N = qs.shape[0]
    us = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
    phi = synth.plane_wave_phi(L, qs, us)
    mom = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [-1, 0, 1], [2, 0, 0],
                    [0, 1, 1], [1, 0, 1]], dtype=np.int32)
    B = O.baryon_blocks(phi, L, mom)
    M = O.meson_blocks(phi, L, mom)
    hits_B = hits_M = 0
    for p, n in enumerate(mom):
        for i in range(N):
            for j in range(N):
                hit = np.all((qs[j] - qs[i] - n) % L == 0)
                ref = np.vdot(us[i], us[j]) if hit else 0.0
                hits_M += hit
                assert abs(M[p, i, j] - ref) < 1e-12
        for (i, j, k) in sorted_triples(N):
            hit = np.all((qs[i] + qs[j] + qs[k] - n) % L == 0)
            ref = np.linalg.det(np.stack([us[i], us[j], us[k]], axis=1)) / np.sqrt(V) if hit else 0.0
            hits_B += hit
            assert abs(B[p, colex(i, j, k)] - ref) < 1e-12
    assert hits_B >= 5 and hits_M >= 10          # the closed form is not vacuous


def test_delta_vectors_closed_form():
    """phi_i = unit vector at (site x_i, colour a_i): B is ph_p(x) eps_{a_i a_j a_k} when the
    three vectors sit on one site, else 0; M[p]_ij = ph_p(x_i) delta_ij-site-and-colour."""
    L = 3
    V = L ** 3
    sites = [5, 5, 5, 7, 7, 20, 5]
    cols = [0, 1, 2, 2, 0, 1, 0]
    N = len(sites)
    phi = np.zeros((N, V, 3), dtype=np.complex128)
    for n, (x, a) in enumerate(zip(sites, cols)):
        phi[n, x, a] = 1.0
    ph = np_phase(L, MOMS)
    B = O.baryon_blocks(phi, L, MOMS)
    M = O.meson_blocks(phi, L, MOMS)
    eps = np.zeros((3, 3, 3))
    for (a, b, c) in itertools.permutations(range(3)):
        eps[a, b, c] = np.linalg.det(np.eye(3)[[a, b, c]])
    for (i, j, k) in sorted_triples(N):
        same = sites[i] == sites[j] == sites[k]
        ref = ph[:, sites[i]] * eps[cols[i], cols[j], cols[k]] if same else np.zeros(len(MOMS))
        np.testing.assert_allclose(B[:, colex(i, j, k)], ref, atol=1e-14)
    for i in range(N):
        for j in range(N):
            same = sites[i] == sites[j] and cols[i] == cols[j]
            ref = ph[:, sites[i]] if same else np.zeros(len(MOMS))
            np.testing.assert_allclose(M[:, i, j], ref, atol=1e-14)


# -------------------------------------------------------------- invariances

def random_unitary3(rng, n):
    z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    return q * (d / np.abs(d))[:, None, :]


def test_su3_rotation_invariance_and_u3_negative_control():
    L, N = 3, 6
    V = L ** 3
    rng = np.random.default_rng(31)
    phi = gaussian_phi(L, N, 8)
    U = random_unitary3(rng, V)                               # U(3) per site
    det = np.linalg.det(U)
    Usu3 = U / (det ** (1.0 / 3.0))[:, None, None]            # det = 1
    assert np.allclose(np.linalg.det(Usu3), 1.0)
    rot = np.einsum("xab,nxb->nxa", Usu3, phi)
    B0, M0 = O.baryon_blocks(phi, L, MOMS), O.meson_blocks(phi, L, MOMS)
    B1, M1 = O.baryon_blocks(rot, L, MOMS), O.meson_blocks(rot, L, MOMS)
    np.testing.assert_allclose(B1, B0, rtol=1e-11, atol=1e-11 * np.abs(B0).max())
    np.testing.assert_allclose(M1, M0, rtol=1e-11, atol=1e-11 * np.abs(M0).max())
    # negative control: a site-dependent det phase must change B (M, unitary-invariant, must not)
    rot3 = np.einsum("xab,nxb->nxa", U, phi)
    B3, M3 = O.baryon_blocks(rot3, L, MOMS), O.meson_blocks(rot3, L, MOMS)
    assert np.abs(B3 - B0).max() > 1e-3 * np.abs(B0).max()
    np.testing.assert_allclose(M3, M0, rtol=1e-11, atol=1e-11 * np.abs(M0).max())
    # and with the det phase folded back in per site, B is recovered
    ph = np_phase(L, MOMS)
    for (i, j, k) in sorted_triples(N)[:6]:
        mats = np.stack([rot3[i], rot3[j], rot3[k]], axis=2)
        ref = ph @ np.linalg.det(mats)
        np.testing.assert_allclose(B3[:, colex(i, j, k)], ref, rtol=1e-11, atol=1e-11)


def test_translation_multiplies_blocks_by_phase():
    """phi'(x) = phi(x + a) (periodic) => blocks times exp(+2 pi i n_p.a / L)."""
    L, N = 4, 5
    phi = gaussian_phi(L, N, 4)
    a = np.array([1, 3, 2])
    c = coords(L)
    src = ((c + a) % L) @ np.array([1, L, L * L])
    shifted = phi[:, src, :]
    fac = np.exp(2j * np.pi * (MOMS @ a) / L)
    B0, M0 = O.baryon_blocks(phi, L, MOMS), O.meson_blocks(phi, L, MOMS)
    B1, M1 = O.baryon_blocks(shifted, L, MOMS), O.meson_blocks(shifted, L, MOMS)
    np.testing.assert_allclose(B1, fac[:, None] * B0, rtol=1e-11, atol=1e-11 * np.abs(B0).max())
    np.testing.assert_allclose(M1, fac[:, None, None] * M0, rtol=1e-11, atol=1e-11 * np.abs(M0).max())


# ------------------------------------------------------------- input recipe

def test_momentum_shell_sizes():
    assert [synth.momentum_shell(n).shape[0] for n in range(5)] == [1, 7, 19, 27, 33]
    m = synth.momentum_shell(2)
    n2 = (m ** 2).sum(axis=1)
    assert np.all(np.diff(n2) >= 0) and tuple(m[0]) == (0, 0, 0)


def test_generator_is_orthonormal_and_seeded():
    a = synth.random_phi(3, 10, T=2)
    b = synth.random_phi(3, 10, T=2)
    assert a.dtype == np.complex64 and a.shape == (2, 10, 27, 3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a[0], a[1])
    g = np.einsum("ixa,jxa->ij", a[0].conj().astype(np.complex128), a[0].astype(np.complex128))
    np.testing.assert_allclose(g, np.eye(10), atol=1e-6)
