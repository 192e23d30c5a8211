"""Python access to the FP64 CPU oracle (``laph_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports,
links or runs anything in this folder.

The oracle computes, for one timeslice, the LapH meson and baryon blocks
formed from N complex colour vectors (paper, section "Innovations",
subsection "QUDA": quark-antiquark doublets and three-quark triplets built
from the LapH eigenvectors):

    B[p][i,j,k] = sum_x exp(-2 pi i ((n_p.x) mod L)/L) eps_abc phi_i^a phi_j^b phi_k^c
    M[p][i][j]  = sum_x exp(-2 pi i ((n_p.x) mod L)/L) conj(phi_i^a) phi_j^a

the same contractions of three (two) different sets of vectors, e.g.
stochastic-LapH quark sinks (same passage), the projection of one set of
vectors onto another (subsection "Eigenvector Projection"), and the 3-d
gauge-covariant Laplacian whose lowest eigenvectors are the LapH vectors
(subsection "Scalable Lanczos Eigensolver"):

    B3[p][i][j][k] = sum_x ph_p(x) eps_abc phi_i^a psi_j^b chi_k^c   (dense)
    M2[p][i][j]    = sum_x ph_p(x) conj(phi_i^a) psi_j^a

in double precision with plain loops (see ``laph_oracle.c``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "laph_oracle.c")
_LIB = os.path.join(_HERE, "liblaph_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``laph_oracle.c`` into ``liblaph_oracle.so`` (gcc, OpenMP, no fast-math).

    ``LAPH_ORACLE_LIB`` names a different, already built library instead; the
    mutation tests use it to load copies of the oracle with planted mistakes.
    """
    override = os.environ.get("LAPH_ORACLE_LIB")
    if override:
        return override
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            lib.oracle_phase_table.argtypes = [ctypes.c_int, ip, ctypes.c_int, dp]
            lib.oracle_phase_table.restype = None
            lib.oracle_baryon_triples.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int,
                                                  ctypes.c_int64, ip, dp]
            lib.oracle_baryon_triples.restype = ctypes.c_int
            lib.oracle_baryon_blocks.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, dp]
            lib.oracle_baryon_blocks.restype = ctypes.c_int
            lib.oracle_meson_blocks.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, dp]
            lib.oracle_meson_blocks.restype = ctypes.c_int
            lib.oracle_baryon_dense.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_baryon_dense.restype = None
            lib.oracle_diquarks.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_diquarks.restype = None
            lib.oracle_triplet_triples.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int,
                                                   ctypes.c_int64, ip, dp]
            lib.oracle_triplet_triples.restype = ctypes.c_int
            lib.oracle_triplet_blocks.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, dp]
            lib.oracle_triplet_blocks.restype = ctypes.c_int
            lib.oracle_doublet_blocks.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, dp]
            lib.oracle_doublet_blocks.restype = ctypes.c_int
            lib.oracle_projection.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, dp]
            lib.oracle_projection.restype = ctypes.c_int
            lib.oracle_laplacian.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_laplacian.restype = None
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _prep(phi: np.ndarray, L: int, momenta):
    phi = np.ascontiguousarray(phi, dtype=np.complex128)
    V = L ** 3
    if phi.ndim != 3 or phi.shape[1] != V or phi.shape[2] != 3:
        raise ValueError(f"phi must be [N][L^3][3], got {phi.shape} for L={L}")
    mom = np.ascontiguousarray(np.asarray(momenta, dtype=np.int32).reshape(-1, 3))
    return phi, mom


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all host cores)."""
    return int(_load().oracle_num_threads())


def phase_table(L: int, momenta) -> np.ndarray:
    """complex128 [P][L^3]: exp(-2 pi i ((n_p.x) mod L)/L)."""
    mom = np.ascontiguousarray(np.asarray(momenta, dtype=np.int32).reshape(-1, 3))
    out = np.empty((mom.shape[0], L ** 3), dtype=np.complex128)
    _load().oracle_phase_table(L, _iptr(mom), mom.shape[0], _dptr(out))
    return out


def baryon_blocks(phi: np.ndarray, L: int, momenta) -> np.ndarray:
    """Packed baryon blocks, complex128 [P][C(N,3)], colex index C(k,3)+C(j,2)+i."""
    phi, mom = _prep(phi, L, momenta)
    N = phi.shape[0]
    n3 = N * (N - 1) * (N - 2) // 6
    out = np.zeros((mom.shape[0], n3), dtype=np.complex128)
    if n3:
        rc = _load().oracle_baryon_blocks(_dptr(phi), L, N, _iptr(mom), mom.shape[0], _dptr(out))
        if rc != 0:
            raise RuntimeError("oracle_baryon_blocks failed")
    return out


def baryon_triples(phi: np.ndarray, L: int, momenta, ijk) -> np.ndarray:
    """B for arbitrary index triples (any order): complex128 [n][P]."""
    phi, mom = _prep(phi, L, momenta)
    ijk = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((ijk.shape[0], mom.shape[0]), dtype=np.complex128)
    if ijk.shape[0]:
        rc = _load().oracle_baryon_triples(_dptr(phi), L, phi.shape[0], _iptr(mom), mom.shape[0],
                                           ijk.shape[0], _iptr(ijk), _dptr(out))
        if rc != 0:
            raise RuntimeError("oracle_baryon_triples failed (bad index or allocation)")
    return out


def meson_blocks(phi: np.ndarray, L: int, momenta) -> np.ndarray:
    """Meson blocks, complex128 [P][N][N]."""
    phi, mom = _prep(phi, L, momenta)
    N = phi.shape[0]
    out = np.zeros((mom.shape[0], N, N), dtype=np.complex128)
    rc = _load().oracle_meson_blocks(_dptr(phi), L, N, _iptr(mom), mom.shape[0], _dptr(out))
    if rc != 0:
        raise RuntimeError("oracle_meson_blocks failed")
    return out


def diquarks(phi: np.ndarray, L: int) -> np.ndarray:
    """complex128 [C(N,2)][V][3]: D_q(x)_c = eps_cab phi_i^a phi_j^b, q = C(j,2)+i."""
    phi, _ = _prep(phi, L, np.zeros((1, 3), dtype=np.int32))
    N = phi.shape[0]
    out = np.zeros((N * (N - 1) // 2, L ** 3, 3), dtype=np.complex128)
    _load().oracle_diquarks(_dptr(phi), L, N, _dptr(out))
    return out


def baryon_dense(packed: np.ndarray, N: int) -> np.ndarray:
    """Dense antisymmetric tensor complex128 [P][N][N][N] from the packed form."""
    packed = np.ascontiguousarray(packed, dtype=np.complex128)
    P = packed.shape[0]
    out = np.empty((P, N, N, N), dtype=np.complex128)
    _load().oracle_baryon_dense(_dptr(packed), N, P, _dptr(out))
    return out


def _prep_fields(fields, L: int, momenta):
    out = []
    for f in fields:
        f, mom = _prep(f, L, momenta)
        out.append(f)
    if any(f.shape != out[0].shape for f in out):
        raise ValueError("the fields must have the same shape [N][L^3][3]")
    return out, mom


def triplet_blocks(phi: np.ndarray, psi: np.ndarray, chi: np.ndarray, L: int, momenta) -> np.ndarray:
    """Dense three-field triplets, complex128 [P][N][N][N]: [p][i][j][k] = sum_x ph eps phi_i psi_j chi_k."""
    (phi, psi, chi), mom = _prep_fields((phi, psi, chi), L, momenta)
    N = phi.shape[0]
    out = np.zeros((mom.shape[0], N, N, N), dtype=np.complex128)
    rc = _load().oracle_triplet_blocks(_dptr(phi), _dptr(psi), _dptr(chi), L, N, _iptr(mom), mom.shape[0],
                                       _dptr(out))
    if rc != 0:
        raise RuntimeError("oracle_triplet_blocks failed")
    return out


def triplet_triples(phi: np.ndarray, psi: np.ndarray, chi: np.ndarray, L: int, momenta, ijk) -> np.ndarray:
    """Three-field triplets for a list of (i, j, k): complex128 [n][P]."""
    (phi, psi, chi), mom = _prep_fields((phi, psi, chi), L, momenta)
    ijk = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((ijk.shape[0], mom.shape[0]), dtype=np.complex128)
    if ijk.shape[0]:
        rc = _load().oracle_triplet_triples(_dptr(phi), _dptr(psi), _dptr(chi), L, phi.shape[0], _iptr(mom),
                                            mom.shape[0], ijk.shape[0], _iptr(ijk), _dptr(out))
        if rc != 0:
            raise RuntimeError("oracle_triplet_triples failed (bad index or allocation)")
    return out


def doublet_blocks(phi: np.ndarray, psi: np.ndarray, L: int, momenta) -> np.ndarray:
    """Two-field doublets, complex128 [P][N][N]: [p][i][j] = sum_x ph conj(phi_i) . psi_j."""
    (phi, psi), mom = _prep_fields((phi, psi), L, momenta)
    N = phi.shape[0]
    out = np.zeros((mom.shape[0], N, N), dtype=np.complex128)
    rc = _load().oracle_doublet_blocks(_dptr(phi), _dptr(psi), L, N, _iptr(mom), mom.shape[0], _dptr(out))
    if rc != 0:
        raise RuntimeError("oracle_doublet_blocks failed")
    return out


def projection(v: np.ndarray, s: np.ndarray, L: int, momenta=((0, 0, 0),)) -> np.ndarray:
    """Projection of the vectors s onto the vectors v, complex128 [P][Nv][Ns]:
    [p][i][j] = sum_x ph_p(x) sum_a conj(v_i^a) s_j^a (n = 0: the inner products <v_i, s_j>)."""
    v, mom = _prep(v, L, momenta)
    s, _ = _prep(s, L, momenta)
    Nv, Ns = v.shape[0], s.shape[0]
    out = np.zeros((mom.shape[0], Nv, Ns), dtype=np.complex128)
    rc = _load().oracle_projection(_dptr(v), _dptr(s), L, Nv, Ns, _iptr(mom), mom.shape[0], _dptr(out))
    if rc != 0:
        raise RuntimeError("oracle_projection failed")
    return out


def laplacian(U: np.ndarray, f: np.ndarray, L: int) -> np.ndarray:
    """(-Delta f) for one timeslice: U complex [3][L^3][3][3], f complex [nvec][L^3][3] (or [L^3][3])."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    single = f.ndim == 2
    f = np.ascontiguousarray(f[None] if single else f, dtype=np.complex128)
    V = L ** 3
    if U.shape != (3, V, 3, 3) or f.shape[1:] != (V, 3):
        raise ValueError("U must be [3][L^3][3][3] and f [nvec][L^3][3]")
    out = np.empty_like(f)
    _load().oracle_laplacian(_dptr(U), _dptr(f), L, f.shape[0], _dptr(out))
    return out[0] if single else out


def laplacian_matrix(U: np.ndarray, L: int) -> np.ndarray:
    """Dense (3V x 3V) matrix of -Delta (small L only): the oracle applied to every unit vector."""
    V = L ** 3
    eye = np.eye(3 * V, dtype=np.complex128).reshape(3 * V, V, 3)
    return laplacian(U, eye, L).reshape(3 * V, 3 * V).T


def lowest_eigenpairs(U: np.ndarray, L: int, n: int):
    """The n smallest eigenvalues (ascending) and eigenvectors complex128 [n][L^3][3] of -Delta
    (small L only): numpy's Hermitian eigensolver on the dense matrix."""
    w, v = np.linalg.eigh(laplacian_matrix(U, L))
    return w[:n], v[:, :n].T.reshape(n, L ** 3, 3)


def lanczos_eigenpairs(U: np.ndarray, L: int, n_ev: int, m: int, degree: int = 0, lo: float = 0.0, seed: int = 0):
    """The n_ev lowest eigenvalues of -Delta on one timeslice by plain FP64 Lanczos (paper, section "Innovations",
    subsection "Scalable Lanczos Eigensolver"), in the conventions the GPU solver states: m steps from a seeded
    random unit vector, each new vector orthogonalised against the whole basis by two classical Gram-Schmidt passes,
    alpha_j from the first pass and beta_j the norm after the second; the operator is -Delta (this module's stencil)
    or, for degree d > 0, the Chebyshev filter T_d((-Delta - c) / e) with c = (12 + lo) / 2, e = (12 - lo) / 2;
    the Ritz vectors of the wanted end of the tridiagonal matrix's spectrum (numpy's eigh as the step: the smallest
    for d = 0, the largest for even d, the most negative for odd d); eigenvalues are Rayleigh quotients with -Delta,
    residuals |(-Delta) x - lambda x| / |x|.  U complex [3][L^3][3][3].  Returns (eigenvalues ascending, residuals)."""
    V = L ** 3
    n = 3 * V
    U = np.ascontiguousarray(U, dtype=np.complex128)
    A = lambda x: laplacian(U, x.reshape(V, 3), L).reshape(n)

    def op(v):
        if degree == 0:
            return A(v)
        c, e = 0.5 * (12.0 + lo), 0.5 * (12.0 - lo)
        y0, y1 = v, (A(v) - c * v) / e
        for _ in range(2, degree + 1):
            y0, y1 = y1, 2.0 * (A(y1) - c * y1) / e - y0
        return y1

    rng = np.random.default_rng(seed)
    Q = np.zeros((m + 1, n), dtype=np.complex128)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Q[0] = v / np.linalg.norm(v)
    alpha, beta = np.zeros(m), np.zeros(m)
    for j in range(m):
        w = op(Q[j])
        c1 = Q[: j + 1].conj() @ w
        w = w - Q[: j + 1].T @ c1
        w = w - Q[: j + 1].T @ (Q[: j + 1].conj() @ w)
        alpha[j], beta[j] = c1[j].real, np.linalg.norm(w)
        Q[j + 1] = w / beta[j]
    Tm = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    _, S = np.linalg.eigh(Tm)
    pick = np.arange(m - 1, m - 1 - n_ev, -1) if (degree > 0 and degree % 2 == 0) else np.arange(n_ev)
    X = S[:, pick].T @ Q[:m]
    AX = np.stack([A(x) for x in X])
    lam = np.einsum("ij,ij->i", X.conj(), AX).real / np.einsum("ij,ij->i", X.conj(), X).real
    res = np.linalg.norm(AX - lam[:, None] * X, axis=1) / np.linalg.norm(X, axis=1)
    order = np.argsort(lam)
    return lam[order], res[order]
