"""Seeded synthetic inputs for the LapH block contraction.

This module only makes inputs: momentum lists and colour-vector fields.  It
holds none of the block arithmetic, imports nothing else from this package
and is shared by the CUDA path's tests/benchmark and by the oracle's tests.

The paper's gauge ensembles (64^3 x 192 and 96^3 x 192, section
"Performance Measurement Method") and the LapH eigenvectors computed on them
are not available, so the vectors (and, for the Laplacian eigensolver, the
gauge links) are stand-ins with the same shapes:
complex Gaussian entries (re, im ~ N(0,1), numpy PCG64), orthonormalised over
the combined (site, colour) index in FP64 -- the result equals Gram-Schmidt
applied in vector order -- and cast to complex64.  Layout: [T][N][L^3][3],
site index x = x0 + L*x1 + L*L*x2.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

SEED_BASE = 20251026


def momentum_shell(n2max: int) -> np.ndarray:
    """All integer momenta n with |n|^2 <= n2max, ordered by |n|^2 then lexicographically.

    Shell sizes: n2max = 0, 1, 2, 3, 4 give 1, 7, 19, 27, 33 momenta.
    """
    r = int(np.floor(np.sqrt(n2max)))
    pts = [n for n in itertools.product(range(-r, r + 1), repeat=3) if sum(c * c for c in n) <= n2max]
    pts.sort(key=lambda n: (sum(c * c for c in n), n))
    return np.asarray(pts, dtype=np.int32).reshape(-1, 3)


def momenta_for_count(P: int) -> np.ndarray:
    """The smallest full shell with P momenta (P in {1, 7, 19, 27, 33})."""
    for n2 in range(0, 5):
        m = momentum_shell(n2)
        if m.shape[0] == P:
            return m
    raise ValueError(f"no momentum shell has {P} momenta")


def seed_for(instance: int, t: int) -> int:
    return SEED_BASE + 1000 * instance + t


def orthonormal_columns(z: np.ndarray) -> np.ndarray:
    """Orthonormalise the columns of z (FP64 complex) in order.

    Householder QR, then each column is rotated by the phase of R's diagonal
    entry so that R has a positive real diagonal: this is the unique
    factorisation that Gram-Schmidt produces.
    """
    q, r = np.linalg.qr(z, mode="reduced")
    d = np.diag(r)
    ph = d / np.abs(d)
    return q * ph[None, :]


def random_phi_timeslice(L: int, N: int, seed: int, orthonormal: bool = True) -> np.ndarray:
    """complex64 [N][L^3][3] for one timeslice."""
    V = L ** 3
    if N > 3 * V and orthonormal:
        raise ValueError("cannot orthonormalise more than 3*L^3 vectors")
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((3 * V, N)) + 1j * rng.standard_normal((3 * V, N))
    if orthonormal:
        z = orthonormal_columns(z)
    # column n is vector n flattened over (site, colour) with index 3*x + a
    return np.ascontiguousarray(z.T.reshape(N, V, 3)).astype(np.complex64)


def random_phi(L: int, N: int, T: int = 1, instance: int = 0, orthonormal: bool = True,
               t0: int = 0) -> np.ndarray:
    """complex64 [T][N][L^3][3]; timeslice t uses seed SEED_BASE + 1000*instance + (t0 + t)."""
    V = L ** 3
    out = np.empty((T, N, V, 3), dtype=np.complex64)
    for t in range(T):
        out[t] = random_phi_timeslice(L, N, seed_for(instance, t0 + t), orthonormal)
    return out


@dataclass(frozen=True)
class Instance:
    """One independent problem of a ragged batch."""
    L: int
    T: int
    N: int
    momenta: np.ndarray

    @property
    def P(self) -> int:
        return int(self.momenta.shape[0])

    @property
    def V(self) -> int:
        return self.L ** 3


def ragged_instances(count: int = 200, seed: int = SEED_BASE, Ls=(16, 24, 32), Nrange=(24, 96),
                     Pset=(1, 7, 19, 33), Trange=(1, 8)) -> list[Instance]:
    """Ragged batch: L from Ls, N uniform in Nrange, P from Pset, T uniform in Trange."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        L = int(rng.choice(Ls))
        N = int(rng.integers(Nrange[0], Nrange[1] + 1))
        P = int(rng.choice(Pset))
        T = int(rng.integers(Trange[0], Trange[1] + 1))
        out.append(Instance(L=L, T=T, N=N, momenta=momenta_for_count(P)))
    return out


def plane_wave_phi(L: int, qs, us) -> np.ndarray:
    """complex64/complex128 test fields phi_i^a(x) = exp(+2 pi i q_i.x / L) u_i^a / sqrt(V).

    qs: [N][3] integer wave vectors, us: [N][3] complex colour spinors.
    Returned as complex128 [N][V][3].
    """
    V = L ** 3
    x = np.arange(V)
    xc = np.stack([x % L, (x // L) % L, x // (L * L)], axis=1)  # [V][3]
    qs = np.asarray(qs).reshape(-1, 3)
    us = np.asarray(us, dtype=np.complex128).reshape(-1, 3)
    ang = 2.0 * np.pi * (xc @ qs.T) / L  # [V][N]
    wave = np.exp(1j * ang).T / np.sqrt(V)  # [N][V]
    return wave[:, :, None] * us[:, None, :]


def random_su3(n: int, rng: np.random.Generator) -> np.ndarray:
    """n seeded SU(3) matrices, complex128 [n][3][3]: QR of a complex Gaussian (phases of R's diagonal
    removed, which makes Q Haar-distributed in U(3)), then divided by a cube root of the determinant."""
    z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


def random_links(L: int, T: int = 1, instance: int = 0, eps: float | None = None) -> np.ndarray:
    """Seeded gauge links complex64 [T][3][L^3][3][3]: U_mu(x) for the three spatial directions mu.

    eps None: independent Haar-like SU(3) links (a maximally rough field).  eps > 0: links
    exp(i eps H) built from the polar part of 1 + i eps H for Hermitian Gaussian H, i.e. a field close
    to the identity, smoother like a smeared gauge field.
    """
    V = L ** 3
    out = np.empty((T, 3, V, 3, 3), dtype=np.complex64)
    for t in range(T):
        rng = np.random.default_rng(seed_for(1000 + instance, t))
        if eps is None:
            out[t] = random_su3(3 * V, rng).reshape(3, V, 3, 3)
        else:
            h = rng.standard_normal((3 * V, 3, 3)) + 1j * rng.standard_normal((3 * V, 3, 3))
            h = 0.5 * (h + np.conj(np.transpose(h, (0, 2, 1))))
            m = np.eye(3)[None] + 1j * eps * h
            u, _, vh = np.linalg.svd(m)
            q = u @ vh
            det = np.linalg.det(q)
            out[t] = (q / (det ** (1.0 / 3.0))[:, None, None]).reshape(3, V, 3, 3)
    return out


def random_links_device(L: int, T: int, eps: float, seed: int, device="cuda"):
    """Smoothed links of the same distribution as random_links(eps=eps), drawn on the device with torch's
    generator (other numbers than the numpy path, for large benchmark inputs).  The polar factor of
    M = 1 + i eps H (H Hermitian Gaussian) is unique, so it is computed by the Newton-Schulz iteration
    X <- X (3 - X^dagger X) / 2 from X = M / |M|_F (singular values in (0, 1], converging to 1), using batched
    3 x 3 products only; then divided by a cube root of its determinant.  complex64 [T][3][L^3][3][3]."""
    import torch
    V = L ** 3
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty((T, 3, V, 3, 3), dtype=torch.complex64, device=device)
    eye = torch.eye(3, dtype=torch.complex128, device=device)
    for t in range(T):
        h = torch.view_as_complex(torch.randn((3 * V, 3, 3, 2), generator=g, device=device, dtype=torch.float64))
        h = 0.5 * (h + h.conj().transpose(1, 2))
        x = eye + 1j * eps * h
        x = x / torch.linalg.vector_norm(x, dim=(1, 2))[:, None, None]
        for _ in range(40):
            x = 0.5 * x @ (3.0 * eye - x.conj().transpose(1, 2) @ x)
        a, b, c = x[:, 0], x[:, 1], x[:, 2]
        det = (a[:, 0] * (b[:, 1] * c[:, 2] - b[:, 2] * c[:, 1]) - a[:, 1] * (b[:, 0] * c[:, 2] - b[:, 2] * c[:, 0])
               + a[:, 2] * (b[:, 0] * c[:, 1] - b[:, 1] * c[:, 0]))
        x = x * torch.exp(-1j * torch.angle(det) / 3.0)[:, None, None]
        out[t] = x.reshape(3, V, 3, 3).to(torch.complex64)
    return out
