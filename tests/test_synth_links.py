"""CPU checks of the seeded gauge-link generators used as inputs by the Laplacian and Lanczos tests and benchmark.

The device generator forms the polar factor of 1 + i eps H by a Newton-Schulz iteration; the polar factor of a
nonsingular matrix is unique, so it must equal the SVD route (U V^dagger) on the same H, and both must be SU(3).
"""
import numpy as np
import pytest

from paper_2510_26313_gb300 import synth


def su3_defects(m):
    m = m.reshape(-1, 3, 3).astype(np.complex128)
    unit = np.abs(m @ np.conj(np.transpose(m, (0, 2, 1))) - np.eye(3)).max()
    det = np.abs(np.linalg.det(m) - 1).max()
    return unit, det


@pytest.mark.parametrize("eps", [None, 0.25, 0.6])
def test_numpy_links_are_su3(eps):
    unit, det = su3_defects(synth.random_links(3, 2, instance=1, eps=eps))
    assert unit < 5e-7 and det < 5e-7


def test_device_links_equal_the_svd_polar_factor_on_the_same_draws():
    torch = pytest.importorskip("torch")
    L, eps, seed = 3, 0.6, 11
    U = synth.random_links_device(L, 1, eps, seed, device="cpu").numpy()
    unit, det = su3_defects(U)
    assert unit < 5e-7 and det < 5e-7
    # redraw the same Hermitian matrices and take the polar factor through the SVD
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    h = torch.view_as_complex(torch.randn((3 * L ** 3, 3, 3, 2), generator=g, dtype=torch.float64)).numpy()
    h = 0.5 * (h + np.conj(np.transpose(h, (0, 2, 1))))
    u, _, vh = np.linalg.svd(np.eye(3)[None] + 1j * eps * h)
    q = u @ vh
    q = q / (np.linalg.det(q) ** (1.0 / 3.0))[:, None, None]
    np.testing.assert_allclose(U[0].reshape(-1, 3, 3), q, atol=2e-7)


def test_device_links_smoothness_matches_the_numpy_generator():
    """Same distribution: the mean of Re tr U / 3 over many links agrees between the two generators."""
    pytest.importorskip("torch")
    a = synth.random_links(6, 1, instance=3, eps=0.6).reshape(-1, 3, 3)
    b = synth.random_links_device(6, 1, 0.6, 5, device="cpu").numpy().reshape(-1, 3, 3)
    ta = np.trace(a, axis1=1, axis2=2).real.mean() / 3
    tb = np.trace(b, axis1=1, axis2=2).real.mean() / 3
    assert abs(ta - tb) < 0.01 and 0.5 < ta < 0.95
