"""laph_blocks_noalloc: the allocation-free FP32 entry point.

Collected last on purpose (its scratch is a file-scope device array that
persists between calls): the GPU test calls it several times in a row, on
different shapes and output selections, through the C ABI and checks each
result against the plan-based FP32 entry points laph_baryon_blocks /
laph_meson_blocks and against the FP64 oracle.  The CPU tests check the
argument and size rejections, which happen before any CUDA call.
"""
import ctypes

import numpy as np
import pytest

from helpers import TOL_SPLIT, ensure_built, rel_frob
from paper_2510_26313_gb300 import synth

LAPH_ERR_ARG = -1
LAPH_ERR_WORKSPACE = -3


def _mom_ptr(mom):
    return mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def test_noalloc_rejects_bad_arguments_without_gpu():
    ensure_built()
    from paper_2510_26313_gb300 import binding
    L = binding.lib()
    mom = np.zeros((1, 3), dtype=np.int32)
    fake = ctypes.c_void_p(0x1000)
    # null input, no output, N < 3 with baryons, too many momenta, misaligned output
    assert L.laph_blocks_noalloc(None, 4, 1, 5, _mom_ptr(mom), 1, fake, fake, None) == LAPH_ERR_ARG
    assert L.laph_blocks_noalloc(fake, 4, 1, 5, _mom_ptr(mom), 1, None, None, None) == LAPH_ERR_ARG
    assert L.laph_blocks_noalloc(fake, 4, 1, 2, _mom_ptr(mom), 1, fake, None, None) == LAPH_ERR_ARG
    many = np.zeros((65, 3), dtype=np.int32)
    assert L.laph_blocks_noalloc(fake, 4, 1, 5, _mom_ptr(many), 65, None, fake, None) == LAPH_ERR_ARG
    assert L.laph_blocks_noalloc(fake, 4, 1, 5, _mom_ptr(mom), 1, None, ctypes.c_void_p(0x1008), None) == LAPH_ERR_ARG
    # phase table of 64 momenta at L = 64 (128 MiB) exceeds the fixed scratch array
    big = np.zeros((64, 3), dtype=np.int32)
    assert L.laph_blocks_noalloc(fake, 64, 1, 5, _mom_ptr(big), 64, None, fake, None) == LAPH_ERR_WORKSPACE
    # so does the tile table of many timeslices
    assert L.laph_blocks_noalloc(fake, 6, 100000, 200, _mom_ptr(big), 64, fake, fake, None) == LAPH_ERR_WORKSPACE


@pytest.mark.gpu
def test_noalloc_matches_plan_entry_points_twice_in_a_row():
    ensure_built()
    import torch
    torch.cuda.set_device(0)
    from oracle import oracle as O
    from paper_2510_26313_gb300 import binding

    calls = [
        # (L, T, N, momenta, instance, outputs): several row/column tiles and ragged site chunks with both
        # outputs, then baryons only (no meson rows: the first row tile starts with pairs) and mesons only
        # (no pair rows), including N = 2, where no baryon block exists
        (6, 2, 40, synth.momentum_shell(1), 11, "BM"),
        (5, 1, 13, synth.momentum_shell(2), 12, "BM"),
        (5, 1, 13, synth.momentum_shell(1), 13, "B"),
        (6, 1, 40, synth.momentum_shell(1), 14, "M"),
        (4, 1, 2, synth.momentum_shell(1), 15, "M"),
    ]
    for L, T, N, mom, inst, outs in calls:
        phi_h = synth.random_phi(L, N, T=T, instance=inst)
        phi = torch.from_numpy(phi_h).cuda()
        P = mom.shape[0]
        # outputs start as NaN: the entry point must not rely on cleared memory
        B = torch.full((T, P, N * (N - 1) * (N - 2) // 6), float("nan"), dtype=torch.complex128,
                       device="cuda") if "B" in outs else None
        M = torch.full((T, P, N, N), float("nan"), dtype=torch.complex128, device="cuda") if "M" in outs else None
        binding.blocks_noalloc(phi, L, mom, B, M)
        torch.cuda.synchronize()
        if B is not None:
            b = B.cpu().numpy()
            assert np.isfinite(b).all()
            refB = binding.baryon_blocks(phi, L, mom, mode="fp32").cpu().numpy()
            assert rel_frob(b, refB) <= TOL_SPLIT
            orB = np.stack([O.baryon_blocks(phi_h[t], L, mom) for t in range(T)])
            assert rel_frob(b, orB) <= TOL_SPLIT
        if M is not None:
            m = M.cpu().numpy()
            assert np.isfinite(m).all()
            refM = binding.meson_blocks(phi, L, mom, mode="fp32").cpu().numpy()
            assert rel_frob(m, refM) <= TOL_SPLIT
            orM = np.stack([O.meson_blocks(phi_h[t], L, mom) for t in range(T)])
            assert rel_frob(m, orM) <= TOL_SPLIT


@pytest.mark.gpu
def test_noalloc_binding_refuses_mismatched_outputs():
    """The binding checks dtype, shape, contiguity and device of the outputs before the C call, which cannot
    check the size of a device buffer; nothing is launched."""
    ensure_built()
    import torch
    torch.cuda.set_device(0)
    from paper_2510_26313_gb300 import binding
    L, T, N = 4, 1, 6
    mom = synth.momentum_shell(0)
    phi = torch.from_numpy(synth.random_phi(L, N, T=T, instance=16)).cuda()
    good_M = torch.empty((T, 1, N, N), dtype=torch.complex128, device="cuda")
    bad = [
        torch.empty((T, 1, N, N - 1), dtype=torch.complex128, device="cuda"),   # too small
        torch.empty((T, 1, N, N), dtype=torch.complex64, device="cuda"),        # wrong dtype
        torch.empty((T, 1, N, N), dtype=torch.complex128),                      # host memory
        torch.empty((T, 1, N, 2 * N), dtype=torch.complex128, device="cuda")[..., ::2],   # not contiguous
    ]
    for out in bad:
        with pytest.raises(ValueError):
            binding.blocks_noalloc(phi, L, mom, None, out)
    with pytest.raises(ValueError):
        binding.blocks_noalloc(phi, L, mom, torch.empty((T, 1, 3), dtype=torch.complex128, device="cuda"), good_M)
    with pytest.raises(ValueError):
        binding.blocks_noalloc(phi, L, mom, None, None)
