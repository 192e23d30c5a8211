"""laph_blocks_noalloc: the allocation-free FP32 entry point.

Collected last on purpose (its scratch is a file-scope device array that
persists between calls): the GPU test calls it twice in a row, on different
shapes, through the C ABI and checks each result against the plan-based
FP32 entry points laph_baryon_blocks / laph_meson_blocks.  The CPU tests
check the argument and size rejections, which happen before any CUDA call.
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
    from paper_2510_26313_gb300 import binding

    calls = [
        # (L, T, N, momenta, instance): several row/column tiles, ragged site chunks
        (6, 2, 40, synth.momentum_shell(1), 11),
        (5, 1, 13, synth.momentum_shell(2), 12),
    ]
    for L, T, N, mom, inst in calls:
        phi = torch.from_numpy(synth.random_phi(L, N, T=T, instance=inst)).cuda()
        P = mom.shape[0]
        # outputs start as NaN: the entry point must not rely on cleared memory
        B = torch.full((T, P, N * (N - 1) * (N - 2) // 6), float("nan"), dtype=torch.complex128, device="cuda")
        M = torch.full((T, P, N, N), float("nan"), dtype=torch.complex128, device="cuda")
        binding.blocks_noalloc(phi, L, mom, B, M)
        torch.cuda.synchronize()
        refB = binding.baryon_blocks(phi, L, mom, mode="fp32")
        refM = binding.meson_blocks(phi, L, mom, mode="fp32")
        torch.cuda.synchronize()
        b, m = B.cpu().numpy(), M.cpu().numpy()
        assert np.isfinite(b).all() and np.isfinite(m).all()
        assert rel_frob(b, refB.cpu().numpy()) <= TOL_SPLIT
        assert rel_frob(m, refM.cpu().numpy()) <= TOL_SPLIT
