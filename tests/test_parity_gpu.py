"""GPU parity: the CUDA path against the FP64 oracle, element by element.

Relative Frobenius error per output (B and M separately) and the worst
per-(t,p) slice, bounded by 1e-5 for the FP32 and split-precision paths and
by the stated per-mode bound for single-term FP16/BF16.
"""
import math

import numpy as np
import pytest

from helpers import ensure_built, rel_frob, tol_for, worst_slice
from oracle import oracle as O
from paper_2510_26313_gb300 import synth

pytestmark = pytest.mark.gpu

SPLIT_MODES = ["fp32", "f16x3", "bf16x3"]
ALL_MODES = SPLIT_MODES + ["f16", "bf16"]


@pytest.fixture(scope="module")
def laph():
    ensure_built()
    import torch
    torch.cuda.set_device(0)
    from paper_2510_26313_gb300 import binding
    return binding


def _run(laph, phi_h, L, mom, mode):
    import torch
    phi = torch.from_numpy(phi_h).cuda()
    B = laph.baryon_blocks(phi, L, mom, mode=mode) if phi_h.shape[1] >= 3 else None
    M = laph.meson_blocks(phi, L, mom, mode=mode)
    torch.cuda.synchronize()
    return (B.cpu().numpy() if B is not None else None), M.cpu().numpy()


def _oracle(phi_h, L, mom):
    Bs = [O.baryon_blocks(phi_h[t], L, mom) for t in range(phi_h.shape[0])] if phi_h.shape[1] >= 3 else None
    Ms = [O.meson_blocks(phi_h[t], L, mom) for t in range(phi_h.shape[0])]
    return (np.stack(Bs) if Bs is not None else None), np.stack(Ms)


CASES = [
    # (L, T, N, momenta, instance): shapes chosen to span several tiles and ragged tails
    (8, 1, 16, np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.int32), 1),   # the L=8, N=16 plain case
    (5, 2, 13, synth.momentum_shell(1), 2),                                       # V=125: ragged site chunks
    (6, 1, 40, synth.momentum_shell(2), 3),                                       # several row/column tiles
    (4, 1, 3, synth.momentum_shell(0), 4),                                        # one triple
    (7, 1, 70, np.array([[0, 0, 0], [2, -1, 3]], dtype=np.int32), 5),             # N > 64: more row tiles
    (17, 1, 14, synth.momentum_shell(1), 6),                                      # V=4913: two site blocks of the
                                                                                  # FP64 reduction, the last ragged
]


@pytest.mark.parametrize("mode", ALL_MODES)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_blocks_match_oracle(laph, mode, case):
    L, T, N, mom, inst = CASES[case]
    phi_h = synth.random_phi(L, N, T=T, instance=inst)
    B, M = _run(laph, phi_h, L, mom, mode)
    rB, rM = _oracle(phi_h, L, mom)
    tol = tol_for(mode)
    eB, eM = rel_frob(B, rB), rel_frob(M, rM)
    print(f"mode={mode} L={L} N={N} P={len(mom)}: rel B {eB:.2e} M {eM:.2e}")
    assert eB <= tol and eM <= tol
    assert worst_slice(B, rB, 2) <= 4 * tol and worst_slice(M, rM, 2) <= 4 * tol


@pytest.mark.parametrize("mode", SPLIT_MODES)
def test_medium_config_two_timeslices(laph, mode):
    """L=24, N=32, 7 momenta (|n|^2 <= 1): two timeslices of the medium configuration."""
    L, N = 24, 32
    mom = synth.momentum_shell(1)
    phi_h = synth.random_phi(L, N, T=2, instance=0)
    B, M = _run(laph, phi_h, L, mom, mode)
    rB, rM = _oracle(phi_h, L, mom)
    eB, eM = rel_frob(B, rB), rel_frob(M, rM)
    print(f"medium mode={mode}: rel B {eB:.2e} M {eM:.2e}")
    assert eB <= 1e-5 and eM <= 1e-5


def test_meson_only_small_N(laph):
    L = 4
    mom = synth.momentum_shell(1)
    for N in (1, 2):
        phi_h = synth.random_phi(L, N, T=1, instance=10 + N)
        import torch
        M = laph.meson_blocks(torch.from_numpy(phi_h).cuda(), L, mom, mode="fp32").cpu().numpy()
        assert rel_frob(M[0], O.meson_blocks(phi_h[0], L, mom)) <= 1e-5


def test_baryon_rejects_N_below_3(laph):
    import torch
    phi = torch.from_numpy(synth.random_phi(4, 2, T=1)).cuda()
    with pytest.raises(laph.LaphError) as e:
        laph.baryon_blocks(phi, 4, synth.momentum_shell(0), mode="fp32")
    assert e.value.status == laph.LAPH_ERR_ARG


def test_phase_table_matches_oracle(laph):
    for L, n2 in [(5, 2), (8, 4), (12, 1)]:
        mom = synth.momentum_shell(n2)
        got = laph.phase_table(L, mom).cpu().numpy()
        np.testing.assert_allclose(got, O.phase_table(L, mom), rtol=0, atol=2e-15)  # sincospi vs cos/sin: a few ulp


def test_diquarks_match_oracle(laph):
    import torch
    # V even with whole 64-site blocks (transposed 16-byte stores), V odd, a partial last
    # block with many pairs per warp, and a vector count beyond the shared-memory window
    for L, N, T in [(4, 7, 2), (5, 6, 1), (6, 40, 1), (4, 150, 1)]:
        phi_h = synth.random_phi(L, N, T=T, instance=20 + L)
        D = laph.diquarks(torch.from_numpy(phi_h).cuda(), L).cpu().numpy()
        for t in range(T):
            ref = O.diquarks(phi_h[t], L)
            assert rel_frob(D[t], ref) <= 1e-6


def test_dense_fill_is_exact(laph):
    import torch
    N, P, T = 9, 4, 2
    rng = np.random.default_rng(3)
    packed = rng.standard_normal((T, P, N * (N - 1) * (N - 2) // 6)) + 1j * rng.standard_normal(
        (T, P, N * (N - 1) * (N - 2) // 6))
    dense = laph.baryon_dense(torch.from_numpy(packed).cuda(), N).cpu().numpy()
    for t in range(T):
        ref = O.baryon_dense(packed[t], N)
        assert np.array_equal(dense[t].view(np.uint64), ref.view(np.uint64))   # bit for bit, signed zeros included


def test_plan_ragged_batch_matches_oracle(laph):
    """Several instances of different L, N, P and T in one plan execution."""
    import torch
    specs = [(4, 2, 5, synth.momentum_shell(1)), (6, 1, 11, synth.momentum_shell(0)),
             (5, 3, 8, synth.momentum_shell(2)), (3, 1, 20, np.array([[1, 1, 1], [0, 0, 0]], dtype=np.int32))]
    runs = [(mode, 0) for mode in SPLIT_MODES] + [("f16x3", laph.PLAN_CHUNK_PER_TIMESLICE)]
    for mode, flags in runs:
        plan = laph.Plan(specs, mode=mode, flags=flags)
        if flags:
            # every (instance, timeslice) is its own chunk: one B-operand pass and one contraction each
            assert plan.contraction_launches() == sum(T for _, T, _, _ in specs)
        phis_h = [synth.random_phi(L, N, T=T, instance=40 + n) for n, (L, T, N, _) in enumerate(specs)]
        phis = [torch.from_numpy(p).cuda() for p in phis_h]
        Bs, Ms = plan.alloc_outputs()
        ws = plan.alloc_workspace()
        plan.execute(phis, Bs, Ms, ws)
        torch.cuda.synchronize()
        assert plan.device_status() == laph.LAPH_OK
        for n, (L, T, N, mom) in enumerate(specs):
            rB, rM = _oracle(phis_h[n], L, mom)
            assert rel_frob(Bs[n].cpu().numpy(), rB) <= 1e-5
            assert rel_frob(Ms[n].cpu().numpy(), rM) <= 1e-5
        plan.close()


def test_plan_execute_is_capturable_in_a_cuda_graph(laph):
    import torch
    L, T, N = 6, 2, 12
    mom = synth.momentum_shell(1)
    phi_h = synth.random_phi(L, N, T=T, instance=60)
    runs = [(mode, 0) for mode in SPLIT_MODES] + [("bf16x3", laph.PLAN_CHUNK_PER_TIMESLICE)]
    for mode, flags in runs:
        plan = laph.Plan([(L, T, N, mom)], mode=mode, flags=flags)
        phi = torch.from_numpy(phi_h).cuda()
        Bs, Ms = plan.alloc_outputs()
        ws = plan.alloc_workspace()
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan.execute([phi], Bs, Ms, ws, stream=s)
        Bs[0].zero_()
        Ms[0].zero_()
        g.replay()
        torch.cuda.synchronize()
        rB, rM = _oracle(phi_h, L, mom)
        assert rel_frob(Bs[0].cpu().numpy(), rB) <= 1e-5
        assert rel_frob(Ms[0].cpu().numpy(), rM) <= 1e-5
        plan.close()


def test_execute_host_buffers(laph):
    """Host inputs and outputs; the tensor-core path pipelines copies and compute chunk by chunk."""
    import torch
    L, T, N = 5, 3, 9
    mom = synth.momentum_shell(1)
    phi_h = synth.random_phi(L, N, T=T, instance=61)
    rB, rM = _oracle(phi_h, L, mom)
    for mode, flags in [("fp32", 0), ("f16x3", 0), ("f16x3", laph.PLAN_CHUNK_PER_TIMESLICE)]:
        plan = laph.Plan([(L, T, N, mom)], mode=mode, flags=flags)
        ws = torch.empty(plan.host_workspace_size(), dtype=torch.uint8, device="cuda")
        Bh = np.zeros((T, len(mom), N * (N - 1) * (N - 2) // 6), dtype=np.complex128)
        Mh = np.zeros((T, len(mom), N, N), dtype=np.complex128)
        plan.execute_host([phi_h], [Bh], [Mh], ws)
        assert rel_frob(Bh, rB) <= 1e-5 and rel_frob(Mh, rM) <= 1e-5
        plan.close()


def test_invariances_at_size(laph):
    """L=16, N=32: SU(3) rotation leaves B, M unchanged; a translation multiplies them by
    exp(+2 pi i n.a/L); orthonormal vectors give M[p=0] = 1."""
    import torch
    L, N = 16, 32
    V = L ** 3
    mom = synth.momentum_shell(1)
    phi_h = synth.random_phi(L, N, T=1, instance=70)
    rng = np.random.default_rng(9)
    z = rng.standard_normal((V, 3, 3)) + 1j * rng.standard_normal((V, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    U = q * (d / np.abs(d))[:, None, :]
    U = U / (np.linalg.det(U) ** (1 / 3))[:, None, None]
    rot = np.einsum("xab,tnxb->tnxa", U, phi_h.astype(np.complex128)).astype(np.complex64)
    a = np.array([3, 0, 5])
    x = np.arange(V)
    c = np.stack([x % L, (x // L) % L, x // (L * L)], axis=1)
    src = ((c + a) % L) @ np.array([1, L, L * L])
    shifted = np.ascontiguousarray(phi_h[:, :, src, :])
    fac = np.exp(2j * np.pi * (mom @ a) / L)
    for mode in SPLIT_MODES:
        B0, M0 = _run(laph, phi_h, L, mom, mode)
        B1, M1 = _run(laph, rot, L, mom, mode)
        B2, M2 = _run(laph, shifted, L, mom, mode)
        assert rel_frob(B1, B0) <= 2e-5 and rel_frob(M1, M0) <= 2e-5
        assert rel_frob(B2, fac[None, :, None] * B0) <= 2e-5
        assert rel_frob(M2, fac[None, :, None, None] * M0) <= 2e-5
        np.testing.assert_allclose(M0[0, 0], np.eye(N), atol=2e-6 if mode == "fp32" else 1e-5)


def test_stalled_producer_times_out_and_context_stays_usable(laph):
    """A producer warp that never arrives (the plan's stall hook) makes the MMA's bounded wait
    expire: the kernel records a timeout, every role returns, and the context stays usable."""
    import torch
    L, T, N = 4, 1, 10
    mom = synth.momentum_shell(1)
    phi_h = synth.random_phi(L, N, T=T, instance=90)
    phi = torch.from_numpy(phi_h).cuda()
    plan = laph.Plan([(L, T, N, mom)], mode="f16x3", flags=laph.PLAN_DEBUG_STALL)
    Bs, Ms = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    plan.execute([phi], Bs, Ms, ws)
    torch.cuda.synchronize()
    assert plan.device_status() == laph.LAPH_ERR_TIMEOUT
    plan.close()
    B, M = _run(laph, phi_h, L, mom, "f16x3")
    rB, rM = _oracle(phi_h, L, mom)
    assert rel_frob(B, rB) <= 1e-5 and rel_frob(M, rM) <= 1e-5


def _sampled_triples(N, n, seed):
    rng = np.random.default_rng(seed)
    trip = sorted({tuple(int(v) for v in sorted(rng.choice(N, 3, replace=False))) for _ in range(n)})
    idx = [math.comb(k, 3) + math.comb(j, 2) + i for (i, j, k) in trip]
    return trip, idx


def test_metric_workload_parity(laph):
    """L=32, T=64, N=64, P=19 (|n|^2 <= 2), the benchmark's inputs and its chunked launch
    configuration: every baryon triple and meson entry of the first timeslice, sampled
    baryon triples and the whole meson blocks of the last timeslice, against the oracle."""
    import torch
    L, T, N = 32, 64, 64
    mom = synth.momentum_shell(2)
    phi_h = synth.random_phi(L, N, T=T, instance=0)
    plan = laph.Plan([(L, T, N, mom)], mode="f16x3")
    assert plan.contraction_launches() > 1
    phi = torch.from_numpy(phi_h).cuda()
    Bs, Ms = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    plan.execute([phi], Bs, Ms, ws)
    torch.cuda.synchronize()
    assert plan.device_status() == laph.LAPH_OK
    rB0, rM0 = _oracle(phi_h[:1], L, mom)
    eB = rel_frob(Bs[0][:1].cpu().numpy(), rB0)
    eM = rel_frob(Ms[0][:1].cpu().numpy(), rM0)
    print(f"L=32 N=64 P=19 timeslice 0, all entries: rel B {eB:.2e} M {eM:.2e}")
    assert eB <= 1e-5 and eM <= 1e-5
    assert worst_slice(Bs[0][:1].cpu().numpy(), rB0, 2) <= 2e-5
    trip, idx = _sampled_triples(N, 400, 5)
    t = T - 1
    ref = O.baryon_triples(phi_h[t], L, mom, trip)                 # [n][P]
    got = Bs[0][t][:, idx].cpu().numpy().T
    eBs = rel_frob(got, ref)
    eMl = rel_frob(Ms[0][t].cpu().numpy(), O.meson_blocks(phi_h[t], L, mom))
    print(f"timeslice {t}: rel B (400 sampled triples) {eBs:.2e} M {eMl:.2e}")
    assert eBs <= 1e-5 and eMl <= 1e-5
    plan.close()


def test_large_streamed_shape_sampled_parity(laph):
    """L=48, N=128, 33 momenta (|n|^2 <= 4): one timeslice per chunk, 128 staged row vectors.
    Sampled triples, and the meson blocks of a subset of vectors (M[i][j] depends only on
    vectors i and j)."""
    import torch
    L, T, N = 48, 1, 128
    mom = synth.momentum_shell(4)
    assert mom.shape[0] == 33
    phi_h = synth.random_phi(L, N, T=T, instance=7)
    plan = laph.Plan([(L, T, N, mom)], mode="f16x3")
    phi = torch.from_numpy(phi_h).cuda()
    Bs, Ms = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    plan.execute([phi], Bs, Ms, ws)
    torch.cuda.synchronize()
    assert plan.device_status() == laph.LAPH_OK
    trip, idx = _sampled_triples(N, 200, 6)
    ref = O.baryon_triples(phi_h[0], L, mom, trip)
    eB = rel_frob(Bs[0][0][:, idx].cpu().numpy().T, ref)
    sub = np.sort(np.random.default_rng(8).choice(N, 12, replace=False))
    rM = O.meson_blocks(phi_h[0][sub], L, mom)
    gM = Ms[0][0].cpu().numpy()[:, sub][:, :, sub]
    eM = rel_frob(gM, rM)
    print(f"L=48 N=128 P=33: rel B ({len(trip)} sampled triples) {eB:.2e}, M (12 x 12 vectors) {eM:.2e}")
    assert eB <= 1e-5 and eM <= 1e-5
    plan.close()


@pytest.mark.parametrize("mode", ["f16x3", "bf16x3"])
def test_separate_drain_interval_for_tiles_without_mesons(laph, mode):
    """laph_plan_options.chunk_sites_b: tiles without meson rows drain at another interval than the tiles that hold
    meson rows (here 2x and 1/2x); several row tiles of both kinds, ragged site blocks; blocks within the bound."""
    import torch
    for L, T, N, mom, inst in [CASES[2], CASES[4], CASES[5]]:
        phi_h = synth.random_phi(L, N, T=T, instance=inst)
        rB, rM = _oracle(phi_h, L, mom)
        for csb in (256, 64):
            plan = laph.Plan([(L, T, N, mom)], mode=mode, chunk_sites_b=csb)
            assert plan.drain_sites() == (128, csb)
            Bs, Ms = plan.alloc_outputs()
            plan.execute([torch.from_numpy(phi_h).cuda()], Bs, Ms, plan.alloc_workspace())
            torch.cuda.synchronize()
            assert plan.device_status() == laph.LAPH_OK
            eB, eM = rel_frob(Bs[0].cpu().numpy(), rB), rel_frob(Ms[0].cpu().numpy(), rM)
            print(f"chunk_sites_b={csb} mode={mode} L={L} N={N}: rel B {eB:.2e} M {eM:.2e}")
            assert eB <= tol_for(mode) and eM <= tol_for(mode)
            plan.close()


@pytest.mark.parametrize("mode", ["f16x3", "bf16x3"])
def test_complex64_outputs_are_the_rounded_complex128_outputs(laph, mode):
    """PLAN_OUT_C64: every B and M entry is the complex128 result of the same schedule rounded once to complex64
    (bitwise), through the device execute, a ragged batch and the host-buffer execute; the binding refuses
    complex128 buffers for such a plan."""
    import torch
    specs = [(L, T, N, mom) for (L, T, N, mom, _) in (CASES[2], CASES[4], CASES[5])]
    phis_h = [synth.random_phi(L, N, T=T, instance=170 + n) for n, (L, T, N, _) in enumerate(specs)]
    phis = [torch.from_numpy(p).cuda() for p in phis_h]
    ref = laph.Plan(specs, mode=mode)
    rB, rM = ref.alloc_outputs()
    ref.execute(phis, rB, rM, ref.alloc_workspace())
    plan = laph.Plan(specs, mode=mode, flags=laph.PLAN_OUT_C64)
    Bs, Ms = plan.alloc_outputs()
    assert Bs[0].dtype == torch.complex64
    plan.execute(phis, Bs, Ms, plan.alloc_workspace())
    torch.cuda.synchronize()
    assert plan.device_status() == laph.LAPH_OK
    for n, (L, T, N, mom) in enumerate(specs):
        b128, m128 = rB[n].cpu().numpy(), rM[n].cpu().numpy()
        assert np.array_equal(Bs[n].cpu().numpy(), b128.astype(np.complex64))
        assert np.array_equal(Ms[n].cpu().numpy(), m128.astype(np.complex64))
        oB, oM = _oracle(phis_h[n], L, mom)
        assert rel_frob(Bs[n].cpu().numpy(), oB) <= tol_for(mode) and rel_frob(Ms[n].cpu().numpy(), oM) <= tol_for(mode)
    # host buffers
    L, T, N, mom = specs[0]
    one = laph.Plan([specs[0]], mode=mode, flags=laph.PLAN_OUT_C64)
    hws = torch.empty(one.host_workspace_size(), dtype=torch.uint8, device="cuda")
    Bh = np.zeros((T, len(mom), N * (N - 1) * (N - 2) // 6), dtype=np.complex64)
    Mh = np.zeros((T, len(mom), N, N), dtype=np.complex64)
    one.execute_host([phis_h[0]], [Bh], [Mh], hws)
    assert np.array_equal(Bh, rB[0].cpu().numpy().astype(np.complex64))
    assert np.array_equal(Mh, rM[0].cpu().numpy().astype(np.complex64))
    with pytest.raises(ValueError):
        one.execute_host([phis_h[0]], [Bh.astype(np.complex128)], [Mh], hws)
    with pytest.raises(ValueError):
        one.execute([phis[0]], [rB[0]], [Ms[0]], one.alloc_workspace())
    # the autotuner's accuracy probe reads complex64 outputs too
    tuned = laph.Plan([specs[0]], mode=mode, flags=laph.PLAN_OUT_C64 | laph.PLAN_AUTOTUNE)
    probed = [r["probe_err"] for r in tuned.tuning() if r["probe_err"] >= 0]
    assert probed and all(0 < e < 1e-4 for e in probed)
    tB, tM = tuned.alloc_outputs()
    tuned.execute([phis[0]], tB, tM, tuned.alloc_workspace())
    torch.cuda.synchronize()
    oB, oM = _oracle(phis_h[0], L, mom)
    assert rel_frob(tB[0].cpu().numpy(), oB) <= tol_for(mode) and rel_frob(tM[0].cpu().numpy(), oM) <= tol_for(mode)
    for p_ in (ref, plan, one, tuned):
        p_.close()


def test_complex64_triplets_and_doublets(laph):
    """PLAN_OUT_C64 with several fields: dense triplets and doublets equal the complex128 results rounded once."""
    import torch
    L, T, N = 5, 2, 9
    mom = synth.momentum_shell(1)
    f = [torch.from_numpy(synth.random_phi(L, N, T=T, instance=180 + q)).cuda() for q in range(3)]
    for skip, nf in ((laph.PLAN_SKIP_M, 3), (laph.PLAN_SKIP_B, 2)):
        outs = []
        for extra in (0, laph.PLAN_OUT_C64):
            plan = laph.Plan([(L, T, N, mom)], mode="f16x3", flags=laph.PLAN_FIELDS | skip | extra)
            Bs, Ms = plan.alloc_outputs()
            o = Bs if skip == laph.PLAN_SKIP_M else Ms
            plan.execute_fields([f[:nf]], o, plan.alloc_workspace())
            torch.cuda.synchronize()
            outs.append(o[0].cpu().numpy())
            plan.close()
        assert outs[1].dtype == np.complex64 and np.array_equal(outs[1], outs[0].astype(np.complex64))


def test_default_tile_width_keeps_a_four_deep_stage_ring(laph):
    """The default tile is 104 columns wide unless the row vectors a tile stages would then leave a stage ring shallower
    than four buffers (about N > 80 at 128 rows), where it is 96; an explicit width or layout is kept."""
    mom = synth.momentum_shell(1)
    for N, cols in [(64, 104), (40, 104), (96, 96)]:
        plan = laph.Plan([(4, 1, N, mom)], mode="f16x3")
        assert plan.describe()["tile_cols"] == cols, (N, plan.describe())
        plan.close()
    plan = laph.Plan([(4, 1, 96, mom)], mode="f16x3", tile_cols=104)
    assert plan.describe()["tile_cols"] == 104
    plan.close()


@pytest.mark.parametrize("mode", ["f16x3", "bf16x3", "f16"])
@pytest.mark.parametrize("cols", [64, 80, 104])
def test_other_column_widths_match_oracle(laph, mode, cols):
    """Tiles of 64, 80 and 104 complex columns (UMMA N = 128, 160 and 208; at 208 the accumulator and the running
    sums fill tensor memory up to the A slots): single instances with ragged column tails and several site blocks,
    and a ragged batch in one plan."""
    import torch
    for L, T, N, mom, inst in [CASES[2], CASES[4], CASES[5]]:
        phi_h = synth.random_phi(L, N, T=T, instance=inst)
        plan = laph.Plan([(L, T, N, mom)], mode=mode, tile_cols=cols)
        assert plan.describe()["tile_cols"] == cols
        Bs, Ms = plan.alloc_outputs()
        ws = plan.alloc_workspace()
        plan.execute([torch.from_numpy(phi_h).cuda()], Bs, Ms, ws)
        torch.cuda.synchronize()
        assert plan.device_status() == laph.LAPH_OK
        rB, rM = _oracle(phi_h, L, mom)
        eB, eM = rel_frob(Bs[0].cpu().numpy(), rB), rel_frob(Ms[0].cpu().numpy(), rM)
        print(f"{cols} columns mode={mode} L={L} N={N}: rel B {eB:.2e} M {eM:.2e}")
        assert eB <= tol_for(mode) and eM <= tol_for(mode)
        plan.close()
    specs = [(4, 2, 5, synth.momentum_shell(1)), (5, 3, 8, synth.momentum_shell(2)),
             (3, 1, 20, np.array([[1, 1, 1], [0, 0, 0]], dtype=np.int32))]
    plan = laph.Plan(specs, mode=mode, tile_cols=cols)
    phis_h = [synth.random_phi(L, N, T=T, instance=140 + n) for n, (L, T, N, _) in enumerate(specs)]
    Bs, Ms = plan.alloc_outputs()
    plan.execute([torch.from_numpy(p).cuda() for p in phis_h], Bs, Ms, plan.alloc_workspace())
    torch.cuda.synchronize()
    for n, (L, T, N, mom) in enumerate(specs):
        rB, rM = _oracle(phis_h[n], L, mom)
        assert rel_frob(Bs[n].cpu().numpy(), rB) <= tol_for(mode)
        assert rel_frob(Ms[n].cpu().numpy(), rM) <= tol_for(mode)
    plan.close()


@pytest.mark.parametrize("mode", ["f16x3", "bf16x3", "f16"])
@pytest.mark.parametrize("cols", [176, 192, 208, 128])
def test_row_doubled_layout_matches_oracle(laph, mode, cols):
    """Layout 1 (two real A rows per complex row, 64 complex rows per tile, half-size B stage images): single
    instances with several row tiles that mix meson and diquark rows, ragged column tails, skipped leading columns
    and several site blocks, and a ragged batch in one plan."""
    import torch
    for L, T, N, mom, inst in [CASES[0], CASES[2], CASES[4], CASES[5]]:
        phi_h = synth.random_phi(L, N, T=T, instance=inst)
        plan = laph.Plan([(L, T, N, mom)], mode=mode, tile_cols=cols, layout=1)
        d = plan.describe()
        assert d["tile_cols"] == cols and d["tile_rows"] == 64
        Bs, Ms = plan.alloc_outputs()
        plan.execute([torch.from_numpy(phi_h).cuda()], Bs, Ms, plan.alloc_workspace())
        torch.cuda.synchronize()
        assert plan.device_status() == laph.LAPH_OK
        rB, rM = _oracle(phi_h, L, mom)
        eB, eM = rel_frob(Bs[0].cpu().numpy(), rB), rel_frob(Ms[0].cpu().numpy(), rM)
        print(f"layout 1, {cols} columns, mode={mode} L={L} N={N}: rel B {eB:.2e} M {eM:.2e}")
        assert eB <= tol_for(mode) and eM <= tol_for(mode)
        plan.close()
    specs = [(4, 2, 5, synth.momentum_shell(1)), (5, 3, 8, synth.momentum_shell(2)),
             (3, 1, 20, np.array([[1, 1, 1], [0, 0, 0]], dtype=np.int32))]
    plan = laph.Plan(specs, mode=mode, tile_cols=cols, layout=1)
    phis_h = [synth.random_phi(L, N, T=T, instance=150 + n) for n, (L, T, N, _) in enumerate(specs)]
    Bs, Ms = plan.alloc_outputs()
    plan.execute([torch.from_numpy(p).cuda() for p in phis_h], Bs, Ms, plan.alloc_workspace())
    torch.cuda.synchronize()
    for n, (L, T, N, mom) in enumerate(specs):
        rB, rM = _oracle(phis_h[n], L, mom)
        assert rel_frob(Bs[n].cpu().numpy(), rB) <= tol_for(mode)
        assert rel_frob(Ms[n].cpu().numpy(), rM) <= tol_for(mode)
    plan.close()


def test_row_doubled_layout_fields_and_projection(laph):
    """Layout 1 on the several-field plans: three-field triplets and a projection of two vector counts against the
    oracle."""
    import torch
    L, T, N = 4, 2, 9
    mom = synth.momentum_shell(1)
    f = [synth.random_phi(L, N, T=T, instance=160 + k, orthonormal=False) for k in range(3)]
    plan = laph.Plan([(L, T, N, mom)], mode="f16x3", flags=laph.PLAN_FIELDS | laph.PLAN_SKIP_M, layout=1)
    Bs, _ = plan.alloc_outputs()
    plan.execute_fields([[torch.from_numpy(x).cuda() for x in f]], Bs, plan.alloc_workspace())
    torch.cuda.synchronize()
    for t in range(T):
        ref = O.triplet_blocks(f[0][t], f[1][t], f[2][t], L, mom)
        assert rel_frob(Bs[0][t].cpu().numpy(), ref) <= 1e-5
    plan.close()
    v = synth.random_phi(L, 7, T=T, instance=170, orthonormal=False)
    sv = synth.random_phi(L, 30, T=T, instance=171, orthonormal=False)
    plan = laph.Plan([(L, T, 7, np.zeros((1, 3), dtype=np.int32), 30)], mode="f16x3",
                     flags=laph.PLAN_FIELDS | laph.PLAN_SKIP_B, layout=1, tile_cols=128)
    _, Ms = plan.alloc_outputs()
    plan.execute_fields([[torch.from_numpy(v).cuda(), torch.from_numpy(sv).cuda()]], Ms, plan.alloc_workspace())
    torch.cuda.synchronize()
    for t in range(T):
        assert rel_frob(Ms[0][t].cpu().numpy(), O.projection(v[t], sv[t], L)) <= 1e-5
    plan.close()


def test_row_doubled_layout_in_a_cuda_graph_with_host_buffers_and_chunks(laph):
    """Layout 1 through the other execution paths: a plan captured in a CUDA graph and replayed, one timeslice per
    chunk (several B-operand passes, contractions and FP64 reductions per execute), and the host-buffer execute."""
    import torch
    L, T, N = 6, 3, 12
    mom = synth.momentum_shell(1)
    phi_h = synth.random_phi(L, N, T=T, instance=190)
    rB, rM = _oracle(phi_h, L, mom)
    for flags in (0, laph.PLAN_CHUNK_PER_TIMESLICE):
        plan = laph.Plan([(L, T, N, mom)], mode="f16x3", flags=flags, layout=1, sum_sites=64)
        assert plan.sum_sites()[1] >= 2                        # several site blocks per output
        phi = torch.from_numpy(phi_h).cuda()
        Bs, Ms = plan.alloc_outputs()
        ws = plan.alloc_workspace()
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan.execute([phi], Bs, Ms, ws, stream=s)
        Bs[0].zero_()
        Ms[0].zero_()
        g.replay()
        torch.cuda.synchronize()
        assert rel_frob(Bs[0].cpu().numpy(), rB) <= 1e-5 and rel_frob(Ms[0].cpu().numpy(), rM) <= 1e-5
        hws = torch.empty(plan.host_workspace_size(), dtype=torch.uint8, device="cuda")
        Bh = np.zeros((T, len(mom), N * (N - 1) * (N - 2) // 6), dtype=np.complex128)
        Mh = np.zeros((T, len(mom), N, N), dtype=np.complex128)
        plan.execute_host([phi_h], [Bh], [Mh], hws)
        assert rel_frob(Bh, rB) <= 1e-5 and rel_frob(Mh, rM) <= 1e-5
        plan.close()


@pytest.mark.parametrize("mode", ALL_MODES)
def test_degenerate_lattices_and_minimal_shapes(laph, mode):
    """L = 1 (one site: every momentum phase is 1, one site block), L = 2 with N = 3V = 24 (a complete basis), and N = 3
    (a single triple): every mode against the oracle."""
    for L, N, mom, inst in [(1, 3, np.array([[0, 0, 0], [1, 0, 0]], dtype=np.int32), 180),
                            (2, 24, synth.momentum_shell(1), 181), (3, 3, synth.momentum_shell(2), 182)]:
        phi_h = synth.random_phi(L, N, T=2, instance=inst)
        B, M = _run(laph, phi_h, L, mom, mode)
        rB, rM = _oracle(phi_h, L, mom)
        tol = tol_for(mode)
        assert rel_frob(B, rB) <= tol and rel_frob(M, rM) <= tol, (L, N, mode)


def test_many_vectors_beyond_the_staging_limit(laph):
    """N = 200 vectors: the tensor-core path cannot stage a tile's row vectors (more than 160) and says so with
    LAPH_ERR_UNSUPPORTED at plan creation; the FP32 path computes the blocks, checked against the oracle on sampled
    triples and on whole meson blocks."""
    import torch
    L, N = 4, 180
    mom = synth.momentum_shell(1)
    with pytest.raises(laph.LaphError) as e:
        laph.Plan([(L, 1, N, mom)], mode="f16x3")
    assert e.value.status == laph.LAPH_ERR_UNSUPPORTED
    phi_h = synth.random_phi(L, N, T=1, instance=183)
    phi = torch.from_numpy(phi_h).cuda()
    B = laph.baryon_blocks(phi, L, mom, mode="fp32").cpu().numpy()
    M = laph.meson_blocks(phi, L, mom, mode="fp32").cpu().numpy()
    trip, idx = _sampled_triples(N, 300, 9)
    assert rel_frob(B[0][:, idx].T, O.baryon_triples(phi_h[0], L, mom, trip)) <= 1e-5
    assert rel_frob(M[0], O.meson_blocks(phi_h[0], L, mom)) <= 1e-5


def test_autotuned_plan_matches_oracle(laph):
    """PLAN_AUTOTUNE times candidate schedules at creation -- tile widths, tile orders, chunkings, site-block sizes
    and drain intervals, the last checked by the accuracy probe -- and keeps the fastest; the chosen schedule gives
    the same blocks."""
    import torch
    L, T, N = 6, 3, 20
    mom = synth.momentum_shell(1)
    plan = laph.Plan([(L, T, N, mom)], mode="f16x3", flags=laph.PLAN_AUTOTUNE)
    sch = plan.schedule()
    assert len(sch["candidate_ms"]) >= 2 and all(ms > 0 for ms in sch["candidate_ms"])
    assert sch["tile_order"] in (0, 1) and sch["n_chunks"] == plan.contraction_launches()
    rec = plan.tuning()
    assert len(rec) >= 10 and {(r["tile_cols"], r["layout"]) for r in rec} >= {(64, 0), (96, 0), (176, 1)}
    assert len({r["sum_sites"] for r in rec}) >= 2 and len({r["chunk_sites"] for r in rec}) >= 2
    probed = [r for r in rec if r["probe_err"] >= 0]
    assert len(probed) >= 2 and all(r["probe_err"] < 1e-4 for r in probed)
    desc = plan.describe()
    assert any(r["tile_cols"] == desc["tile_cols"] and r["chunk_sites"] == desc["chunk_sites"] and
               r["chunk_sites_b"] == plan.drain_sites()[1] and r["sum_sites"] == plan.sum_sites()[0] for r in rec)
    print("autotune:", [(r["tile_cols"], r["tile_order"], r["sum_sites"], r["chunk_sites"], r["chunk_sites_b"],
                         round(r["ms"], 3), r["probe_err"]) for r in rec], "chosen", desc, plan.drain_sites())
    phi_h = synth.random_phi(L, N, T=T, instance=95)
    Bs, Ms = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    plan.execute([torch.from_numpy(phi_h).cuda()], Bs, Ms, ws)
    torch.cuda.synchronize()
    assert plan.device_status() == laph.LAPH_OK
    rB, rM = _oracle(phi_h, L, mom)
    assert rel_frob(Bs[0].cpu().numpy(), rB) <= 1e-5 and rel_frob(Ms[0].cpu().numpy(), rM) <= 1e-5
    plan.close()
