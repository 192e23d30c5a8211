"""GPU parity of the three-field triplets, two-field doublets and projection against the FP64 oracle.

    B3[t][p][i][j][k] = sum_x ph_p(x) eps_abc phi_i^a psi_j^b chi_k^c   (dense)
    M2[t][p][i][j]    = sum_x ph_p(x) conj(phi_i^a) psi_j^a
    Pr[t][p][i][j]    = the same with Nv vectors v and Ns vectors s (inner products at n = 0)

Element-by-element relative Frobenius error per output and worst per-(t, p)
slice, bounded by 1e-5 for the split-precision tensor-core modes, at shapes
that span several row and column tiles with ragged tails, through the
one-shot entry points and through a ragged plan replayed from a CUDA graph.
"""
import numpy as np
import pytest

from helpers import ensure_built, rel_frob, worst_slice
from oracle import oracle as O
from paper_2510_26313_gb300 import synth

pytestmark = pytest.mark.gpu

SPLIT_TC = ["f16x3", "bf16x3"]

CASES = [
    # (L, T, N, momenta, instance)
    (4, 1, 5, synth.momentum_shell(1), 1),     # 25 rows, one row and one column tile
    (5, 2, 13, synth.momentum_shell(2), 2),    # 169 rows: 2 row tiles; 247 columns: 3 column tiles; V=125
    (3, 1, 1, synth.momentum_shell(0), 3),     # N = 1: one entry
    (4, 1, 20, np.array([[0, 0, 0], [1, -1, 2]], dtype=np.int32), 4),   # 400 rows: 4 row tiles
]


@pytest.fixture(scope="module")
def laph():
    ensure_built()
    import torch
    torch.cuda.set_device(0)
    from paper_2510_26313_gb300 import binding
    return binding


def three_fields(L, N, T, inst):
    return [synth.random_phi(L, N, T=T, instance=100 * f + inst) for f in range(3)]


def oracle_triplets(fs, L, mom):
    return np.stack([O.triplet_blocks(fs[0][t], fs[1][t], fs[2][t], L, mom) for t in range(fs[0].shape[0])])


def oracle_doublets(fs, L, mom):
    return np.stack([O.doublet_blocks(fs[0][t], fs[1][t], L, mom) for t in range(fs[0].shape[0])])


@pytest.mark.parametrize("mode", SPLIT_TC)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_triplets_match_oracle(laph, mode, case):
    import torch
    L, T, N, mom, inst = CASES[case]
    fs = three_fields(L, N, T, inst)
    B = laph.triplet_blocks(*[torch.from_numpy(f).cuda() for f in fs], L, mom, mode=mode)
    torch.cuda.synchronize()
    got, ref = B.cpu().numpy(), oracle_triplets(fs, L, mom)
    e = rel_frob(got, ref)
    print(f"mode={mode} L={L} N={N} P={len(mom)}: rel B3 {e:.2e}")
    assert e <= 1e-5
    assert worst_slice(got, ref, 2) <= 4e-5


@pytest.mark.parametrize("mode", SPLIT_TC)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_doublets_match_oracle(laph, mode, case):
    import torch
    L, T, N, mom, inst = CASES[case]
    fs = three_fields(L, N, T, inst)[:2]
    M = laph.doublet_blocks(*[torch.from_numpy(f).cuda() for f in fs], L, mom, mode=mode)
    torch.cuda.synchronize()
    got, ref = M.cpu().numpy(), oracle_doublets(fs, L, mom)
    e = rel_frob(got, ref)
    print(f"mode={mode} L={L} N={N} P={len(mom)}: rel M2 {e:.2e}")
    assert e <= 1e-5
    assert worst_slice(got, ref, 2) <= 4e-5


def test_one_field_gives_the_dense_baryon_and_meson_blocks(laph):
    """phi = psi = chi: the triplets are the antisymmetric baryon tensor, the doublets the meson blocks."""
    import torch
    L, T, N = 5, 1, 9
    mom = synth.momentum_shell(1)
    phi_h = synth.random_phi(L, N, T=T, instance=7)
    phi = torch.from_numpy(phi_h).cuda()
    B3 = laph.triplet_blocks(phi, phi, phi, L, mom).cpu().numpy()
    M2 = laph.doublet_blocks(phi, phi, L, mom).cpu().numpy()
    dense = O.baryon_dense(O.baryon_blocks(phi_h[0], L, mom), N)
    assert rel_frob(B3[0], dense) <= 1e-5
    assert rel_frob(M2[0], O.meson_blocks(phi_h[0], L, mom)) <= 1e-5
    # entries with a repeated index vanish up to rounding
    rep = np.array([B3[0][:, a, a, c] for a in range(N) for c in range(N)])
    assert np.abs(rep).max() <= 1e-5 * np.abs(B3).max()


@pytest.mark.parametrize("triplets", [True, False])
def test_fields_plan_ragged_batch_in_a_cuda_graph(laph, triplets):
    import torch
    insts = [(5, 1, 7, synth.momentum_shell(1)), (4, 2, 11, synth.momentum_shell(2))]
    flags = laph.PLAN_FIELDS | (laph.PLAN_SKIP_M if triplets else laph.PLAN_SKIP_B)
    plan = laph.Plan(insts, mode="f16x3", flags=flags)
    nf = 3 if triplets else 2
    host = [three_fields(L, N, T, 20 + n)[:nf] for n, (L, T, N, _) in enumerate(insts)]
    dev = [[torch.from_numpy(f).cuda() for f in fs] for fs in host]
    Bs, Ms = plan.alloc_outputs()
    outs = Bs if triplets else Ms
    ws = plan.alloc_workspace()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.execute_fields(dev, outs, ws, stream=s)
    for o in outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert plan.device_status() == laph.LAPH_OK
    for n, (L, T, N, mom) in enumerate(insts):
        ref = oracle_triplets(host[n], L, mom) if triplets else oracle_doublets(host[n], L, mom)
        assert rel_frob(outs[n].cpu().numpy(), ref) <= 1e-5
    plan.close()


def test_triplets_at_L32_N64_P19_sampled_parity(laph):
    """The shape of the L=32, N=64, 19-momentum workload: sampled (i, j, k) of every momentum against the oracle."""
    import torch
    L, T, N = 32, 2, 64
    mom = synth.momentum_shell(2)
    fs = three_fields(L, N, T, 9)
    B = laph.triplet_blocks(*[torch.from_numpy(f).cuda() for f in fs], L, mom)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    ijk = rng.integers(0, N, size=(48, 3))
    ijk[:4] = [[0, 0, 0], [N - 1, N - 1, N - 1], [0, N - 1, 5], [N - 1, 0, N - 2]]   # corners, repeats
    for t in range(T):
        ref = O.triplet_triples(fs[0][t], fs[1][t], fs[2][t], L, mom, ijk)            # [n][P]
        got = B[t][:, ijk[:, 0], ijk[:, 1], ijk[:, 2]].cpu().numpy().T
        assert rel_frob(got, ref) <= 1e-5
    M = laph.doublet_blocks(*[torch.from_numpy(f).cuda() for f in fs[:2]], L, mom)
    assert rel_frob(M[0].cpu().numpy(), O.doublet_blocks(fs[0][0], fs[1][0], L, mom)) <= 1e-5


# ------------------------------------------------------------ projection

PROJ_CASES = [
    # (L, T, Nv, Ns, momenta, instance)
    (4, 2, 10, 37, np.zeros((1, 3), dtype=np.int32), 1),          # plain inner products
    (5, 1, 130, 20, synth.momentum_shell(1), 2),                   # Nv > 128: two row tiles
    (6, 1, 3, 200, np.zeros((1, 3), dtype=np.int32), 3),           # Ns = 200: three column tiles, ragged
]


@pytest.mark.parametrize("mode", SPLIT_TC)
@pytest.mark.parametrize("case", range(len(PROJ_CASES)))
def test_projection_matches_oracle(laph, mode, case):
    import torch
    L, T, Nv, Ns, mom, inst = PROJ_CASES[case]
    v = synth.random_phi(L, Nv, T=T, instance=inst)
    s = synth.random_phi(L, Ns, T=T, instance=50 + inst)
    got = laph.projection(torch.from_numpy(v).cuda(), torch.from_numpy(s).cuda(), L, mom, mode=mode).cpu().numpy()
    ref = np.stack([O.projection(v[t], s[t], L, mom) for t in range(T)])
    e = rel_frob(got, ref)
    print(f"mode={mode} L={L} Nv={Nv} Ns={Ns} P={len(mom)}: rel {e:.2e}")
    assert got.shape == (T, len(mom), Nv, Ns)
    assert e <= 1e-5
    assert worst_slice(got, ref, 2) <= 4e-5


def test_projection_recovers_expansion_coefficients_at_size(laph):
    """s_j = sum_i C_ij v_i with orthonormal v (L=16, 96 vectors): <v_i, s_j> = C_ij."""
    import torch
    L, Nv, Ns = 16, 96, 160
    v = synth.random_phi(L, Nv, T=1, instance=5)
    rng = np.random.default_rng(9)
    C = (rng.standard_normal((Nv, Ns)) + 1j * rng.standard_normal((Nv, Ns))).astype(np.complex64)
    s = np.einsum("ij,ixa->jxa", C, v[0]).astype(np.complex64)[None]
    got = laph.projection(torch.from_numpy(v).cuda(), torch.from_numpy(np.ascontiguousarray(s)).cuda(), L)
    assert rel_frob(got[0, 0].cpu().numpy(), C) <= 1e-5


def test_odd_stage_ring_over_long_tiles_and_repeated_executes(laph):
    """128 staged vectors per tile leave room for only 3 stage buffers, so the two A-producer groups take turns on
    each buffer; long tiles (L=32, 4096 stages) and back-to-back executes exercise the barrier phases of that
    ring.  Sampled inner products of every execute against the oracle."""
    import torch
    L, T, Nv, Ns = 32, 4, 128, 512
    v = synth.random_phi(L, Nv, T=T, instance=31)
    s = synth.random_phi(L, Ns, T=T, instance=32)
    mom = np.zeros((1, 3), dtype=np.int32)
    plan = laph.Plan([(L, T, Nv, mom, Ns)], mode="f16x3", flags=laph.PLAN_FIELDS | laph.PLAN_SKIP_B)
    _, Ms = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    vd, sd = torch.from_numpy(v).cuda(), torch.from_numpy(s).cuda()
    rows, cols = np.arange(0, Nv, 17), np.arange(3, Ns, 61)
    for t in (0, T - 1):
        ref = O.projection(v[t][rows], s[t][cols], L, mom)[0]
        for _ in range(3):
            Ms[0].zero_()
            plan.execute_fields([[vd, sd]], Ms, ws)
            torch.cuda.synchronize()
            assert plan.device_status() == laph.LAPH_OK
            got = Ms[0][t, 0].cpu().numpy()[np.ix_(rows, cols)]
            assert rel_frob(got, ref) <= 1e-5
    plan.close()
