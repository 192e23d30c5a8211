"""The Python binding refuses buffers the C side would read or write out of bounds.

The C entry points receive plain device pointers and cannot check the size of
a buffer, so the binding checks every tensor it passes: dtype, contiguity,
exact shape, the current device, and the workspace's size.  Each call below
is wrong in one way and must raise ValueError before any launch; a correct
call afterwards still runs (nothing was left half done).
"""
import numpy as np
import pytest

from helpers import ensure_built
from paper_2510_26313_gb300 import synth

pytestmark = pytest.mark.gpu

L, T, N = 4, 2, 6
MOM = [(0, 0, 0), (1, 0, 0)]


@pytest.fixture(scope="module")
def laph():
    ensure_built()
    import torch
    torch.cuda.set_device(0)
    from paper_2510_26313_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def phi():
    import torch
    return torch.from_numpy(synth.random_phi(L, N, T=T, instance=71)).cuda()


def test_one_shot_outputs_are_checked(laph, phi):
    import torch
    P, C3 = len(MOM), N * (N - 1) * (N - 2) // 6
    dev = phi.device
    bad = [
        lambda: laph.baryon_blocks(phi, L, MOM, out=torch.empty((T, P, C3 - 1), dtype=torch.complex128, device=dev)),
        lambda: laph.baryon_blocks(phi, L, MOM, out=torch.empty((T, P, C3), dtype=torch.complex64, device=dev)),
        lambda: laph.meson_blocks(phi, L, MOM, out=torch.empty((T, P, N, N - 1), dtype=torch.complex128, device=dev)),
        lambda: laph.meson_blocks(phi, L, MOM, out=torch.empty((T, P, N, N), dtype=torch.complex128)),   # host
        lambda: laph.meson_blocks(phi, L, MOM,
                                  out=torch.empty((T, P, N, 2 * N), dtype=torch.complex128, device=dev)[..., ::2]),
        lambda: laph.triplet_blocks(phi, phi, phi, L, MOM,
                                    out=torch.empty((T, P, N, N, N - 1), dtype=torch.complex128, device=dev)),
        lambda: laph.doublet_blocks(phi, phi, L, MOM, out=torch.empty((T, P, N, N + 1), dtype=torch.complex128,
                                                                       device=dev)),
        lambda: laph.projection(phi, phi[:, :3].contiguous(), L, MOM,
                                out=torch.empty((T, P, N, N), dtype=torch.complex128, device=dev)),
        lambda: laph.diquarks(phi, L, out=torch.empty((T, N * (N - 1) // 2 - 1, L ** 3, 3), dtype=torch.complex64,
                                                      device=dev)),
        lambda: laph.baryon_dense(torch.empty((T, P, C3 + 1), dtype=torch.complex128, device=dev), N),
        lambda: laph.baryon_dense(torch.empty((T, P, C3), dtype=torch.complex128, device=dev), N,
                                  out=torch.empty((T, P, N, N, N - 1), dtype=torch.complex128, device=dev)),
    ]
    for k, call in enumerate(bad):
        with pytest.raises(ValueError):
            call()
            pytest.fail(f"case {k} was accepted")
    M = laph.meson_blocks(phi, L, MOM, mode="fp32")
    torch.cuda.synchronize()
    assert M.shape == (T, P, N, N) and torch.isfinite(torch.view_as_real(M)).all()


def test_plan_inputs_workspace_and_outputs_are_checked(laph, phi):
    import torch
    plan = laph.Plan([(L, T, N, MOM)], mode="f16x3")
    Bs, Ms = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    assert ws is not None and ws.numel() > 1
    fewer_vectors = phi[:, :N - 1].contiguous()
    fewer_slices = phi[:1].contiguous()
    bad = [
        lambda: plan.execute([fewer_vectors], Bs, Ms, ws),
        lambda: plan.execute([fewer_slices], Bs, Ms, ws),
        lambda: plan.execute([phi, phi], Bs, Ms, ws),                   # two fields for one instance
        lambda: plan.execute([phi], Bs, Ms, ws[:-1]),                   # workspace one byte short
        lambda: plan.execute([phi], Bs, Ms, None),
        lambda: plan.execute([phi], [Bs[0][:, :, :-1].contiguous()], Ms, ws),
    ]
    for k, call in enumerate(bad):
        with pytest.raises(ValueError):
            call()
            pytest.fail(f"case {k} was accepted")
    hws = torch.empty(plan.host_workspace_size(), dtype=torch.uint8, device="cuda")
    phi_h = phi.cpu().numpy()
    Bh, Mh = [np.empty(s[0], np.complex128) for s in plan.output_shapes()], \
        [np.empty(s[1], np.complex128) for s in plan.output_shapes()]
    bad_host = [
        lambda: plan.execute_host([phi_h[:, :N - 1].copy()], Bh, Mh, hws),
        lambda: plan.execute_host([phi_h.astype(np.complex128)], Bh, Mh, hws),
        lambda: plan.execute_host([phi_h], Bh, Mh, hws[:-1]),
    ]
    for k, call in enumerate(bad_host):
        with pytest.raises(ValueError):
            call()
            pytest.fail(f"host case {k} was accepted")
    plan.execute([phi], Bs, Ms, ws)
    plan.execute_host([phi_h], Bh, Mh, hws)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    Md = Ms[0].cpu().numpy()
    assert np.linalg.norm(Md - Mh[0]) <= 1e-5 * np.linalg.norm(Md)
    plan.close()


def test_field_plans_check_every_field(laph, phi):
    import torch
    psi = phi[:, :3].contiguous()
    dbl = laph.Plan([(L, T, N, MOM, 3)], mode="f16x3", flags=laph.PLAN_FIELDS | laph.PLAN_SKIP_B)
    _, outs = dbl.alloc_outputs()
    ws = dbl.alloc_workspace()
    with pytest.raises(ValueError):
        dbl.execute_fields([(phi, phi)], outs, ws)                      # psi must hold n_col = 3 vectors
    with pytest.raises(ValueError):
        dbl.execute_fields([(phi, psi, psi)], outs, ws)                 # a doublet takes two fields
    dbl.execute_fields([(phi, psi)], outs, ws)
    trp = laph.Plan([(L, T, N, MOM)], mode="f16x3", flags=laph.PLAN_FIELDS | laph.PLAN_SKIP_M)
    outs3, _ = trp.alloc_outputs()
    ws3 = trp.alloc_workspace()
    with pytest.raises(ValueError):
        trp.execute_fields([(phi, phi, psi)], outs3, ws3)
    trp.execute_fields([(phi, phi, phi)], outs3, ws3)
    torch.cuda.synchronize()
    assert dbl.device_status() == 0 and trp.device_status() == 0
    dbl.close()
    trp.close()


def test_laplacian_and_lanczos_outputs_are_checked(laph):
    import torch
    Lz = 4
    U = torch.from_numpy(synth.random_links(Lz, 1, instance=5, eps=0.6)).cuda()
    f = torch.zeros((1, 2, Lz ** 3, 3), dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError):
        laph.laplacian(U, f, Lz, out=torch.empty((1, 1, Lz ** 3, 3), dtype=torch.complex64, device="cuda"))
    with pytest.raises(ValueError):
        laph.lanczos(U, Lz, 4, 20, out=torch.empty((1, 3, Lz ** 3, 3), dtype=torch.complex64, device="cuda"))
    with pytest.raises(ValueError):
        laph.lanczos(U, Lz, 4, 20, workspace=torch.empty(16, dtype=torch.uint8))          # host workspace
    _, ev, _ = laph.lanczos(U, Lz, 4, 20)
    assert np.all(np.isfinite(ev))
