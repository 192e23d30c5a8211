"""Thin ctypes binding over the C ABI in ``include/laph.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are torch tensors on the current CUDA device (torch is used
for device memory and streams); every function raises ``LaphError`` on a
non-zero status, and loading fails loudly if the library was not built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblaph_gb300.so")
ABI_VERSION = 10100   # laph_version() of the library whose structures this binding declares

LAPH_OK = 0
LAPH_ERR_ARG = -1
LAPH_ERR_CUDA = -2
LAPH_ERR_WORKSPACE = -3
LAPH_ERR_UNSUPPORTED = -4
LAPH_ERR_TIMEOUT = -5
LAPH_ERR_DEVICE = -6

MODES = {"fp32": 0, "f16x3": 1, "bf16x3": 2, "f16": 3, "bf16": 4}
PLAN_SKIP_B = 0x1
PLAN_SKIP_M = 0x2
PLAN_AUTOTUNE = 0x4
PLAN_TIMING = 0x8
PLAN_DEBUG_STALL = 0x10000
PLAN_CHUNK_PER_TIMESLICE = 0x20000
PLAN_FIELDS = 0x40000
PLAN_OUT_C64 = 0x80000

_lib = None


class LaphError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().laph_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


class laph_instance(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("T", ctypes.c_int), ("N", ctypes.c_int), ("n_mom", ctypes.c_int),
                ("momenta", ctypes.POINTER(ctypes.c_int32)), ("n_col", ctypes.c_int)]


class laph_plan_options(ctypes.Structure):
    _fields_ = [("chunk_sites", ctypes.c_int), ("sum_sites", ctypes.c_int), ("tile_cols", ctypes.c_int),
                ("layout", ctypes.c_int), ("chunk_sites_b", ctypes.c_int)]


class laph_tune_record(ctypes.Structure):
    _fields_ = [("tile_cols", ctypes.c_int), ("layout", ctypes.c_int), ("sum_sites", ctypes.c_int),
                ("chunk_sites", ctypes.c_int), ("chunk_sites_b", ctypes.c_int),
                ("tile_order", ctypes.c_int), ("timeslices_per_chunk", ctypes.c_int64), ("ms", ctypes.c_float),
                ("probe_err", ctypes.c_double)]


class laph_lanczos_params(ctypes.Structure):
    _fields_ = [("n_krylov", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("seed", ctypes.c_uint32), ("ts_group", ctypes.c_int), ("pdl", ctypes.c_int),
                ("link_rows", ctypes.c_int)]


class laph_lanczos_stats(ctypes.Structure):
    _fields_ = [("total_ms", ctypes.c_double), ("setup_ms", ctypes.c_double), ("apply_ms", ctypes.c_double),
                ("orth_ms", ctypes.c_double), ("ritz_ms", ctypes.c_double), ("launches", ctypes.c_int64),
                ("apply_launches", ctypes.c_int64), ("links_two_rows", ctypes.c_int), ("ts_group", ctypes.c_int),
                ("host_steps", ctypes.c_int)]


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} not built: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        ip32 = ctypes.POINTER(ctypes.c_int32)
        vpp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "laph_triple_index": (i64, [i32, i32, i32]),
            "laph_status_string": (ctypes.c_char_p, [i32]),
            "laph_last_cuda_error": (ctypes.c_char_p, []),
            "laph_version": (i32, []),
            "laph_phase_table": (i32, [i32, ip32, i32, vp, vp]),
            "laph_diquarks": (i32, [vp, i32, i32, i32, vp, vp]),
            "laph_baryon_dense": (i32, [vp, i32, i32, i32, vp, vp]),
            "laph_baryon_blocks": (i32, [vp, i32, i32, i32, ip32, i32, vp, i32, vp]),
            "laph_meson_blocks": (i32, [vp, i32, i32, i32, ip32, i32, vp, i32, vp]),
            "laph_triplet_blocks": (i32, [vp, vp, vp, i32, i32, i32, ip32, i32, vp, i32, vp]),
            "laph_doublet_blocks": (i32, [vp, vp, i32, i32, i32, ip32, i32, vp, i32, vp]),
            "laph_plan_execute_fields": (i32, [vp, vpp, vpp, vp, vp]),
            "laph_projection": (i32, [vp, vp, i32, i32, i32, i32, ip32, i32, vp, i32, vp]),
            "laph_plan_create": (i32, [ctypes.POINTER(laph_instance), i32, i32, ctypes.c_uint, ctypes.POINTER(vp)]),
            "laph_plan_create_opts": (i32, [ctypes.POINTER(laph_instance), i32, i32, ctypes.c_uint,
                                            ctypes.POINTER(laph_plan_options), ctypes.POINTER(vp)]),
            "laph_plan_sum_sites": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "laph_plan_tuning": (i32, [vp, i32, ctypes.POINTER(laph_tune_record), ctypes.POINTER(i32)]),
            "laph_plan_drain_sites": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "laph_plan_workspace_size": (i32, [vp, ctypes.POINTER(sz)]),
            "laph_plan_execute": (i32, [vp, vpp, vpp, vpp, vp, vp]),
            "laph_plan_host_workspace_size": (i32, [vp, ctypes.POINTER(sz)]),
            "laph_plan_execute_host": (i32, [vp, vpp, vpp, vpp, vp, vp]),
            "laph_get_device_status": (i32, [vp, vp, ctypes.POINTER(i32)]),
            "laph_plan_describe": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                         ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64)]),
            "laph_plan_set_chunk_sites": (i32, [vp, i32]),
            "laph_plan_kernel_times": (i32, [vp, i32, ctypes.POINTER(ctypes.c_float)]),
            "laph_plan_operand_times": (i32, [vp, i32, ctypes.POINTER(ctypes.c_float)]),
            "laph_plan_reduce_times": (i32, [vp, i32, ctypes.POINTER(ctypes.c_float)]),
            "laph_plan_tensor_flops": (i32, [vp, ctypes.POINTER(ctypes.c_double)]),
            "laph_plan_contraction_launches": (i32, [vp, ctypes.POINTER(i32)]),
            "laph_plan_launches_per_execute": (i32, [vp, ctypes.POINTER(i32)]),
            "laph_plan_schedule": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                         ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)]),
            "laph_plan_destroy": (i32, [vp]),
            "laph_blocks_noalloc": (i32, [vp, i32, i32, i32, ip32, i32, vp, vp, vp]),
            "laph_laplacian": (i32, [vp, vp, vp, i32, i32, i32, vp]),
            "laph_lanczos": (i32, [vp, i32, i32, i32, ctypes.POINTER(laph_lanczos_params), vp,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp, sz,
                                   ctypes.POINTER(laph_lanczos_stats), vp]),
            "laph_lanczos_workspace_size": (i32, [i32, i32, i32, ctypes.POINTER(laph_lanczos_params),
                                                  ctypes.POINTER(sz)]),
            "laph_tridiag_eigen": (i32, [i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        # the ctypes structures above have the sizes of this ABI version; an older build would write past them
        if L.laph_version() != ABI_VERSION:
            raise RuntimeError(f"CUDA library {LIB_PATH} has ABI version {L.laph_version()}, the binding expects "
                               f"{ABI_VERSION}: rebuild it with __graft_entry__.build()")
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != LAPH_OK:
        raise LaphError(rc, where)


def _mode(mode) -> int:
    if isinstance(mode, str):
        return MODES[mode]
    return int(mode)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _momenta(momenta) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(momenta, dtype=np.int32).reshape(-1, 3))


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def triple_index(i: int, j: int, k: int) -> int:
    return int(lib().laph_triple_index(i, j, k))


def _on_current_device(t) -> bool:
    import torch
    return t.device.index == torch.cuda.current_device()


def _check_tensor(t, dtype, shape, name):
    """t must be a contiguous CUDA tensor of `dtype` and exactly `shape` on the current CUDA device: the C side
    reads or writes exactly that many elements there and cannot check the size of a device buffer."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not _on_current_device(t):
        raise ValueError(f"{name} must be on the current CUDA device")


def _check_workspace(ws, nbytes, name="workspace"):
    """A device workspace of at least `nbytes` bytes on the current CUDA device (None when nbytes is 0)."""
    import torch
    if nbytes == 0 and ws is None:
        return
    if not (isinstance(ws, torch.Tensor) and ws.is_cuda and ws.is_contiguous() and _on_current_device(ws)):
        raise ValueError(f"{name} must be a contiguous CUDA tensor on the current device ({nbytes} bytes)")
    if ws.numel() * ws.element_size() < nbytes:
        raise ValueError(f"{name} holds {ws.numel() * ws.element_size()} bytes, {nbytes} are needed")


def _check_phi(phi, L, T=None, N=None, name="phi"):
    """A field complex64 [T][N][L^3][3] on the current CUDA device; T and N are checked when given."""
    import torch
    if not (isinstance(phi, torch.Tensor) and phi.is_cuda and phi.dtype == torch.complex64 and phi.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous complex64 CUDA tensor [T][N][L^3][3]")
    if phi.dim() != 4 or phi.shape[2] != L ** 3 or phi.shape[3] != 3:
        raise ValueError(f"{name} must be [T][N][L^3][3], got {tuple(phi.shape)} for L={L}")
    if (T is not None and phi.shape[0] != T) or (N is not None and phi.shape[1] != N):
        raise ValueError(f"{name} must be [{T}][{N}][{L ** 3}][3], got {tuple(phi.shape)}")
    if not _on_current_device(phi):
        raise ValueError(f"{name} must be on the current CUDA device")
    return int(phi.shape[0]), int(phi.shape[1])


def _check_host_phi(a, shape, name):
    """A host field: a contiguous complex64 numpy array or CPU tensor of exactly `shape` (the C side copies
    that many bytes from it)."""
    import torch
    if isinstance(a, torch.Tensor):
        ok = not a.is_cuda and a.dtype == torch.complex64 and a.is_contiguous() and tuple(a.shape) == tuple(shape)
    else:
        ok = isinstance(a, np.ndarray) and a.dtype == np.complex64 and a.flags.c_contiguous and \
            tuple(a.shape) == tuple(shape)
    if not ok:
        raise ValueError(f"{name} must be a contiguous host complex64 buffer of shape {tuple(shape)}")


def phase_table(L: int, momenta, device=None):
    """complex128 [P][L^3] device tensor: exp(-2 pi i ((n_p.x) mod L)/L) in FP64."""
    import torch
    mom = _momenta(momenta)
    out = torch.empty((mom.shape[0], L ** 3), dtype=torch.complex128, device=device or "cuda")
    if not _on_current_device(out):
        raise ValueError("the phase table is computed on the current CUDA device")
    _check(lib().laph_phase_table(L, mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), mom.shape[0],
                                  _ptr(out), _stream(None)), "laph_phase_table")
    return out


def diquarks(phi, L: int, out=None, stream=None):
    """complex64 [T][C(N,2)][L^3][3]: D_q(x,c) = (phi_i(x) x phi_j(x))_c, q = C(j,2)+i."""
    import torch
    T, N = _check_phi(phi, L)
    if out is None:
        out = torch.empty((T, N * (N - 1) // 2, L ** 3, 3), dtype=torch.complex64, device=phi.device)
    _check_tensor(out, torch.complex64, (T, N * (N - 1) // 2, L ** 3, 3), "out")
    _check(lib().laph_diquarks(_ptr(phi), L, T, N, _ptr(out), _stream(stream)), "laph_diquarks")
    return out


def baryon_dense(packed, N: int, out=None, stream=None):
    """complex128 [T][P][N][N][N] from the packed [T][P][C(N,3)] form."""
    import torch
    if not (isinstance(packed, torch.Tensor) and packed.dim() == 3):
        raise ValueError("packed must be a complex128 CUDA tensor [T][P][C(N,3)]")
    T, P = int(packed.shape[0]), int(packed.shape[1])
    _check_tensor(packed, torch.complex128, (T, P, N * (N - 1) * (N - 2) // 6), "packed")
    if out is None:
        out = torch.empty((T, P, N, N, N), dtype=torch.complex128, device=packed.device)
    _check_tensor(out, torch.complex128, (T, P, N, N, N), "out")
    _check(lib().laph_baryon_dense(_ptr(packed), T, N, P, _ptr(out), _stream(stream)), "laph_baryon_dense")
    return out


def baryon_blocks(phi, L: int, momenta, mode="f16x3", out=None, stream=None):
    """Packed baryon blocks complex128 [T][P][C(N,3)] (one-shot entry point; blocking)."""
    import torch
    T, N = _check_phi(phi, L)
    mom = _momenta(momenta)
    if out is None:
        out = torch.empty((T, mom.shape[0], N * (N - 1) * (N - 2) // 6), dtype=torch.complex128, device=phi.device)
    _check_tensor(out, torch.complex128, (T, mom.shape[0], N * (N - 1) * (N - 2) // 6), "out")
    rc = lib().laph_baryon_blocks(_ptr(phi), L, T, N, mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  mom.shape[0], _ptr(out), _mode(mode), _stream(stream))
    _check(rc, "laph_baryon_blocks")
    return out


def meson_blocks(phi, L: int, momenta, mode="f16x3", out=None, stream=None):
    """Meson blocks complex128 [T][P][N][N] (one-shot entry point; blocking)."""
    import torch
    T, N = _check_phi(phi, L)
    mom = _momenta(momenta)
    if out is None:
        out = torch.empty((T, mom.shape[0], N, N), dtype=torch.complex128, device=phi.device)
    _check_tensor(out, torch.complex128, (T, mom.shape[0], N, N), "out")
    rc = lib().laph_meson_blocks(_ptr(phi), L, T, N, mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 mom.shape[0], _ptr(out), _mode(mode), _stream(stream))
    _check(rc, "laph_meson_blocks")
    return out


def _check_fields(fields, L, same_n=True):
    T, N = _check_phi(fields[0], L)
    for f in fields[1:]:
        Tf, Nf = _check_phi(f, L)
        if Tf != T or f.device != fields[0].device or (same_n and Nf != N):
            raise ValueError("the fields must have the same shape and device")
    return T, N


def triplet_blocks(phi, psi, chi, L: int, momenta, mode="f16x3", out=None, stream=None):
    """Three-field triplets complex128 [T][P][N][N][N], dense (one-shot; blocking)."""
    import torch
    T, N = _check_fields((phi, psi, chi), L)
    mom = _momenta(momenta)
    if out is None:
        out = torch.empty((T, mom.shape[0], N, N, N), dtype=torch.complex128, device=phi.device)
    _check_tensor(out, torch.complex128, (T, mom.shape[0], N, N, N), "out")
    rc = lib().laph_triplet_blocks(_ptr(phi), _ptr(psi), _ptr(chi), L, T, N,
                                   mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), mom.shape[0], _ptr(out),
                                   _mode(mode), _stream(stream))
    _check(rc, "laph_triplet_blocks")
    return out


def doublet_blocks(phi, psi, L: int, momenta, mode="f16x3", out=None, stream=None):
    """Two-field doublets complex128 [T][P][N][N] (one-shot; blocking)."""
    import torch
    T, N = _check_fields((phi, psi), L)
    mom = _momenta(momenta)
    if out is None:
        out = torch.empty((T, mom.shape[0], N, N), dtype=torch.complex128, device=phi.device)
    _check_tensor(out, torch.complex128, (T, mom.shape[0], N, N), "out")
    rc = lib().laph_doublet_blocks(_ptr(phi), _ptr(psi), L, T, N, mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   mom.shape[0], _ptr(out), _mode(mode), _stream(stream))
    _check(rc, "laph_doublet_blocks")
    return out


def projection(v, s, L: int, momenta=((0, 0, 0),), mode="f16x3", out=None, stream=None):
    """Projection of the vectors s onto the vectors v, complex128 [T][P][Nv][Ns]:
    sum_x ph_p(x) conj(v_i) . s_j (the inner products <v_i, s_j> at n = 0); one-shot, blocking."""
    import torch
    T, Nv = _check_phi(v, L)
    Ts, Ns = _check_phi(s, L)
    if Ts != T or s.device != v.device:
        raise ValueError("v and s must have the same timeslices and device")
    mom = _momenta(momenta)
    if out is None:
        out = torch.empty((T, mom.shape[0], Nv, Ns), dtype=torch.complex128, device=v.device)
    _check_tensor(out, torch.complex128, (T, mom.shape[0], Nv, Ns), "out")
    rc = lib().laph_projection(_ptr(v), _ptr(s), L, T, Nv, Ns, mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               mom.shape[0], _ptr(out), _mode(mode), _stream(stream))
    _check(rc, "laph_projection")
    return out


def _check_links(U, L):
    import torch
    if U.dtype != torch.complex64 or not U.is_cuda or not U.is_contiguous():
        raise ValueError("U must be a contiguous complex64 CUDA tensor [T][3][L^3][3][3]")
    if U.dim() != 5 or tuple(U.shape[1:]) != (3, L ** 3, 3, 3):
        raise ValueError(f"U must have shape [T][3][{L ** 3}][3][3], got {tuple(U.shape)}")
    if not _on_current_device(U):
        raise ValueError("U must be on the current CUDA device")
    return U.shape[0]


def laplacian(U, f, L: int, out=None, stream=None):
    """(-Delta) f on every timeslice, complex64 [T][nvec][L^3][3] (asynchronous on `stream`)."""
    import torch
    T = _check_links(U, L)
    Tf, nvec = _check_phi(f, L)
    if Tf != T or f.device != U.device:
        raise ValueError("f and U must have the same timeslices and device")
    if out is None:
        out = torch.empty_like(f)
    _check_tensor(out, torch.complex64, tuple(f.shape), "out")
    rc = lib().laph_laplacian(_ptr(U), _ptr(f), _ptr(out), L, T, nvec, _stream(stream))
    _check(rc, "laph_laplacian")
    return out


def lanczos_workspace_size(L: int, T: int, n_ev: int, n_krylov: int, cheb_degree: int = 0,
                           cheb_lo: float = 0.0) -> int:
    p = laph_lanczos_params(n_krylov, cheb_degree, cheb_lo, 0)
    n = ctypes.c_size_t()
    _check(lib().laph_lanczos_workspace_size(L, T, n_ev, ctypes.byref(p), ctypes.byref(n)),
           "laph_lanczos_workspace_size")
    return n.value


def lanczos(U, L: int, n_ev: int, n_krylov: int, cheb_degree: int = 0, cheb_lo: float = 0.0, seed: int = 0,
            out=None, workspace=None, stream=None, stats=None, ts_group: int = 0, pdl: bool = False,
            link_rows: int = 0):
    """The n_ev lowest eigenpairs of -Delta per timeslice (blocking).

    Returns (evecs complex64 [T][n_ev][L^3][3] on the device, evals float64 [T][n_ev] and
    residual norms float64 [T][n_ev] as numpy arrays).  workspace: a uint8 CUDA tensor of
    lanczos_workspace_size bytes (None: the call allocates its own).  stats: a dict that receives
    the call's event-timed breakdown (total_ms, setup_ms, apply_ms, orth_ms, ritz_ms, launches,
    apply_launches)."""
    import torch
    T = _check_links(U, L)
    if out is None:
        out = torch.empty((T, n_ev, L ** 3, 3), dtype=torch.complex64, device=U.device)
    _check_tensor(out, torch.complex64, (T, n_ev, L ** 3, 3), "out")
    if workspace is not None:
        _check_workspace(workspace, 0)
    p = laph_lanczos_params(n_krylov, cheb_degree, cheb_lo, seed, ts_group, int(pdl), link_rows)
    ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else None
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    ev = np.zeros((T, n_ev), dtype=np.float64)
    rs = np.zeros((T, n_ev), dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    st = laph_lanczos_stats()
    rc = lib().laph_lanczos(_ptr(U), L, T, n_ev, ctypes.byref(p), _ptr(out), ev.ctypes.data_as(dp),
                            rs.ctypes.data_as(dp), ws, ws_bytes, ctypes.byref(st) if stats is not None else None,
                            _stream(stream))
    _check(rc, "laph_lanczos")
    if stats is not None:
        stats.update({k: getattr(st, k) for k, _ in laph_lanczos_stats._fields_})
    return out, ev, rs


def tridiag_eigen(d, e):
    """Host QL solver: eigenvalues (ascending) and eigenvectors (columns) of a symmetric tridiagonal matrix."""
    d = np.array(d, dtype=np.float64)
    e = np.ascontiguousarray(np.asarray(e, dtype=np.float64))
    n = d.shape[0]
    z = np.zeros((n, n), dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib().laph_tridiag_eigen(n, d.ctypes.data_as(dp), e.ctypes.data_as(dp) if n > 1 else None,
                                  z.ctypes.data_as(dp))
    _check(rc, "laph_tridiag_eigen")
    return d, z


def _check_out(out, shape, phi, name):
    """An output tensor must be exactly what the C side will write: complex128, contiguous, the stated
    shape, on phi's device, which must be the current device."""
    import torch
    _check_tensor(out, torch.complex128, shape, name)
    if out.device != phi.device:
        raise ValueError(f"{name} and phi must be on the current CUDA device")


def blocks_noalloc(phi, L: int, momenta, out_B, out_M, stream=None):
    """FP32 B and/or M into caller-owned outputs with no device allocation.

    out_B: complex128 [T][P][C(N,3)] or None; out_M: complex128 [T][P][N][N]
    or None.  Asynchronous on `stream`; the library's fixed scratch array is
    shared by all calls, so calls must not overlap on the GPU.  The outputs
    are checked here (dtype, device, contiguity, exact shape) because the C
    entry point cannot check the size of a device buffer.
    """
    T, N = _check_phi(phi, L)
    mom = _momenta(momenta)
    P = mom.shape[0]
    if out_B is None and out_M is None:
        raise ValueError("at least one of out_B and out_M is needed")
    if out_B is not None:
        _check_out(out_B, (T, P, N * (N - 1) * (N - 2) // 6), phi, "out_B")
    if out_M is not None:
        _check_out(out_M, (T, P, N, N), phi, "out_M")
    rc = lib().laph_blocks_noalloc(_ptr(phi), L, T, N, mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   mom.shape[0], _ptr(out_B) if out_B is not None else None,
                                   _ptr(out_M) if out_M is not None else None, _stream(stream))
    _check(rc, "laph_blocks_noalloc")
    return out_B, out_M


class Plan:
    """A batch of (possibly ragged) instances with capture-safe execution.

    instances: list of (L, T, N, momenta).  Outputs per instance n:
    B[n] complex128 [T][P][C(N,3)], M[n] complex128 [T][P][N][N].
    """

    def __init__(self, instances, mode="f16x3", flags: int = 0, chunk_sites: int = 0, sum_sites: int = 0,
                 tile_cols: int = 0, layout: int = 0, chunk_sites_b: int = 0):
        # (L, T, N, momenta) or, for doublet plans of two vector counts, (L, T, N, momenta, n_col)
        self._moms = [_momenta(inst[3]) for inst in instances]
        self.n_col = [int(inst[4]) if len(inst) > 4 else 0 for inst in instances]
        arr = (laph_instance * len(instances))()
        for n, inst in enumerate(instances):
            L, T, N = inst[0], inst[1], inst[2]
            m = self._moms[n]
            arr[n] = laph_instance(L, T, N, m.shape[0], m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   self.n_col[n])
        self.instances = [(int(inst[0]), int(inst[1]), int(inst[2]), self._moms[n]) for n, inst in enumerate(instances)]
        self.flags = flags
        self.mode = _mode(mode)
        h = ctypes.c_void_p()
        opts = laph_plan_options(int(chunk_sites), int(sum_sites), int(tile_cols), int(layout), int(chunk_sites_b))
        _check(lib().laph_plan_create_opts(arr, len(instances), self.mode, flags, ctypes.byref(opts), ctypes.byref(h)),
               "laph_plan_create_opts")
        self._h = h

    @property
    def handle(self):
        return self._h

    def workspace_size(self) -> int:
        b = ctypes.c_size_t()
        _check(lib().laph_plan_workspace_size(self._h, ctypes.byref(b)), "laph_plan_workspace_size")
        return int(b.value)

    def host_workspace_size(self) -> int:
        b = ctypes.c_size_t()
        _check(lib().laph_plan_host_workspace_size(self._h, ctypes.byref(b)), "laph_plan_host_workspace_size")
        return int(b.value)

    def describe(self) -> dict:
        v = [ctypes.c_int() for _ in range(5)]
        nt = ctypes.c_int64()
        _check(lib().laph_plan_describe(self._h, *[ctypes.byref(x) for x in v], ctypes.byref(nt)),
               "laph_plan_describe")
        return dict(mode=v[0].value, tile_rows=v[1].value, tile_cols=v[2].value, chunk_sites=v[3].value,
                    grid=v[4].value, n_tiles=int(nt.value))

    def sum_sites(self) -> tuple:
        """(sites per block of the FP64 site reduction, largest number of blocks of any instance)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().laph_plan_sum_sites(self._h, ctypes.byref(a), ctypes.byref(b)), "laph_plan_sum_sites")
        return int(a.value), int(b.value)

    def kernel_times(self, n: int) -> list:
        """Durations (ms) of the last n contraction-kernel launches (needs PLAN_TIMING)."""
        arr = (ctypes.c_float * n)()
        _check(lib().laph_plan_kernel_times(self._h, n, arr), "laph_plan_kernel_times")
        return [float(x) for x in arr]

    def operand_times(self, n: int) -> list:
        """Durations (ms) of the last n B-operand launches of the tensor-core path (needs PLAN_TIMING)."""
        arr = (ctypes.c_float * n)()
        _check(lib().laph_plan_operand_times(self._h, n, arr), "laph_plan_operand_times")
        return [float(x) for x in arr]

    def reduce_times(self, n: int) -> list:
        """Durations (ms) of the last n FP64 site reductions of the tensor-core path (needs PLAN_TIMING)."""
        arr = (ctypes.c_float * n)()
        _check(lib().laph_plan_reduce_times(self._h, n, arr), "laph_plan_reduce_times")
        return [float(x) for x in arr]

    def tensor_flops(self) -> float:
        """Flops the tensor pipe executes per execute (all split terms, padding and triangle waste)."""
        v = ctypes.c_double()
        _check(lib().laph_plan_tensor_flops(self._h, ctypes.byref(v)), "laph_plan_tensor_flops")
        return float(v.value)

    def contraction_launches(self) -> int:
        """Contraction-kernel launches per execute (one per chunk of timeslices)."""
        v = ctypes.c_int()
        _check(lib().laph_plan_contraction_launches(self._h, ctypes.byref(v)), "laph_plan_contraction_launches")
        return int(v.value)

    def schedule(self) -> dict:
        """Tensor-core schedule: timeslices per chunk (0: filled by bytes), tile order, chunks,
        and the autotuner's candidate timings (ms) when PLAN_AUTOTUNE was given."""
        pc, order, nc, ncand = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_float * 8)()
        _check(lib().laph_plan_schedule(self._h, ctypes.byref(pc), ctypes.byref(order), ctypes.byref(nc),
                                        ctypes.byref(ncand), ms), "laph_plan_schedule")
        return {"timeslices_per_chunk": int(pc.value), "tile_order": int(order.value), "n_chunks": int(nc.value),
                "candidate_ms": [float(ms[k]) for k in range(min(ncand.value, 8))]}

    def drain_sites(self) -> tuple:
        """(drain interval of tiles with meson rows, of the others), in sites."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().laph_plan_drain_sites(self._h, ctypes.byref(a), ctypes.byref(b)), "laph_plan_drain_sites")
        return int(a.value), int(b.value)

    def tuning(self) -> list:
        """The autotuner's candidates (PLAN_AUTOTUNE): dicts of tile_cols, sum_sites, chunk_sites, tile_order,
        timeslices_per_chunk, ms and probe_err (-1 when not probed)."""
        n = ctypes.c_int()
        _check(lib().laph_plan_tuning(self._h, 0, None, ctypes.byref(n)), "laph_plan_tuning")
        recs = (laph_tune_record * max(n.value, 1))()
        _check(lib().laph_plan_tuning(self._h, n.value, recs, None), "laph_plan_tuning")
        return [{k: getattr(recs[i], k) for k, _ in laph_tune_record._fields_} for i in range(n.value)]

    def launches_per_execute(self) -> int:
        v = ctypes.c_int()
        _check(lib().laph_plan_launches_per_execute(self._h, ctypes.byref(v)), "laph_plan_launches_per_execute")
        return int(v.value)

    def alloc_workspace(self, device=None):
        import torch
        n = self.workspace_size()
        if n == 0:
            return None
        return torch.empty(n, dtype=torch.uint8, device=device or "cuda")

    def output_shapes(self):
        """Per instance, the shapes of its B (or B3) and M (or M2) outputs; None where skipped."""
        out = []
        for n, (L, T, N, m) in enumerate(self.instances):
            P = m.shape[0]
            shapeB = (T, P, N, N, N) if self.flags & PLAN_FIELDS else (T, P, N * (N - 1) * (N - 2) // 6)
            Nc = self.n_col[n] or N
            out.append((None if self.flags & PLAN_SKIP_B else shapeB, None if self.flags & PLAN_SKIP_M else (T, P, N, Nc)))
        return out

    @property
    def out_dtype(self):
        """torch dtype of the outputs: complex64 with PLAN_OUT_C64, else complex128."""
        import torch
        return torch.complex64 if self.flags & PLAN_OUT_C64 else torch.complex128

    def alloc_outputs(self, device=None):
        import torch
        Bs, Ms = [], []
        for sB, sM in self.output_shapes():
            Bs.append(None if sB is None else torch.empty(sB, dtype=self.out_dtype, device=device or "cuda"))
            Ms.append(None if sM is None else torch.empty(sM, dtype=self.out_dtype, device=device or "cuda"))
        return Bs, Ms

    def _check_outputs(self, Bs, Ms, host=False):
        """Every output the plan writes must be a contiguous buffer of the plan's dtype and exact shape (the C side
        cannot check the size of a buffer); device outputs on the current CUDA device."""
        import torch
        want = np.complex64 if self.flags & PLAN_OUT_C64 else np.complex128
        for n, (sB, sM) in enumerate(self.output_shapes()):
            for outs, shape, name in ((Bs, sB, "B"), (Ms, sM, "M")):
                if shape is None:
                    continue
                t = outs[n] if outs is not None and n < len(outs) else None
                if t is None:
                    raise ValueError(f"{name}[{n}] is required")
                if isinstance(t, torch.Tensor):
                    ok = t.dtype == self.out_dtype and t.is_contiguous() and tuple(t.shape) == tuple(shape)
                    ok = ok and (not t.is_cuda if host else (t.is_cuda and t.device.index == torch.cuda.current_device()))
                else:
                    ok = host and isinstance(t, np.ndarray) and t.dtype == want and t.flags.c_contiguous and \
                        tuple(t.shape) == tuple(shape)
                if not ok:
                    where = "host" if host else "current-device CUDA"
                    raise ValueError(f"{name}[{n}] must be a contiguous {where} {np.dtype(want).name} buffer of shape "
                                     f"{tuple(shape)}")

    @staticmethod
    def _ptr_array(ts):
        arr = (ctypes.c_void_p * len(ts))()
        for n, t in enumerate(ts):
            arr[n] = None if t is None else t.data_ptr()
        return arr

    def _check_inputs(self, phis, workspace, nbytes):
        """One field per instance, of the instance's shape, and a workspace of the plan's size."""
        if phis is None or len(phis) != len(self.instances):
            raise ValueError(f"{len(self.instances)} fields are needed, one per instance")
        _check_workspace(workspace, nbytes)

    def execute(self, phis, Bs, Ms, workspace, stream=None):
        self._check_inputs(phis, workspace, self.workspace_size())
        for n, ((L, T, N, _), phi) in enumerate(zip(self.instances, phis)):
            _check_phi(phi, L, T, N, f"phi[{n}]")
        self._check_outputs(Bs, Ms)
        pa = self._ptr_array(phis)
        ba = self._ptr_array(Bs) if Bs is not None else None
        ma = self._ptr_array(Ms) if Ms is not None else None
        ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else ctypes.c_void_p()
        _check(lib().laph_plan_execute(self._h, pa, ba, ma, ws, _stream(stream)), "laph_plan_execute")

    def execute_fields(self, fields, outs, workspace, stream=None):
        """LAPH_PLAN_FIELDS plans: fields[n] = (phi, psi, chi) for triplets, (phi, psi) for
        doublets; outs[n] the instance's B3 or M2."""
        self._check_inputs(fields, workspace, self.workspace_size())
        flat = []
        per = 2 if self.flags & PLAN_SKIP_B else 3
        for n, ((L, T, N, _), fs) in enumerate(zip(self.instances, fields)):
            if len(fs) != per:
                raise ValueError(f"fields[{n}] must hold {per} fields")
            for q, f in enumerate(fs):
                _check_phi(f, L, T, (self.n_col[n] or N) if q == 1 and per == 2 else N, f"fields[{n}][{q}]")
            flat.extend(fs)
        if self.flags & PLAN_SKIP_M:
            self._check_outputs(outs, None)
        else:
            self._check_outputs(None, outs)
        fa = self._ptr_array(flat)
        oa = self._ptr_array(outs)
        ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else ctypes.c_void_p()
        _check(lib().laph_plan_execute_fields(self._h, fa, oa, ws, _stream(stream)), "laph_plan_execute_fields")

    def execute_host(self, phis_host, Bs_host, Ms_host, workspace, stream=None):
        """Host (numpy / pinned torch CPU) inputs and outputs; blocking."""
        def addr(a):
            if a is None:
                return None
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        self._check_inputs(phis_host, workspace, self.host_workspace_size())
        for n, ((L, T, N, _), a) in enumerate(zip(self.instances, phis_host)):
            _check_host_phi(a, (T, N, L ** 3, 3), f"phi[{n}]")
        self._check_outputs(Bs_host, Ms_host, host=True)
        pa = (ctypes.c_void_p * len(phis_host))(*[addr(a) for a in phis_host])
        ba = (ctypes.c_void_p * len(Bs_host))(*[addr(a) for a in Bs_host]) if Bs_host is not None else None
        ma = (ctypes.c_void_p * len(Ms_host))(*[addr(a) for a in Ms_host]) if Ms_host is not None else None
        _check(lib().laph_plan_execute_host(self._h, pa, ba, ma, ctypes.c_void_p(workspace.data_ptr()),
                                            _stream(stream)), "laph_plan_execute_host")

    def device_status(self, stream=None) -> int:
        st = ctypes.c_int()
        _check(lib().laph_get_device_status(self._h, _stream(stream), ctypes.byref(st)), "laph_get_device_status")
        return int(st.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().laph_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
