"""CPU checks of the C ABI: the library builds, loads and exports every symbol
include/laph.h declares; host-only utilities and argument checks behave.
No compute call is made (no GPU here)."""
import ctypes
import os
import re

import pytest

from helpers import ROOT, ensure_built


@pytest.fixture(scope="module")
def lib():
    ensure_built()
    from paper_2510_26313_gb300 import binding
    return binding.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "laph.h")).read()
    return sorted(set(re.findall(r"LAPH_API\s+[\w\s\*]+?\b(laph_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["laph_baryon_blocks", "laph_meson_blocks", "laph_triplet_blocks", "laph_doublet_blocks",
                 "laph_plan_execute_fields", "laph_projection", "laph_plan_create", "laph_plan_execute",
                 "laph_plan_workspace_size", "laph_plan_destroy", "laph_phase_table", "laph_diquarks",
                 "laph_baryon_dense", "laph_get_device_status", "laph_triple_index", "laph_status_string",
                 "laph_laplacian", "laph_lanczos", "laph_tridiag_eigen"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2510_26313_gb300 import binding
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in laph.h but not exported by {binding.LIB_PATH}"
        # the binding sets result and argument types for every entry point (an untyped ctypes call would pass and
        # return plain ints, truncating 64-bit pointers and sizes)
        assert getattr(lib, n).argtypes is not None and getattr(lib, n).restype is not None, n


def test_triple_index_is_colex(lib):
    from paper_2510_26313_gb300 import binding
    seen = []
    for k in range(12):
        for j in range(k):
            for i in range(j):
                seen.append(binding.triple_index(i, j, k))
    assert seen == list(range(len(seen)))          # colex order enumerates 0..C(12,3)-1
    assert binding.triple_index(1, 1, 2) == -1
    assert binding.triple_index(2, 1, 3) == -1


def test_status_strings(lib):
    for code in [0, -1, -2, -3, -4, -5, -6]:
        assert lib.laph_status_string(code)
    assert lib.laph_version() == 10100   # 1.1: the structs of include/laph.h at their present sizes


def test_plan_create_rejects_bad_arguments_before_touching_cuda(lib):
    from paper_2510_26313_gb300 import binding
    mom = (ctypes.c_int32 * 3)(0, 0, 0)
    h = ctypes.c_void_p()
    bad = [
        binding.laph_instance(0, 1, 8, 1, mom),      # L < 1
        binding.laph_instance(4, 0, 8, 1, mom),      # T < 1
        binding.laph_instance(4, 1, 2, 1, mom),      # N < 3 with baryons
        binding.laph_instance(4, 1, 8, 0, mom),      # no momenta
        binding.laph_instance(2, 1, 25, 1, mom),     # N > 3 V
    ]
    for inst in bad:
        arr = (binding.laph_instance * 1)(inst)
        assert lib.laph_plan_create(arr, 1, 0, 0, ctypes.byref(h)) == binding.LAPH_ERR_ARG
    arr = (binding.laph_instance * 1)(binding.laph_instance(4, 1, 8, 1, mom))
    assert lib.laph_plan_create(arr, 1, 9, 0, ctypes.byref(h)) == binding.LAPH_ERR_ARG          # bad mode
    assert lib.laph_plan_create(arr, 1, 0, 3, ctypes.byref(h)) == binding.LAPH_ERR_ARG          # skip both
    big = (ctypes.c_int32 * 3)(1 << 21, 0, 0)
    arr = (binding.laph_instance * 1)(binding.laph_instance(4, 1, 8, 1, big))
    assert lib.laph_plan_create(arr, 1, 0, 0, ctypes.byref(h)) == binding.LAPH_ERR_ARG          # |n| too large
    assert lib.laph_plan_create(None, 1, 0, 0, ctypes.byref(h)) == binding.LAPH_ERR_ARG
    # several fields: needs exactly one of the skip flags, and a tensor-core mode
    arr = (binding.laph_instance * 1)(binding.laph_instance(4, 1, 2, 1, mom))
    assert lib.laph_plan_create(arr, 1, 1, binding.PLAN_FIELDS, ctypes.byref(h)) == binding.LAPH_ERR_ARG
    assert lib.laph_plan_create(arr, 1, 0, binding.PLAN_FIELDS | binding.PLAN_SKIP_M,
                                ctypes.byref(h)) == binding.LAPH_ERR_UNSUPPORTED                 # FP32 SIMT
    # a second vector count only for doublet plans, and not negative
    for flags, n_col in [(0, 9), (binding.PLAN_FIELDS | binding.PLAN_SKIP_M, 9),
                         (binding.PLAN_FIELDS | binding.PLAN_SKIP_B, -1)]:
        arr = (binding.laph_instance * 1)(binding.laph_instance(4, 1, 8, 1, mom, n_col))
        assert lib.laph_plan_create(arr, 1, 1, flags, ctypes.byref(h)) == binding.LAPH_ERR_ARG


def test_plan_options_are_checked_before_touching_cuda(lib):
    """laph_plan_create_opts refuses negative or oversized drain intervals and site blocks, tile widths without a
    compiled kernel and unknown layouts, before any CUDA call."""
    from paper_2510_26313_gb300 import binding
    mom = (ctypes.c_int32 * 3)(0, 0, 0)
    h = ctypes.c_void_p()
    arr = (binding.laph_instance * 1)(binding.laph_instance(4, 1, 8, 1, mom))
    for opts in [binding.laph_plan_options(-1, 0, 0, 0), binding.laph_plan_options(0, -8, 0, 0),
                 binding.laph_plan_options(1 << 25, 0, 0, 0), binding.laph_plan_options(0, 0, 72, 0),
                 binding.laph_plan_options(0, 0, 176, 0), binding.laph_plan_options(0, 0, 96, 1),
                 binding.laph_plan_options(0, 0, 112, 0), binding.laph_plan_options(0, 0, 104, 1),
                 binding.laph_plan_options(0, 0, 224, 1),
                 binding.laph_plan_options(0, 0, 0, 2), binding.laph_plan_options(0, 0, 0, -1),
                 binding.laph_plan_options(0, 0, 0, 0, -8), binding.laph_plan_options(0, 0, 0, 0, 1 << 25)]:
        assert lib.laph_plan_create_opts(arr, 1, 1, 0, ctypes.byref(opts), ctypes.byref(h)) == binding.LAPH_ERR_ARG
    # complex64 outputs are a tensor-core option: the FP32 mode accumulates in its complex128 outputs
    assert lib.laph_plan_create_opts(arr, 1, 0, binding.PLAN_OUT_C64, None, ctypes.byref(h)) == \
        binding.LAPH_ERR_UNSUPPORTED
    assert lib.laph_plan_tuning(None, 0, None, None) == binding.LAPH_ERR_ARG
    assert lib.laph_plan_drain_sites(None, None, None) == binding.LAPH_ERR_ARG
    assert lib.laph_plan_sum_sites(None, None, None) == binding.LAPH_ERR_ARG
    assert lib.laph_plan_tensor_flops(None, None) == binding.LAPH_ERR_ARG


def test_entry_points_reject_null_pointers(lib):
    from paper_2510_26313_gb300 import binding
    mom = (ctypes.c_int32 * 3)(0, 0, 0)
    assert lib.laph_baryon_blocks(None, 4, 1, 8, mom, 1, None, 0, None) == binding.LAPH_ERR_ARG
    assert lib.laph_meson_blocks(None, 4, 1, 8, mom, 1, None, 0, None) == binding.LAPH_ERR_ARG
    assert lib.laph_diquarks(None, 4, 1, 8, None, None) == binding.LAPH_ERR_ARG
    assert lib.laph_baryon_dense(None, 1, 8, 1, None, None) == binding.LAPH_ERR_ARG
    assert lib.laph_phase_table(0, mom, 1, None, None) == binding.LAPH_ERR_ARG
    assert lib.laph_plan_destroy(None) == binding.LAPH_ERR_ARG
    assert lib.laph_triplet_blocks(None, None, None, 4, 1, 8, mom, 1, None, 1, None) == binding.LAPH_ERR_ARG
    assert lib.laph_doublet_blocks(None, None, 4, 1, 8, mom, 1, None, 1, None) == binding.LAPH_ERR_ARG
    assert lib.laph_plan_execute_fields(None, None, None, None, None) == binding.LAPH_ERR_ARG
    assert lib.laph_projection(None, None, 4, 1, 8, 5, mom, 1, None, 1, None) == binding.LAPH_ERR_ARG
    assert lib.laph_projection(None, None, 4, 1, 8, 0, mom, 1, ctypes.c_void_p(16), 1, None) == binding.LAPH_ERR_ARG
    fake = ctypes.c_void_p(256)
    assert lib.laph_laplacian(None, fake, fake, 4, 1, 1, None) == binding.LAPH_ERR_ARG
    assert lib.laph_laplacian(fake, fake, fake, 1, 1, 1, None) == binding.LAPH_ERR_ARG          # L < 2
    assert lib.laph_laplacian(fake, fake, ctypes.c_void_p(260), 4, 1, 1, None) == binding.LAPH_ERR_ARG   # misaligned
    ev = (ctypes.c_double * 64)()
    ok = binding.laph_lanczos_params(40, 0, 0.0, 0)
    assert lib.laph_lanczos(None, 4, 1, 8, ctypes.byref(ok), fake, ev, None, None, 0, None, None) == binding.LAPH_ERR_ARG
    for bad in [binding.laph_lanczos_params(4, 0, 0.0, 0),        # m < n_ev
                binding.laph_lanczos_params(200, 0, 0.0, 0),      # m > 3 L^3 = 192
                binding.laph_lanczos_params(40, 8, 0.0, 0),       # filter without a bound
                binding.laph_lanczos_params(40, 8, 12.5, 0),      # bound above the spectrum
                binding.laph_lanczos_params(40, -1, 1.0, 0),
                binding.laph_lanczos_params(40, 0, 0.0, 0, 0, 0, 1),    # link rows other than 0, 2, 3
                binding.laph_lanczos_params(40, 8, 1.0, 0, -1)]:        # negative filter group
        assert lib.laph_lanczos(fake, 4, 1, 8, ctypes.byref(bad), fake, ev, None, None, 0, None, None) == binding.LAPH_ERR_ARG
        n = ctypes.c_size_t(0)
        assert lib.laph_lanczos_workspace_size(4, 1, 8, ctypes.byref(bad), ctypes.byref(n)) == binding.LAPH_ERR_ARG
    assert lib.laph_tridiag_eigen(0, None, None, None) == binding.LAPH_ERR_ARG
    # workspace: the size query needs no GPU; a workspace too small or misaligned is refused before any launch
    assert binding.lanczos_workspace_size(32, 64, 64, 160, 40, 0.95) >= 8 * 64 * 3 * 32 ** 3 * (160 + 1 + 64)
    assert lib.laph_lanczos(fake, 4, 1, 8, ctypes.byref(ok), fake, ev, None, fake, 1024, None,
                            None) == binding.LAPH_ERR_WORKSPACE
    assert lib.laph_lanczos(fake, 4, 1, 8, ctypes.byref(ok), fake, ev, None, ctypes.c_void_p(264), 1 << 30, None,
                            None) == binding.LAPH_ERR_WORKSPACE


@pytest.mark.parametrize("n", [1, 2, 3, 17, 150])
def test_tridiagonal_eigensolver_against_numpy(lib, n):
    """The host tridiagonal solver behind the Lanczos Ritz values: eigenvalues against numpy's dense solver, eigenvectors
    through the eigen-equation and orthonormality, on random matrices with some zero couplings (split blocks)."""
    import numpy as np
    from paper_2510_26313_gb300 import binding
    rng = np.random.default_rng(n)
    d = rng.standard_normal(n)
    e = rng.standard_normal(max(n - 1, 0))
    e[5::11] = 0.0
    Tm = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    w, z = binding.tridiag_eigen(d, e)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(Tm), atol=1e-12 * max(1.0, np.abs(w).max()))
    np.testing.assert_allclose(Tm @ z, z * w, atol=1e-12 * max(1.0, np.abs(w).max()))
    np.testing.assert_allclose(z.T @ z, np.eye(n), atol=1e-12)


@pytest.mark.parametrize("kind", ["wilkinson21", "graded", "zero_diagonal", "clustered"])
def test_tridiagonal_eigensolver_on_hard_spectra(lib, kind):
    """Matrices that stress the shift and the deflation test: Wilkinson's W21+ (pairs of eigenvalues agreeing to
    about 1e-14), a graded matrix spanning 13 decades, a zero diagonal (eigenvalues in +- pairs) and a cluster of
    nearly equal diagonal entries with tiny couplings; eigenvalues against numpy, eigen-equation and orthonormality."""
    import numpy as np
    from paper_2510_26313_gb300 import binding
    if kind == "wilkinson21":
        d, e = np.abs(np.arange(-10, 11)).astype(float), np.ones(20)
    elif kind == "graded":
        d, e = 10.0 ** (-np.arange(40) / 3), 10.0 ** (-np.arange(39) / 3 - 0.1)
    elif kind == "zero_diagonal":
        d, e = np.zeros(30), np.random.default_rng(1).standard_normal(29)
    else:
        d, e = 1.0 + 1e-14 * np.arange(50), np.full(49, 1e-10)
    Tm = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    w, z = binding.tridiag_eigen(d, e)
    sc = max(1.0, np.abs(w).max())
    np.testing.assert_allclose(w, np.linalg.eigvalsh(Tm), rtol=0, atol=1e-13 * sc)
    np.testing.assert_allclose(Tm @ z, z * w, rtol=0, atol=1e-13 * sc)
    np.testing.assert_allclose(z.T @ z, np.eye(len(d)), rtol=0, atol=1e-13)
    assert np.all(np.diff(w) >= 0)


def test_tridiagonal_eigensolver_on_the_free_chain():
    """-1, 2, -1 chain of n sites (open ends): eigenvalues 2 - 2 cos(pi k / (n + 1)), k = 1..n."""
    import numpy as np
    from paper_2510_26313_gb300 import binding
    ensure_built()
    n = 64
    w, _ = binding.tridiag_eigen(np.full(n, 2.0), np.full(n - 1, -1.0))
    np.testing.assert_allclose(w, 2 - 2 * np.cos(np.pi * np.arange(1, n + 1) / (n + 1)), atol=1e-13)


def test_product_path_does_not_reference_the_oracle():
    """The CUDA library and its binding never name the oracle."""
    pkg = os.path.join(ROOT, "paper_2510_26313_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "laph_oracle" not in txt, f


def test_binding_validates_links_and_vectors_before_calling_the_library(lib):
    """The Laplacian, Lanczos and block wrappers refuse host tensors, wrong dtypes and wrong shapes with ValueError
    (no library call, no GPU needed)."""
    import numpy as np
    torch = pytest.importorskip("torch")
    from paper_2510_26313_gb300 import binding
    L = 4
    U = torch.zeros((1, 3, L ** 3, 3, 3), dtype=torch.complex64)            # host tensor
    f = torch.zeros((1, 2, L ** 3, 3), dtype=torch.complex64)
    with pytest.raises(ValueError):
        binding.laplacian(U, f, L)
    with pytest.raises(ValueError):
        binding.lanczos(U, L, 4, 20)
    with pytest.raises(ValueError):
        binding.lanczos(U.to(torch.complex128), L, 4, 20)
    with pytest.raises(ValueError):
        binding.lanczos(U[:, :2].contiguous(), L, 4, 20)                     # two directions
    phi = torch.zeros((1, 4, L ** 3, 3), dtype=torch.complex64)          # host field
    mom = [(0, 0, 0)]
    for call in (lambda: binding.baryon_blocks(phi, L, mom), lambda: binding.meson_blocks(phi, L, mom),
                 lambda: binding.diquarks(phi, L), lambda: binding.triplet_blocks(phi, phi, phi, L, mom),
                 lambda: binding.doublet_blocks(phi, phi, L, mom), lambda: binding.projection(phi, phi, L),
                 lambda: binding.blocks_noalloc(phi, L, mom, None, None),
                 lambda: binding.baryon_dense(torch.zeros((1, 1, 4), dtype=torch.complex128), 4)):
        with pytest.raises(ValueError):
            call()
    n = binding.lanczos_workspace_size(L, 1, 4, 20)
    assert n >= 8 * 3 * L ** 3 * (20 + 1 + 4)
    with pytest.raises(binding.LaphError):
        binding.lanczos_workspace_size(L, 1, 30, 20)                         # n_ev > n_krylov
    assert np.isfinite(n)


def test_binding_structures_match_the_header(tmp_path):
    """Every struct the binding declares with ctypes has the size and field offsets that a C compiler gives the
    same struct from include/laph.h (a mismatch would let the library write past a Python-side structure)."""
    import shutil
    import subprocess
    from paper_2510_26313_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [binding.laph_instance, binding.laph_plan_options, binding.laph_tune_record,
               binding.laph_lanczos_params, binding.laph_lanczos_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "laph.h"', 'int main(void) {']
    for st in structs:
        name = st.__name__
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ['    return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_side = {(a, b): int(c) for a, b, c in (l.split() for l in out if l.strip())}
    for st in structs:
        name = st.__name__
        assert c_side[(name, "size")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert c_side[(name, field)] == getattr(st, field).offset, (name, field)
