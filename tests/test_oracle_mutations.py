"""The oracle's pins must catch planted mistakes.

Each case copies ``oracle/laph_oracle.c``, plants one plausible mistake
(wrong epsilon sign, missing or misplaced conjugation, wrong phase sign,
transposed site axes, swapped packing, transposed meson output; for the
general-field routines: fields bound to the wrong index, a colour index
swapped, a conjugation on the wrong field, transposed or misindexed
outputs; for the Laplacian: a dropped dagger, the backward link at the
wrong site, a wrong diagonal, a wrong periodic wrap), builds it and runs the
pin tests against it: they must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "laph_oracle.c")

MUTATIONS = {
    "eps_sign": ("{+1.0, +1.0, +1.0, -1.0, -1.0, -1.0}", "{+1.0, +1.0, -1.0, -1.0, -1.0, -1.0}"),
    "meson_no_conj": ("cmul(cconj(phi_at(phi, V, i, x, a)), phi_at(phi, V, j, x, a))",
                      "cmul(phi_at(phi, V, i, x, a), phi_at(phi, V, j, x, a))"),
    "meson_conj_second": ("cmul(cconj(phi_at(phi, V, i, x, a)), phi_at(phi, V, j, x, a))",
                          "cmul(phi_at(phi, V, i, x, a), cconj(phi_at(phi, V, j, x, a)))"),
    "phase_sign": ("double ang = -2.0 * M_PI", "double ang = 2.0 * M_PI"),
    "site_axes": ("int64_t x0 = x % L, x1 = (x / L) % L,", "int64_t x1 = x % L, x0 = (x / L) % L,"),
    "packing_swap": ("ijk[3 * idx] = i;\n                ijk[3 * idx + 1] = j;",
                     "ijk[3 * idx] = j;\n                ijk[3 * idx + 1] = i;"),
    "meson_transpose": ("out[2 * ((p * (int64_t)N + i) * N + j)] = acc[p].re;",
                        "out[2 * ((p * (int64_t)N + j) * N + i)] = acc[p].re;"),
    # three-field triplets and two-field doublets
    "fields_swapped": ("cmul(cmul(phi_at(f1, V, i, x, EPS_PERM[q][0]), phi_at(f2, V, j, x, EPS_PERM[q][1])),",
                       "cmul(cmul(phi_at(f2, V, i, x, EPS_PERM[q][0]), phi_at(f1, V, j, x, EPS_PERM[q][1])),"),
    "fields_colour_swap": ("phi_at(f3, V, k, x, EPS_PERM[q][2]));", "phi_at(f3, V, k, x, EPS_PERM[q][1]));"),
    "doublet_conj_second": ("cmul(cconj(phi_at(f1, V, i, x, a)), phi_at(f2, V, j, x, a))",
                            "cmul(phi_at(f1, V, i, x, a), cconj(phi_at(f2, V, j, x, a)))"),
    "doublet_transpose": ("int64_t o = 2 * ((p * (int64_t)N1 + i) * N2 + j);",
                          "int64_t o = 2 * ((p * (int64_t)N1 + j) * N2 + i);"),
    "projection_counts": ("int i = (int)(ij / N2), j = (int)(ij % N2);", "int i = (int)(ij / N1), j = (int)(ij % N1);"),
    # covariant Laplacian
    "laplacian_no_dagger": ("cplx wf = cmul(cconj((cplx){w[0], w[1]}), phi_at(f, V, (int)n, dn, b));",
                            "cplx wf = cmul((cplx){w[0], w[1]}, phi_at(f, V, (int)n, dn, b));"),
    "laplacian_backward_link_site": ("const double *w = U + 2 * (((mu * V + dn) * 3 + b) * 3 + a);",
                                     "const double *w = U + 2 * (((mu * V + x) * 3 + b) * 3 + a);"),
    "laplacian_diagonal": ("acc[a].re = 6.0 * v.re;", "acc[a].re = 4.0 * v.re;"),
    "laplacian_wrap": ("int64_t up = x + (c[mu] == L - 1 ? -(int64_t)(L - 1) * stride[mu] : stride[mu]);",
                       "int64_t up = x + (c[mu] == L - 1 ? 0 : stride[mu]);"),
    "triplet_dense_index": ("ijk[3 * e + 2] = (int32_t)(e % N);", "ijk[3 * e + 2] = (int32_t)((e / N) % N);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_fail_on_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "laph_oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "liblaph_oracle_mut.so"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", str(lib),
                    str(mutated), "-lm"], check=True)
    env = dict(os.environ, LAPH_ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_fields_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_laplacian_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutation {name}:\n{r.stdout[-2000:]}"
