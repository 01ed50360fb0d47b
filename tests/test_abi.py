"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every function that include/sph.h declares, and its
host-only sizing/validation logic behaves."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2405_03980_gb300 import _binding as B
from paper_2405_03980_gb300 import build as Bld
from paper_2405_03980_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    return sorted(set(re.findall(r"SPH_API[^;(]*?\b(sph_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    Bld.build()
    return B.lib()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.exported_symbols()) == names


def test_status_strings(lib):
    for st in range(-10, 1):
        assert B.sph_status_string(st) != "unknown status"


def test_params_default_matches_workload_recipe(lib):
    p = B.sph_params_default(10.0, 20.0, 0.1)
    w = synth.workload_params(10.0, 20, 0.1)
    for k in ("dx", "h", "rho0", "alpha_P", "p0", "beta_P", "eta_bar", "eta_r", "C_l",
              "C_T", "C_omega", "mass_ratio", "inertia_coef", "Omega", "dt", "col_dist",
              "col_e"):
        assert getattr(p, k) == pytest.approx(w[k], rel=1e-15), k
    assert list(p.box_lo) == pytest.approx(list(w["box_lo"]))
    assert list(p.box_hi) == pytest.approx(list(w["box_hi"]))


def test_buffer_sizes_scale_and_validate(lib):
    c = synth.workload("cyl_8960")
    p = B.params_from_dict(c.params)
    s1 = B.sph_state_bytes(p, [c.n])
    w1 = B.sph_workspace_bytes(p, [c.n])
    assert s1 > 200 * c.n and w1 > 160 * 4 * c.n
    s2 = B.sph_state_bytes([p, p], [c.n, c.n])
    assert s2 > 1.9 * s1
    bad = B.params_from_dict(dict(c.params, h=-1.0))
    assert B.sph_state_bytes(bad, [c.n]) == 0
    bad = B.params_from_dict(dict(c.params, alpha_P=7.5))
    assert B.sph_workspace_bytes(bad, [c.n]) == 0
    bad = B.params_from_dict(c.params, nbr_cap=8)
    assert B.sph_workspace_bytes(bad, [c.n]) == 0
    # a periodic z period shorter than three cells of side 2h is rejected
    bad = B.params_from_dict(dict(c.params, box_hi=(c.params["box_hi"][0], c.params["box_hi"][1], 6.0)))
    assert B.sph_state_bytes(bad, [c.n]) == 0
    # unknown flag bits, and a collision model outside (0, 2h) x [0, 1]
    bad = B.params_from_dict(c.params, flags=512)
    assert B.sph_state_bytes(bad, [c.n]) == 0
    col = B.SPH_FLAGS_DEFAULT | B.SPH_COLLISION | B.SPH_PFILTER
    assert B.sph_state_bytes(B.params_from_dict(c.params, flags=col), [c.n]) > 0
    for kw in (dict(col_dist=2.0 * c.params["h"]), dict(col_dist=0.0), dict(col_e=1.5),
               dict(col_e=-0.1)):
        bad = B.params_from_dict(dict(c.params, **kw), flags=col)
        assert B.sph_state_bytes(bad, [c.n]) == 0, kw
    # (the collision parameters are not checked while the model is off)
    assert B.sph_state_bytes(B.params_from_dict(dict(c.params, col_e=3.0)), [c.n]) > 0
    # mixed precision within one batch is rejected
    q = B.params_from_dict(c.params, precision=B.SPH_MIXED)
    assert B.sph_state_bytes([p, q], [c.n, c.n]) == 0
    # empty instances, and more particles than a 26-bit list index can name
    assert B.sph_state_bytes(p, [0]) == 0
    assert B.sph_workspace_bytes([p, p], [c.n, 0]) == 0
    assert B.sph_state_bytes(p, [(1 << 26) + 1]) == 0
    assert B.sph_state_bytes([p, p], [1 << 25, (1 << 25) + 1]) == 0


def test_init_rejects_bad_arguments_without_touching_the_gpu(lib):
    c = synth.workload("cyl_8960")
    p = B.params_from_dict(c.params)
    ctx = C.c_void_p()
    # null pointers are rejected before any CUDA call
    st = lib.sph_init(C.byref(ctx), C.byref(p), c.n, None, None, None, None, None, 0, None, 0, None)
    assert st == -1 and not ctx.value
    assert lib.sph_step(None, 1) == -1
    assert lib.sph_destroy(None) == 0


def test_params_struct_layout_matches_header(tmp_path):
    """The ctypes mirror of sph_params has the C layout of include/sph.h."""
    prog = tmp_path / "layout.c"
    fields = [f for f, _ in B.SphParams._fields_]
    body = "\n".join(f'  printf("%zu\\n", offsetof(sph_params, {f}));' for f in fields)
    prog.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"sph.h\"\n"
                    "int main(void) {\n" + body +
                    '\n  printf("%zu\\n", sizeof(sph_params));\n  return 0;\n}\n')
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(prog), "-o",
                    str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [getattr(B.SphParams, f).offset for f in fields] + [C.sizeof(B.SphParams)]
    assert out == want


def test_checked_library_builds_and_exports_the_same_symbols():
    """The checked variant (-DSPH_CHECKED, device bounds checks) builds for
    sm_103a from its own objects and exports the same C ABI."""
    path = Bld.build(checked=True)
    assert path.endswith("libsph_gb300_checked.so") and os.path.exists(path)
    L = C.CDLL(path)
    for n in _declared():
        assert hasattr(L, n), n
    L.sph_status_string.restype = C.c_char_p
    assert b"bounds" in L.sph_status_string(-10)
