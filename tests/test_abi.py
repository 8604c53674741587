"""The C ABI library builds, loads and exports every function include/*.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lp_\w+)\s*\(", text, flags=re.M):
            names.add(mt.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("lp_create", "lp_solve", "lp_get_solution", "lp_get_basis", "lp_set_basis",
                 "lp_destroy", "lp_price_static"):
        assert want in names, want


def test_library_exports_every_declared_symbol():
    from paper_1803_04378_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_imports_without_gpu():
    from paper_1803_04378_gb300 import lpgb
    o = lpgb.default_options()
    assert o.reinvert_every == 64 and o.tabu_tenure == 7 and o.bland_after == 50
    assert abs(o.tol_d - 1e-9) < 1e-24 and abs(o.tol_tie - 1e-12) < 1e-27
    assert lpgb.lib().lp_strerror(-4) == b"singular basis during reinversion"


def test_option_defaults_and_validation_on_host():
    """lp_default_options and lp_create's argument checks are host code: they
    run (and reject bad options before any device call) without a GPU."""
    import ctypes

    import numpy as np

    from paper_1803_04378_gb300 import lpgb
    o = lpgb.default_options()
    assert o.engine == lpgb.LP_ENGINE_STRUCTURED and o.anticycling == lpgb.LP_ANTICYCLING_TABU
    assert o.reinvert_refine == 1 and o.refine_tol == 2.0 ** -26
    A = np.ones((3, 4))
    b = np.ones(3)
    c = np.ones(4)
    for bad in (dict(reinvert_refine=2), dict(refine_tol=1e-6), dict(refine_tol=-1.0), dict(refine_tol=float("nan")),
                dict(engine=3), dict(anticycling=2), dict(price_mode=3), dict(graph_iters=0), dict(tol_piv=0.0)):
        h = ctypes.c_void_p()
        rc = lpgb.lib().lp_create(ctypes.byref(h), 3, 4, lpgb._ptr(A), lpgb._ptr(b), lpgb._ptr(c), 0,
                                  ctypes.byref(lpgb.default_options(**bad)))
        assert rc == lpgb.LP_ERR_INVALID_ARG, bad
        assert not h.value
    A[0, 0] = float("inf")
    h = ctypes.c_void_p()
    assert lpgb.lib().lp_create(ctypes.byref(h), 3, 4, lpgb._ptr(A), lpgb._ptr(b), lpgb._ptr(c), 0,
                                ctypes.byref(lpgb.default_options())) == lpgb.LP_ERR_INVALID_ARG
    # a large host A (4.4 M entries) is checked by several threads; the last
    # entry of the last thread's share, and the first of the first
    m, n = 1100, 4000
    Ab, bb, cb = np.ones((m, n)), np.ones(m), np.ones(n)
    for pos in ((m - 1, n - 1), (0, 0), (m // 2, 7)):
        Ab[pos] = float("nan") if pos[0] else float("-inf")
        h = ctypes.c_void_p()
        assert lpgb.lib().lp_create(ctypes.byref(h), m, n, lpgb._ptr(Ab), lpgb._ptr(bb), lpgb._ptr(cb), 0,
                                    ctypes.byref(lpgb.default_options())) == lpgb.LP_ERR_INVALID_ARG, pos
        assert not h.value
        Ab[pos] = 1.0


def test_struct_layout_matches_the_binding(tmp_path):
    """The ctypes mirrors of the ABI's structs have the C layout: a C
    program compiled against the header prints every field's offset and the
    structs' sizes."""
    import ctypes
    import shutil
    import subprocess

    from paper_1803_04378_gb300 import lpgb
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lpgb.h"', "int main(void) {"]
    structs = ((lpgb.lp_options, "lp_options"), (lpgb.lp_result, "lp_result"),
               (lpgb.lp_batch_result, "lp_batch_result"))
    for st, cname in structs:
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for name, _ in st._fields_:
            lines.append(f'printf("{cname} {name} %zu\\n", offsetof({cname}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I", include, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (x.split() for x in out if x)}
    for st, cname in structs:
        assert got[(cname, "sizeof")] == ctypes.sizeof(st)
        for name, _ in st._fields_:
            assert got[(cname, name)] == getattr(st, name).offset, (cname, name)
