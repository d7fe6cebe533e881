"""The C ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/gs.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(gs_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2308_01629_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_wraps_every_declared_symbol():
    import paper_2308_01629_gb300 as gs
    for n in declared_functions():
        assert hasattr(gs, n), n


def test_default_params_are_the_papers():
    import paper_2308_01629_gb300 as gs
    p = gs.gs_default_params()
    assert abs(p.c1 - 512.0 / 729.0) < 1e-7 and abs(p.c2 - 0.6) < 1e-7
    assert abs(p.mu_s - 0.35) < 1e-7 and abs(p.mu_k - 0.30) < 1e-7
    assert p.n_stab == 2 and abs(p.gravity[2] + 9.81) < 1e-6
