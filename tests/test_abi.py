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


def test_static_binning_refuses_bad_arguments_before_any_device_work():
    """gs_bin_points_static checks its arguments on the host and returns
    before any CUDA call, so these refusals run without a GPU (the pointers
    are never dereferenced)."""
    import paper_2308_01629_gb300 as gs
    g = gs.gs_grid_info()
    for k in range(3):
        g.origin[k] = 0.0
        g.dims[k] = 8
    g.h, g.inv_h, g.n_cell = 0.03, 1.0 / 0.03, 512
    ok_pos, ok_idx, ok_start = 1 << 20, 1 << 21, 1 << 22
    call = gs.gs_bin_points_static
    assert call(ok_pos + 8, 10, g, ok_idx, ok_start) == gs.GS_ERR_ARG      # positions not 16-byte aligned
    assert call(ok_pos, 10, g, ok_idx, ok_start + 2) == gs.GS_ERR_ARG      # cell starts not 4-byte aligned
    assert call(ok_pos, 10, g, ok_idx + 1, ok_start) == gs.GS_ERR_ARG      # indices not 4-byte aligned
    assert call(ok_pos, 10, g, ok_idx, None) == gs.GS_ERR_ARG
    assert call(ok_pos, gs.GS_STATIC_BIN_MAX_POINTS + 1, g, ok_idx, ok_start) == gs.GS_ERR_CAPACITY
    g.dims[0] = (1 << 20) + 1                                              # wider than gs_create allows
    g.n_cell = g.dims[0] * 64
    assert call(ok_pos, 10, g, ok_idx, ok_start) == gs.GS_ERR_ARG
    g.dims[0] = 8
    g.n_cell = 511                                                         # inconsistent cell count
    assert call(ok_pos, 10, g, ok_idx, ok_start) == gs.GS_ERR_ARG


def test_hr_slab_ranges_tile_the_slots_by_whole_items():
    """gs_hr_slab_range is host arithmetic: the slabs of a partition are
    contiguous, start at 0, end at n_slots, are made of whole 32-slot items
    and differ by one item at most; bad arguments give GS_ERR_ARG."""
    import paper_2308_01629_gb300 as gs
    for n_slots in (0, 32, 96, 32 * 1000, 32 * 63157):
        for n_parts in (1, 2, 3, 7, 8, 64, 4096):
            ranges = []
            for part in range(n_parts):
                rc, b, e = gs.gs_hr_slab_range(n_slots, part, n_parts)
                assert rc == gs.GS_OK
                ranges.append((b, e))
            assert ranges[0][0] == 0 and ranges[-1][1] == n_slots
            for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
                assert e0 == b1
            sizes = [e - b for b, e in ranges]
            assert all(s % 32 == 0 and s >= 0 for s in sizes)
            assert max(sizes) - min(sizes) <= 32
    for args in ((33, 0, 2), (-32, 0, 1), (64, 2, 2), (64, -1, 2), (64, 0, 0), (64, 0, 4097)):
        assert gs.gs_hr_slab_range(*args)[0] == gs.GS_ERR_ARG


def test_volume_sampler_refuses_bad_arguments_before_any_device_work():
    """gs_sample_volume checks its arguments on the host: these calls return
    before touching a GPU (none is present here)."""
    import numpy as np

    import paper_2308_01629_gb300 as gs
    V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    T = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]])
    C = np.array([[0.1, 0.1, 0.1]])
    assert gs.gs_sample_volume(V, T, C, 0.0)[0] == gs.GS_ERR_ARG              # r <= 0
    assert gs.gs_sample_volume(V, T, C, float("nan"))[0] == gs.GS_ERR_ARG
    assert gs.gs_sample_volume(V, T + 1, C, 0.1)[0] == gs.GS_ERR_ARG           # index 4 of 4 vertices
    assert gs.gs_sample_volume(V, -T, C, 0.1)[0] == gs.GS_ERR_ARG
    assert gs.gs_sample_volume(V, T, [[0.1, float("inf"), 0]], 0.1)[0] == gs.GS_ERR_DOMAIN
    V2 = V.copy()
    V2[1, 0] = float("nan")
    assert gs.gs_sample_volume(V2, T, C, 0.1)[0] == gs.GS_ERR_DOMAIN
    assert gs.gs_sample_volume(V * 1e6, T, C, 1e-6)[0] == gs.GS_ERR_ARG       # too many cells
    # surface candidates must lie on the mesh: within 0.15 r of its bounding box
    assert gs.gs_sample_surface(V, [[0.5, 0.5, -0.02]], 0.1)[0] == gs.GS_ERR_ARG
    assert gs.gs_sample_surface(V, [[1.0, 0.5, 0.0], [1.02, 0.0, 0.0]], 0.1)[0] == gs.GS_ERR_ARG
    assert gs.gs_sample_surface(V, [[0.1, 0.1, 0.0]], 0.0)[0] == gs.GS_ERR_ARG
