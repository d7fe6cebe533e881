"""Binning without allocation (gs_bin_points_static): the entry point for
callers that cannot call cudaMalloc, e.g. code recorded into a CUDA graph
under the global capture mode (where an allocation is an error) or a
real-time loop that must not take cudaMalloc's implicit synchronization.

Its bins are compared with the oracle's stable counting sort of the same
grid contract, including points outside the grid, no point and a single
point, at key widths of one, two and three 8-bit radix passes and at the
largest accepted count; with gs_bin_low on two calls in a row that share
the static scratch; and inside a captured CUDA graph.  This file is
collected last on purpose."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def _grid(gs, orc, r_low, lo, hi):
    o, h, inv_h, dims = orc.grid(r_low, lo, hi)
    g = gs.gs_grid_info()
    for k in range(3):
        g.origin[k] = float(o[k])
        g.dims[k] = int(dims[k])
    g.h, g.inv_h = float(h), float(inv_h)
    g.n_cell = int(np.prod(dims.astype(np.int64)))
    return g, (o, inv_h, dims)


def _oracle_bins(orc, pos4, contract):
    o, inv_h, dims = contract
    keys = orc.cell_keys(pos4, o, inv_h, dims)
    return orc.counting_sort(keys, int(np.prod(dims.astype(np.int64))))


def _static(gs, pos4, grid, stream=None):
    import torch
    n = len(pos4)
    pos = torch.from_numpy(np.ascontiguousarray(pos4, np.float32).reshape(-1, 4)).cuda()
    idx = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    start = torch.full((int(grid.n_cell) + 1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = gs.gs_bin_points_static(pos.data_ptr() if n else None, n, grid, idx.data_ptr(), start.data_ptr(), stream)
    torch.cuda.synchronize()
    return rc, idx.cpu().numpy().view(np.uint32)[:n], start.cpu().numpy().view(np.uint32)


def _points(rng, n, lo, hi, outside=0.0):
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    span = hi - lo
    p = np.zeros((n, 4), np.float32)
    p[:, :3] = rng.uniform(lo - outside * span, hi + outside * span, size=(n, 3))
    return p


@pytest.mark.parametrize("case", ["one_pass", "two_passes", "three_passes", "outside", "single", "empty", "max"])
def test_static_binning_matches_oracle_counting_sort(orc, case):
    import paper_2308_01629_gb300 as gs
    rng = np.random.default_rng(["one_pass", "two_passes", "three_passes", "outside", "single", "empty",
                                 "max"].index(case) + 11)
    r = 0.01
    # cell side ~0.03: 6^3 = 216 cells (8 key bits), 27^3 = 19683 (15),
    # 50 x 50 x 40 = 100,000 (17)
    box = {"one_pass": (0.18, 0.18, 0.18), "two_passes": (0.8, 0.8, 0.8), "three_passes": (1.5, 1.5, 1.2),
           "outside": (0.8, 0.8, 0.8), "single": (0.8, 0.8, 0.8), "empty": (0.8, 0.8, 0.8),
           "max": (1.5, 1.5, 1.2)}[case]
    lo, hi = (0.0, 0.0, 0.0), box
    grid, contract = _grid(gs, orc, r, lo, hi)
    n = {"one_pass": 5000, "two_passes": 20000, "three_passes": 60000, "outside": 20000, "single": 1, "empty": 0,
         "max": gs.GS_STATIC_BIN_MAX_POINTS}[case]
    pos = _points(rng, n, lo, hi, outside=0.3 if case == "outside" else 0.0)
    if case == "outside":
        assert ((pos[:, :3] < 0) | (pos[:, :3] > np.asarray(hi))).any(axis=1).mean() > 0.3
    rc, idx, start = _static(gs, pos, grid)
    assert rc == gs.GS_OK
    ref_idx, ref_start = _oracle_bins(orc, pos, contract)
    np.testing.assert_array_equal(idx, ref_idx)
    np.testing.assert_array_equal(start, ref_start)


def _reference(gs, sc):
    ctx = gs.Context(sc)
    ctx.bin_low()
    idx = ctx.read(gs.GS_FIELD_LR_SORTED_INDEX)
    grid = ctx.grid
    start = ctx.read(gs.GS_FIELD_LR_CELL_START)[:int(grid.n_cell) + 1]   # without the scene's padding cell
    ctx.close()
    return idx, start, grid


def test_static_scratch_binning_matches_gs_bin_low():
    import paper_2308_01629_gb300 as gs
    # two calls in a row: the second one finds the first one's data in the
    # shared scratch and must not depend on it
    for make in (scenes.funnel, scenes.cube):
        sc = make()
        ref_idx, ref_start, grid = _reference(gs, sc)
        rc, idx, start = _static(gs, sc["lr_pos"], grid)
        assert rc == gs.GS_OK
        np.testing.assert_array_equal(idx, ref_idx)
        np.testing.assert_array_equal(start, ref_start)


def test_static_binning_in_a_captured_graph(orc):
    """After one call outside a capture (the first call on a device looks
    up the scratch's address), a call recorded into a CUDA graph under the
    global capture mode replays to the same bins."""
    import torch

    import paper_2308_01629_gb300 as gs
    rng = np.random.default_rng(5)
    lo, hi = (0.0, 0.0, 0.0), (0.8, 0.8, 0.8)
    grid, contract = _grid(gs, orc, 0.01, lo, hi)
    pts = _points(rng, 30000, lo, hi)
    pos = torch.from_numpy(pts).cuda()
    idx = torch.full((len(pts),), -1, dtype=torch.int32, device="cuda")
    start = torch.full((int(grid.n_cell) + 1,), -1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    assert gs.gs_bin_points_static(pos.data_ptr(), len(pts), grid, idx.data_ptr(), start.data_ptr(),
                                   s.cuda_stream) == gs.GS_OK
    s.synchronize()
    idx.fill_(-1)
    start.fill_(-1)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="global"):
        rc = gs.gs_bin_points_static(pos.data_ptr(), len(pts), grid, idx.data_ptr(), start.data_ptr(),
                                     s.cuda_stream)
    assert rc == gs.GS_OK
    assert (idx.cpu().numpy() == -1).all()   # captured, not run
    graph.replay()
    torch.cuda.synchronize()
    ref_idx, ref_start = _oracle_bins(orc, pts, contract)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), ref_idx)
    np.testing.assert_array_equal(start.cpu().numpy().view(np.uint32), ref_start)


def test_static_scratch_rejects_oversize():
    import torch

    import paper_2308_01629_gb300 as gs
    sc = scenes.cube()
    _, _, grid = _reference(gs, sc)
    n = gs.GS_STATIC_BIN_MAX_POINTS + 1
    pos = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    idx = torch.zeros(n, dtype=torch.int32, device="cuda")
    start = torch.zeros(int(grid.n_cell) + 1, dtype=torch.int32, device="cuda")
    # refused on the host before anything is enqueued
    rc = gs.gs_bin_points_static(pos.data_ptr(), n, grid, idx.data_ptr(), start.data_ptr(), None)
    assert rc == gs.GS_ERR_CAPACITY
    torch.cuda.synchronize()
