"""The binning entry point that allocates nothing (for callers that cannot
call cudaMalloc, e.g. inside a CUDA graph capture under the global capture
mode or in a real-time loop that must not synchronize the device) gives the
same bins as gs_bin_low, on two calls in a row that share its static
scratch.  This file is collected last on purpose."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def _reference(gs, sc):
    ctx = gs.Context(sc)
    ctx.bin_low()
    idx = ctx.read(gs.GS_FIELD_LR_SORTED_INDEX)
    grid = ctx.grid
    start = ctx.read(gs.GS_FIELD_LR_CELL_START)[:int(grid.n_cell) + 1]   # without the scene's padding cell
    ctx.close()
    return idx, start, grid


def _static(gs, sc, grid):
    import torch
    n = len(sc["lr_pos"])
    pos = torch.from_numpy(sc["lr_pos"]).cuda()
    idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    start = torch.full((int(grid.n_cell) + 1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = gs.gs_bin_points_static(pos.data_ptr(), n, grid, idx.data_ptr(), start.data_ptr(), None)
    torch.cuda.synchronize()
    return rc, idx.cpu().numpy().view(np.uint32), start.cpu().numpy().view(np.uint32)


def test_static_scratch_binning_matches_gs_bin_low():
    import paper_2308_01629_gb300 as gs
    # two calls in a row: the second one finds the first one's data in the
    # shared scratch and must not depend on it
    for make in (scenes.funnel, scenes.cube):
        sc = make()
        ref_idx, ref_start, grid = _reference(gs, sc)
        rc, idx, start = _static(gs, sc, grid)
        assert rc == gs.GS_OK
        np.testing.assert_array_equal(idx, ref_idx)
        np.testing.assert_array_equal(start, ref_start)


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
