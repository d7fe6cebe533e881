"""Bit-exact parity of the GPU binning (LR cell sort) and HR reordering with
the oracle's stable counting sort on the grid contract."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def _ctx(sc, **kw):
    import paper_2308_01629_gb300 as gs
    return gs, gs.Context(sc, **kw)


def _oracle_grid(orc, sc):
    # the ABI receives r_low and the box as float32
    return orc.grid(float(np.float32(sc["r_low"])), np.float32(sc["box_lo"]).astype(float),
                    np.float32(sc["box_hi"]).astype(float))


@pytest.mark.parametrize("make", [scenes.cube, scenes.funnel, scenes.digging,
                                  lambda: scenes.translated(scenes.cube(), (-0.25, -0.25, -0.25))])
def test_grid_contract_matches_oracle(orc, make):
    sc = make()
    gs, ctx = _ctx(sc)
    o, h, ih, dims = _oracle_grid(orc, sc)
    g = ctx.grid
    assert list(g.origin) == list(o) and np.float32(g.h) == np.float32(h) and np.float32(g.inv_h) == ih
    assert list(g.dims) == list(dims) and g.n_cell == int(np.prod(dims))
    ctx.close()


def _check_lr_binning(orc, sc, ctx, gs):
    ctx.bin_low()
    idx = ctx.read(gs.GS_FIELD_LR_SORTED_INDEX)
    start = ctx.read(gs.GS_FIELD_LR_CELL_START)
    o, h, ih, dims = _oracle_grid(orc, sc)
    keys = orc.cell_keys(sc["lr_pos"], o, ih, dims)
    nc = int(np.prod(dims))
    ref_idx, ref_start = orc.counting_sort(keys, nc)
    np.testing.assert_array_equal(idx, ref_idx)
    np.testing.assert_array_equal(start[:nc + 1], ref_start)
    assert np.all(start[nc + 1:] == len(idx))      # the scene's padding cell is empty


def _cube_at_origin():
    """The cube moved to straddle the origin: a negative grid origin and
    coordinates of both signs."""
    return scenes.translated(scenes.cube(), (-0.25, -0.25, -0.25))


@pytest.mark.parametrize("make", [scenes.cube, scenes.funnel, scenes.digging, _cube_at_origin])
def test_lr_binning_bit_exact(orc, make):
    sc = make()
    gs, ctx = _ctx(sc)
    _check_lr_binning(orc, sc, ctx, gs)
    ctx.close()


def test_lr_binning_outside_box_and_degenerate(orc):
    rng = np.random.default_rng(21)
    base = scenes.cube()
    for case in ("outside", "one_point", "piles", "single", "empty"):
        sc = dict(base)
        if case == "outside":
            lr = np.zeros((3001, 4), np.float32)
            lr[:, :3] = rng.uniform(-0.2, 0.7, size=(3001, 3))
        elif case == "piles":   # cells of 40, 100 and 300 among ordinary ones
            lr = base["lr_pos"].copy()
            pts = rng.uniform(0.1, 0.4, size=(6, 3)).astype(np.float32)
            lr[:120, :3] = np.repeat(pts[:3], 40, axis=0)
            lr[120:320, :3] = np.repeat(pts[3:5], 100, axis=0)
            lr[320:620, :3] = pts[5]
        elif case == "one_point":
            lr = np.zeros((5000, 4), np.float32)
            lr[:, :3] = 0.25
        elif case == "single":
            lr = np.array([[0.1, 0.2, 0.3, 1.0]], np.float32)
        else:
            lr = np.zeros((0, 4), np.float32)
        sc.update(lr_pos=lr, lr_vel=np.zeros_like(lr), hr_pos=np.zeros((0, 4), np.float32),
                  hr_vel=np.zeros((0, 4), np.float32), ratio=1)
        sc["hr_pos"] = np.repeat(lr, 1, axis=0).copy()
        sc["hr_vel"] = np.zeros_like(sc["hr_pos"])
        gs, ctx = _ctx(sc)
        _check_lr_binning(orc, sc, ctx, gs)
        ctx.close()


@pytest.mark.parametrize("make", [scenes.cube, scenes.funnel, scenes.digging])
def test_hr_reorder_bit_exact_and_roundtrip(orc, make):
    sc = make()
    if make is scenes.cube:
        sc = scenes.stir(sc, seed=3)
    _check_hr_reorder(orc, sc)


def _wide_box(sc):
    """The cube in a 5 m box: 8 x cells fine keys far outnumber the HR set,
    so the reorder takes the radix sort instead of the counting sort."""
    sc = dict(sc)
    sc["box_lo"] = [-2.0, -2.0, -2.0]
    sc["box_hi"] = [3.0, 3.0, 3.0]
    return sc


def _clumped(sc):
    """HR particles piled on points: one fine cell of more than 3000 entries
    (a block's LSD passes over many tiles), 40 of 50 or more and 10 of 150
    or more (one warp each, the two register widths)."""
    sc = dict(sc)
    hr = sc["hr_pos"].copy()
    pts = np.random.default_rng(7).uniform(0.15, 0.35, size=(50, 3)).astype(np.float32)
    hr[:3000, :3] = np.float32([0.25, 0.25, 0.3])
    hr[3000:5000, :3] = np.repeat(pts[:40], 50, axis=0)
    hr[5000:6500, :3] = np.repeat(pts[40:], 150, axis=0)
    sc["hr_pos"] = hr
    return sc


@pytest.mark.parametrize("case", ["wide_box", "clumped", "clumped_wide_box", "clumped_three_passes"])
def test_hr_reorder_bit_exact_sort_paths_and_big_cells(orc, case):
    # 74,088 HR slots need 17 index bits: three 8-bit passes, the last one
    # ending in the scratch range (copied back); 8,000 slots need two
    n_side = 21 if case == "clumped_three_passes" else 10
    sc = scenes.stir(scenes.cube(n_side=n_side), seed=5)
    if "clumped" in case:
        sc = _clumped(sc)
    if "wide" in case:
        sc = _wide_box(sc)
    _check_hr_reorder(orc, sc)
    if case == "wide_box":   # 4.6M cells: the cell-start scan over more than 1,024 tiles
        gs, ctx = _ctx(sc)
        assert ctx.grid.n_cell > 1024 * 4096
        _check_lr_binning(orc, sc, ctx, gs)
        ctx.close()


def _check_hr_reorder(orc, sc):
    gs, ctx = _ctx(sc)
    ctx.resort_high()
    m = len(sc["hr_pos"])
    keys = ctx.read(gs.GS_FIELD_HR_SORTED_KEY)[:m]
    internal = ctx.read(gs.GS_FIELD_HR_POS_INTERNAL)[:m]
    o, h, ih, dims = _oracle_grid(orc, sc)
    fk = orc.cell_keys(sc["hr_pos"], o, ih, dims, fine=True)
    ref_idx, _ = orc.counting_sort(fk, int(np.prod(dims)) * 8)
    np.testing.assert_array_equal(internal[:, 3].view(np.uint32), ref_idx)
    np.testing.assert_array_equal(keys, fk[ref_idx])
    np.testing.assert_array_equal(internal[:, :3], sc["hr_pos"][ref_idx, :3])
    # exchanged in original-id order, untouched by the reorder
    np.testing.assert_array_equal(ctx.read(gs.GS_FIELD_HR_POS), sc["hr_pos"])
    np.testing.assert_array_equal(ctx.read(gs.GS_FIELD_HR_VEL), sc["hr_vel"])
    # a second reorder of the already ordered set is the identity on its order
    ctx.resort_high()
    np.testing.assert_array_equal(ctx.read(gs.GS_FIELD_HR_POS_INTERNAL)[:m], internal)
    ctx.close()


def test_hr_velocity_write_after_reorder(orc):
    sc = scenes.stir(scenes.cube(), seed=4)
    gs, ctx = _ctx(sc)
    ctx.resort_high()
    v = np.random.default_rng(5).normal(size=sc["hr_vel"].shape).astype(np.float32)
    v[:, 3] = 0
    ctx.write(gs.GS_FIELD_HR_VEL, v)
    np.testing.assert_array_equal(ctx.read(gs.GS_FIELD_HR_VEL), v)
    np.testing.assert_array_equal(ctx.read(gs.GS_FIELD_HR_POS), sc["hr_pos"])
    ctx.write(gs.GS_FIELD_HR_POS, sc["hr_pos"])
    np.testing.assert_array_equal(ctx.read(gs.GS_FIELD_HR_VEL), v)
    ctx.close()
