"""One scene's HR set split by slabs of its cell-ordered slots, the LR state
computed by every part (the multi-GPU partition, on one GPU): two contexts
restricted to the two halves, their slabs put together, equal the whole
context bit for bit, frame by frame and across HR reorders; the exchange
(gather-back) is the only step between the parts.  Also the partial state's
refusals and the gather-back's checks."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0


def _bucket_scene(size=0.5):
    sc = dict(scenes.digging(size=size))
    sc["sdfs"] = [sc["sdfs"][0], scenes.bucket_sdf(0.0)]
    return sc


def _internal(gs, ctx):
    return ctx.read(gs.GS_FIELD_HR_POS_INTERNAL), ctx.read(gs.GS_FIELD_HR_VEL_INTERNAL)


@pytest.mark.parametrize("graphs", [False, True])
@pytest.mark.parametrize("n_parts", [2, 3])
def test_slab_contexts_put_together_equal_the_whole_context(graphs, n_parts):
    import paper_2308_01629_gb300 as gs
    sc = _bucket_scene()
    whole = gs.Context(sc)
    parts = [gs.Context(sc) for _ in range(n_parts)]
    every = 8                                            # the default HR reorder period
    for k, c in enumerate(parts):
        c.set_hr_slab(k, n_parts)
    for c in [whole] + parts:
        c.set_graphs(graphs)
    ranges = [c.hr_slab_range(k, n_parts) for k, c in enumerate(parts)]
    assert ranges[0][0] == 0 and ranges[-1][1] == whole.hr_slots
    assert all(ranges[k][1] == ranges[k + 1][0] for k in range(n_parts - 1))
    nframes = 2 * every + 3   # three reorders (frames 0, 8, 16)
    for f in range(nframes):
        if f > 0 and f % every == 0:
            # the gather-back before the reorder: every part's own slab
            pieces = [_internal(gs, c) for c in parts]
            pos = np.concatenate([pieces[k][0][b:e] for k, (b, e) in enumerate(ranges)])
            vel = np.concatenate([pieces[k][1][b:e] for k, (b, e) in enumerate(ranges)])
            for c in parts:
                c.hr_slab_assemble(pos, vel)
        for c in [whole] + parts:
            c.set_sdf(1, scenes.bucket_sdf(f * DT))
            c.frame(DT, 4, 8)
        wp, wv = _internal(gs, whole)
        lr = whole.read(gs.GS_FIELD_LR_POS), whole.read(gs.GS_FIELD_LR_VEL)
        for k, c in enumerate(parts):
            b, e = ranges[k]
            p, v = _internal(gs, c)
            np.testing.assert_array_equal(p[b:e], wp[b:e], err_msg=f"frame {f} part {k} pos")
            np.testing.assert_array_equal(v[b:e], wv[b:e], err_msg=f"frame {f} part {k} vel")
            np.testing.assert_array_equal(c.read(gs.GS_FIELD_LR_POS), lr[0], err_msg=f"frame {f} part {k} LR")
            np.testing.assert_array_equal(c.read(gs.GS_FIELD_LR_VEL), lr[1], err_msg=f"frame {f} part {k} LR")
    # a final gather-back gives every part the whole state in original order
    pieces = [_internal(gs, c) for c in parts]
    pos = np.concatenate([pieces[k][0][b:e] for k, (b, e) in enumerate(ranges)])
    vel = np.concatenate([pieces[k][1][b:e] for k, (b, e) in enumerate(ranges)])
    for c in parts:
        c.hr_slab_assemble(pos, vel)
        np.testing.assert_array_equal(c.read(gs.GS_FIELD_HR_POS), whole.read(gs.GS_FIELD_HR_POS))
        np.testing.assert_array_equal(c.read(gs.GS_FIELD_HR_VEL), whole.read(gs.GS_FIELD_HR_VEL))
    for c in [whole] + parts:
        c.sync()
        c.close()


def test_device_tensors_assemble_like_host_arrays():
    torch = pytest.importorskip("torch")
    import paper_2308_01629_gb300 as gs
    sc = scenes.cube(n_side=6)
    a, b = gs.Context(sc), gs.Context(sc)
    for c in (a, b):
        c.set_hr_slab(0, 2)
        c.frame(DT, 2, 4)
    pos, vel = _internal(gs, a)
    a.hr_slab_assemble(pos, vel)
    b.hr_slab_assemble(torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda())
    for x, y in zip(_internal(gs, a), _internal(gs, b)):
        np.testing.assert_array_equal(x, y)
    a.close()
    b.close()


def test_partial_state_refuses_what_needs_the_whole_set():
    import paper_2308_01629_gb300 as gs
    sc = scenes.cube(n_side=6)
    c = gs.Context(sc)
    c.set_hr_slab(1, 2)
    c.frame(DT, 2, 4)                                   # frame 0 reorders, then updates slab 1
    hr = np.zeros((c.n_high, 4), np.float32)
    p, n, dev = gs._ptr_of(hr)
    for code in (gs.gs_read(c.ctx, gs.GS_FIELD_HR_POS, p, n, dev), gs.gs_read(c.ctx, gs.GS_FIELD_HR_VEL, p, n, dev),
                 gs.gs_write(c.ctx, gs.GS_FIELD_HR_POS, p, n, dev), gs.gs_resort_high(c.ctx),
                 gs.gs_set_hr_slab(c.ctx, 0, 2), gs.gs_set_pipeline(c.ctx, 1, 8, 1)):
        assert code == gs.GS_ERR_STATE
    pos, vel = _internal(gs, c)                          # internal reads stay open
    for f in range(1, 8):                                # no reorder due: frames run
        c.frame(DT, 2, 4)
    assert gs.gs_frame(c.ctx, DT, 2, 4) == gs.GS_ERR_STATE   # frame 8 would reorder
    pos, vel = _internal(gs, c)
    c.hr_slab_assemble(pos, vel)
    c.frame(DT, 2, 4)
    c.sync()
    c.close()


def test_gather_back_checks_ids_and_values_and_changes_nothing_on_refusal():
    import paper_2308_01629_gb300 as gs
    sc = scenes.cube(n_side=6)
    c = gs.Context(sc)
    c.set_hr_slab(0, 2)
    c.frame(DT, 2, 4)
    pos, vel = _internal(gs, c)
    bad = pos.copy()
    i = int(np.flatnonzero(pos[:, 3].view(np.uint32) != 0xffffffff)[3])
    j = int(np.flatnonzero(pos[:, 3].view(np.uint32) != 0xffffffff)[7])
    bad[[i, j], 3] = bad[[j, i], 3]                      # two ids swapped
    pp, n, dev = gs._ptr_of(bad)
    pv, _, _ = gs._ptr_of(vel)
    assert gs.gs_hr_slab_assemble(c.ctx, pp, pv, n, dev) == gs.GS_ERR_ARG
    nan = pos.copy()
    nan[i, 1] = np.nan
    pp, n, dev = gs._ptr_of(nan)
    assert gs.gs_hr_slab_assemble(c.ctx, pp, pv, n, dev) == gs.GS_ERR_ARG
    assert gs.gs_hr_slab_assemble(c.ctx, pp, pv, n - 16, dev) == gs.GS_ERR_ARG
    for x, y in zip(_internal(gs, c), (pos, vel)):      # untouched, still partial
        np.testing.assert_array_equal(x, y)
    hr = np.zeros((c.n_high, 4), np.float32)
    p, n, dev = gs._ptr_of(hr)
    assert gs.gs_read(c.ctx, gs.GS_FIELD_HR_POS, p, n, dev) == gs.GS_ERR_STATE
    c.hr_slab_assemble(pos, vel)
    c.read(gs.GS_FIELD_HR_POS)
    c.close()


def test_slab_of_the_whole_set_and_empty_slabs():
    """n_parts = 1 is the whole context; more parts than items leave some
    slabs empty, and an empty slab's context changes no HR slot."""
    import paper_2308_01629_gb300 as gs
    sc = scenes.cube(n_side=4)
    whole, one, empty = gs.Context(sc), gs.Context(sc), gs.Context(sc)
    one.set_hr_slab(0, 1)
    n_items = whole.hr_slots // 32
    ranges = [empty.hr_slab_range(k, n_items + 3) for k in range(n_items + 3)]
    k_empty = next(k for k, (b, e) in enumerate(ranges) if b == e)
    empty.set_hr_slab(k_empty, n_items + 3)
    empty.resort_high()
    before = _internal(gs, empty)
    for c in (whole, one, empty):
        c.frame(DT, 2, 4)
    for x, y in zip(_internal(gs, whole), _internal(gs, one)):
        np.testing.assert_array_equal(x, y)
    for x, y in zip(_internal(gs, empty), before):
        np.testing.assert_array_equal(x, y)
    for c in (whole, one, empty):
        c.close()


def test_slabs_of_a_batched_context_equal_the_whole_batch():
    """Slabs are ranges of the warp items of all scenes' HR slots: a batched
    context split in three equals the whole batch bitwise."""
    import paper_2308_01629_gb300 as gs
    sl = scenes.batch(n_scenes=6, lo_count=300, hi_count=1500)
    whole = gs.Context(sl)
    parts = [gs.Context(sl) for _ in range(3)]
    for k, c in enumerate(parts):
        c.set_hr_slab(k, 3)
    ranges = [c.hr_slab_range(k, 3) for k, c in enumerate(parts)]
    for f in range(9):
        if f == 8:   # the reorder of frame 8 needs every slab
            pieces = [_internal(gs, c) for c in parts]
            pos = np.concatenate([pieces[k][0][b:e] for k, (b, e) in enumerate(ranges)])
            vel = np.concatenate([pieces[k][1][b:e] for k, (b, e) in enumerate(ranges)])
            for c in parts:
                c.hr_slab_assemble(pos, vel)
        for c in [whole] + parts:
            c.frame(DT, 4, 8)
    wp, wv = _internal(gs, whole)
    for k, c in enumerate(parts):
        b, e = ranges[k]
        p, v = _internal(gs, c)
        np.testing.assert_array_equal(p[b:e], wp[b:e])
        np.testing.assert_array_equal(v[b:e], wv[b:e])
    for c in [whole] + parts:
        c.close()
