"""Rigid bodies by shape matching (Sec. 3): body particles collide like
grains and are matched to their rest shape in every solver pass (R xo + c,
R from the polar decomposition of C = sum m (x~ - c) xo^T), counted once in
the Jacobi average.  GPU against the FP64 oracle, the bitwise agreements
that must hold, and a boulder hurled into the digging bed."""
import numpy as np
import pytest

import scenes
from gs_testutil import ATOL_L, RTOL, box_size, within
from test_gpu_step_low import pb_prm

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0


def _lr(gs, ctx):
    x, v = ctx.read(gs.GS_FIELD_LR_POS), ctx.read(gs.GS_FIELD_LR_VEL)
    ctx.sync()
    return x, v


def _oracle(orc, sc, dt, n_stab, iters):
    body = sc["lr_body"].astype(np.int32)
    xo = orc.body_rest_offsets(sc["lr_pos"][:, :3], sc["lr_pos"][:, 3], body)
    return orc.pbd_step(sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["lr_pos"][:, 3], scenes.sdf_table(sc["sdfs"]),
                        pb_prm(sc, dt, n_stab, iters), mode=1, bodies=(body, xo))


def _pairwise(x):
    return np.linalg.norm(x[:, None, :3] - x[None, :, :3], axis=2)


@pytest.mark.parametrize("dt", [1.0 / 60.0, 1.0 / 240.0])
@pytest.mark.parametrize("seed", [0, 1])
def test_solver_pass_with_a_body_matches_oracle(orc, dt, seed):
    import paper_2308_01629_gb300 as gs
    sc = scenes.cube_with_block(seed=scenes.SEED_BASE + 100 + seed)
    ctx = gs.Context(sc, n_stab=0)
    ctx.step_low(dt, 1)
    x, v = _lr(gs, ctx)
    ctx.close()
    rx, rv, sus, st = _oracle(orc, sc, dt, 0, 1)
    assert st["active"] > 0 and sus.mean() < 0.02, st
    L = box_size(sc)
    ok = within(x[:, :3], rx, RTOL, ATOL_L * L) & within(v[:, :3], rv, RTOL, ATOL_L * L / dt)
    bad = np.nonzero(~sus & ~ok)[0]
    assert len(bad) == 0, f"{len(bad)} outside tolerance; first {bad[0]}: {x[bad[0]]} {rx[bad[0]]}"


def test_full_step_with_a_body_matches_oracle_statistically(orc):
    import paper_2308_01629_gb300 as gs
    sc = scenes.cube_with_block()
    dt = 1.0 / 240.0
    ctx = gs.Context(sc)
    ctx.step_low(dt, sc["iters"])
    x, v = _lr(gs, ctx)
    ctx.close()
    rx, rv, sus, st = _oracle(orc, sc, dt, 2, sc["iters"])
    dx = np.linalg.norm(x[:, :3] - rx, axis=1)
    assert np.quantile(dx, 0.99) < 0.05 * sc["r_low"] and dx.max() < 2 * sc["r_low"]
    for a, b in ((x[:, :3], rx), (v[:, :3], rv)):
        np.testing.assert_allclose(a.mean(0), b.mean(0), rtol=1e-3, atol=1e-3 * np.abs(b).mean() + 1e-9)


def test_block_keeps_its_shape_as_the_method_does(orc):
    """The shape-matching delta is averaged with the contact deltas (1 / n_i),
    so a body under load is only nearly rigid; its shape error after ten
    frames must be that of the method (the oracle's)."""
    import paper_2308_01629_gb300 as gs
    sc = scenes.cube_with_block()
    sel = sc["lr_body"] == 1
    ctx = gs.Context(sc)
    ctx.set_graphs(True)
    for _ in range(10):
        ctx.frame(DT, 4, sc["iters"])
    x, _ = _lr(gs, ctx)
    ctx.close()
    body = sc["lr_body"].astype(np.int32)
    xo = orc.body_rest_offsets(sc["lr_pos"][:, :3], sc["lr_pos"][:, 3], body)
    rx, rv = sc["lr_pos"][:, :3].astype(float), sc["lr_vel"][:, :3].astype(float)
    for _ in range(40):
        rx, rv, _, _ = orc.pbd_step(rx, rv, sc["lr_pos"][:, 3], scenes.sdf_table(sc["sdfs"]),
                                    pb_prm(sc, DT / 4, 2, sc["iters"]), mode=1, bodies=(body, xo))
    d0 = _pairwise(sc["lr_pos"][sel])
    err_gpu = np.abs(_pairwise(x[sel]) - d0).max()
    err_ref = np.abs(_pairwise(rx[sel]) - d0).max()
    assert err_gpu < 2.0 * err_ref + 0.01 * sc["r_low"] and err_gpu < 0.5 * sc["r_low"], (err_gpu, err_ref)


def test_frames_with_bodies_agree_bitwise_across_launch_modes_and_batches():
    import paper_2308_01629_gb300 as gs
    sa = scenes.cube_with_block(seed=scenes.SEED_BASE + 110)
    sb = scenes.cube_with_block(seed=scenes.SEED_BASE + 111)
    out = {}
    for mode in ("direct", "graphs", "solver"):
        ctx = gs.Context(sa)
        ctx.set_graphs(mode != "direct")
        if mode == "solver":   # bodies run per-pass launches whatever the solver setting
            try:
                ctx.set_lr_solver(True)
            except gs.GsError:
                ctx.close()
                continue
        for _ in range(4):
            ctx.frame(DT, 4, sa["iters"])
        out[mode] = (*_lr(gs, ctx), ctx.read(gs.GS_FIELD_HR_POS))
        ctx.close()
    for mode in out:
        for a, b in zip(out[mode], out["direct"]):
            np.testing.assert_array_equal(a, b, err_msg=mode)
    batch = gs.Context([sa, sb])
    np.testing.assert_array_equal(batch.read(gs.GS_FIELD_LR_BODY)[len(sa["lr_pos"]):][sb["lr_body"] > 0], 2)
    for _ in range(4):
        batch.frame(DT, 4, sa["iters"])
    bx, bv = _lr(gs, batch)
    one = gs.Context(sb)
    for _ in range(4):
        one.frame(DT, 4, sb["iters"])
    x, v = _lr(gs, one)
    one.close()
    s0, s1 = batch.scene_slice(0, gs.GS_FIELD_LR_POS), batch.scene_slice(1, gs.GS_FIELD_LR_POS)
    np.testing.assert_array_equal(bx[s0], out["direct"][0])
    np.testing.assert_array_equal(bx[s1], x)
    np.testing.assert_array_equal(bv[s1], v)
    batch.close()


def test_boulder_hurled_into_the_bed():
    """Two-way coupling: the boulder stays rigid, the sand slows it down and
    is set in motion around the impact."""
    import paper_2308_01629_gb300 as gs
    sc = scenes.digging_with_boulder()
    sel = sc["lr_body"] == 1
    ctx = gs.Context(sc)
    ctx.set_graphs(True)
    for _ in range(12):
        ctx.frame(DT, 4, sc["iters"])
    x, v = _lr(gs, ctx)
    ctx.close()
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(v))
    d0, d1 = _pairwise(sc["lr_pos"][sel]), _pairwise(x[sel])
    assert np.abs(d1 - d0).max() < 0.5 * sc["r_low"]   # nearly rigid (see the test above)
    z0, z1 = sc["lr_pos"][sel, 2].mean(), x[sel, 2].mean()
    assert z1 < z0 - 0.05   # it fell
    speed = np.linalg.norm(v[sel, :3].mean(0))
    assert speed < 2.0 + 9.81 * 12 * DT - 0.5   # slower than free fall from 2 m/s
    grains = ~sel
    assert np.linalg.norm(v[grains, :3], axis=1).max() > 0.2   # sand set in motion


def test_body_field_errors_and_reverse_mode_refusal():
    import torch

    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300 import diff
    sc = scenes.cube(n_side=6)
    n = len(sc["lr_pos"])
    ctx = gs.Context(sc, stream="torch")
    with pytest.raises(gs.GsError) as e:
        ctx.write(gs.GS_FIELD_LR_BODY, np.full(n, gs.GS_MAX_BODIES + 1, np.uint32))
    assert e.value.code == gs.GS_ERR_ARG
    ids = np.zeros(n, np.uint32)
    ids[:27] = 1
    ctx.write(gs.GS_FIELD_LR_BODY, ids)
    np.testing.assert_array_equal(ctx.read(gs.GS_FIELD_LR_BODY), ids)
    x = torch.tensor(sc["lr_pos"], device="cuda", requires_grad=True)
    v = torch.tensor(sc["lr_vel"], device="cuda", requires_grad=True)
    ox, ov = diff.StepLowFn.apply(ctx, 1.0 / 240.0, 2, x, v)
    with pytest.raises(gs.GsError) as e:
        (ox[:, :3].sum() + ov[:, :3].sum()).backward()
    assert e.value.code == gs.GS_ERR_STATE
    ctx.write(gs.GS_FIELD_LR_BODY, np.zeros(n, np.uint32))   # no bodies: the reverse mode runs again
    ox, ov = diff.StepLowFn.apply(ctx, 1.0 / 240.0, 2, x, v)
    (ox[:, :3].sum() + ov[:, :3].sum()).backward()
    ctx.sync()
    # a body particle of infinite mass is refused
    pos = sc["lr_pos"].copy()
    pos[0, 3] = 0.0
    ctx.write(gs.GS_FIELD_LR_POS, pos)
    ids = np.zeros(n, np.uint32)
    ids[:4] = 1
    with pytest.raises(gs.GsError) as e:
        ctx.write(gs.GS_FIELD_LR_BODY, ids)
    assert e.value.code == gs.GS_ERR_ARG
    ctx.close()
