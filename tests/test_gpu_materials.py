"""Grain materials: per-particle friction coefficients with the cross
coefficients mu_ij = sqrt(mu_i mu_j) of Sec. 3 (static and kinetic alike;
sqrt(mu_i mu_b) against an SDF boundary).  The GPU LR step with a material
table is compared with the FP64 oracle given the same per-particle
coefficients, and checked bit for bit against the paths that must agree with
it (one material equal to the scene's coefficients, graph replay, the
persistent solver, a batch against separate contexts)."""
import numpy as np
import pytest

import scenes
from gs_testutil import ATOL_L, RTOL, box_size, within
from test_gpu_step_low import CASES, pb_prm

pytestmark = pytest.mark.gpu


def _ctx(gs, sc, table, ids, **kw):
    ctx = gs.Context(sc, **kw)
    ctx.set_materials(table, ids)
    return ctx


def _lr(gs, ctx):
    x = ctx.read(gs.GS_FIELD_LR_POS)
    v = ctx.read(gs.GS_FIELD_LR_VEL)
    ctx.sync()
    return x, v


def _oracle_step(orc, sc, dt, n_stab, iters, table, ids):
    mu = np.asarray(table, np.float64)[ids]
    return orc.pbd_step(sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["lr_pos"][:, 3],
                        scenes.sdf_table(sc["sdfs"]), pb_prm(sc, dt, n_stab, iters), mode=1, mu=mu)


def _elementwise(sc, dt, x, v, rx, rv, mask):
    L = box_size(sc)
    okx = within(x[:, :3], rx, RTOL, ATOL_L * L)
    okv = within(v[:, :3], rv, RTOL, ATOL_L * L / dt)
    bad = np.nonzero(mask & ~(okx & okv))[0]
    assert len(bad) == 0, (f"{len(bad)} of {mask.sum()} LR particles outside tolerance; first {bad[0]}: "
                           f"gpu {x[bad[0], :3]} {v[bad[0], :3]} ref {rx[bad[0]]} {rv[bad[0]]}")


@pytest.mark.parametrize("case", ["cube_stir", "funnel", "digging_bucket"])
@pytest.mark.parametrize("dt", [1.0 / 60.0, 1.0 / 240.0])
def test_friction_pass_with_materials_matches_oracle(orc, case, dt):
    """One contact + friction pass (no stabilization) with every particle of
    a random material out of three."""
    import paper_2308_01629_gb300 as gs
    sc = CASES[case]()
    table, ids = scenes.materials(sc, seed=scenes.SEED_BASE + 60)
    ctx = _ctx(gs, sc, table, ids, n_stab=0)
    ctx.step_low(dt, 1)
    x, v = _lr(gs, ctx)
    ctx.close()
    rx, rv, sus, st = _oracle_step(orc, sc, dt, 0, 1, table, ids)
    assert st["active"] > 0 and sus.mean() < 0.01, st
    _elementwise(sc, dt, x, v, rx, rv, ~sus)


@pytest.mark.parametrize("seed", range(3))
def test_full_step_with_materials_matches_oracle(orc, seed):
    import paper_2308_01629_gb300 as gs
    sc = scenes.stir(scenes.cube(seed=scenes.SEED_BASE + 210 + seed), seed=seed, v_scale=0.3)
    table, ids = scenes.materials(sc, seed=scenes.SEED_BASE + 61 + seed)
    dt = 1.0 / 240.0
    ctx = _ctx(gs, sc, table, ids, n_stab=2)
    ctx.step_low(dt, sc["iters"])
    x, v = _lr(gs, ctx)
    ctx.close()
    rx, rv, sus, st = _oracle_step(orc, sc, dt, 2, sc["iters"], table, ids)
    _elementwise(sc, dt, x, v, rx, rv, ~sus)
    dx = np.linalg.norm(x[:, :3] - rx, axis=1)
    assert np.quantile(dx, 0.99) < 0.05 * sc["r_low"] and dx.max() < sc["r_low"]


def test_materials_change_the_result():
    """The table reaches the pass: a smooth material changes the step against
    the scene's coefficients and against a rough material.  (A rough
    material alone need not: where every contact is static under both sets of
    coefficients, static friction cancels the slide whatever the threshold.)"""
    import paper_2308_01629_gb300 as gs
    sc = CASES["cube_stir"]()
    out = []
    for table in (None, [[0.8, 0.6]], [[0.1, 0.05]]):
        ctx = gs.Context(sc)
        if table is not None:
            ctx.set_materials(table)
        ctx.step_low(1.0 / 60.0, sc["iters"])
        out.append(_lr(gs, ctx)[1])
        ctx.close()
    assert not np.array_equal(out[0], out[2]) and not np.array_equal(out[1], out[2])


def test_one_material_with_the_scene_coefficients_is_bitwise_the_plain_step():
    """sqrt(mu mu) = mu exactly, so a single material carrying the scene's
    (mu_s, mu_k) reproduces the step without materials bit for bit."""
    import paper_2308_01629_gb300 as gs
    sc = CASES["digging_bucket"]()
    out = []
    for with_table in (False, True):
        ctx = gs.Context(sc)
        if with_table:
            ctx.set_materials([[sc["mu_s"], sc["mu_k"]]], np.zeros(len(sc["lr_pos"]), np.uint32))
        for _ in range(3):
            ctx.step_low(1.0 / 240.0, sc["iters"])
        out.append(_lr(gs, ctx))
        ctx.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_materials_with_graphs_solver_and_pipelining_agree_bitwise():
    """Per-pass launches, graph-replayed frames, the persistent solver and
    pipelined frames give the same bits with a material table."""
    import paper_2308_01629_gb300 as gs
    sc = scenes.stir(scenes.cube(), seed=5, v_scale=0.3)
    table, ids = scenes.materials(sc, seed=scenes.SEED_BASE + 62, layout="layers")
    ref = None
    for mode in ("plain", "graphs", "solver", "pipelined"):
        ctx = _ctx(gs, sc, table, ids)
        ctx.set_graphs(mode in ("graphs", "pipelined"))
        if mode == "solver":
            try:
                ctx.set_lr_solver(True)
            except gs.GsError:
                ctx.close()
                continue
        if mode == "pipelined":
            ctx.set_pipeline(True, 8, 1)
        for _ in range(4):
            ctx.frame(1.0 / 60.0, 4, sc["iters"])
        got = (*_lr(gs, ctx), ctx.read(gs.GS_FIELD_HR_POS), ctx.read(gs.GS_FIELD_HR_VEL))
        ctx.sync()
        ctx.close()
        if ref is None:
            ref = got
            continue
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b, err_msg=mode)


def test_batch_with_materials_equals_separate_contexts():
    import paper_2308_01629_gb300 as gs
    sl = scenes.batch(seed=scenes.SEED_BASE + 63, n_scenes=6, lo_count=300, hi_count=2000)
    table = scenes.MATERIALS
    ids = [scenes.materials(sc, seed=scenes.SEED_BASE + 64 + k)[1] for k, sc in enumerate(sl)]
    batch = _ctx(gs, sl, table, np.concatenate(ids))
    for _ in range(3):
        batch.frame(1.0 / 60.0, 4, 4)
    bx, bv = _lr(gs, batch)
    for k, sc in enumerate(sl):
        one = _ctx(gs, sc, table, ids[k])
        for _ in range(3):
            one.frame(1.0 / 60.0, 4, 4)
        x, v = _lr(gs, one)
        one.close()
        s = batch.scene_slice(k, gs.GS_FIELD_LR_POS)
        np.testing.assert_array_equal(bx[s], x)
        np.testing.assert_array_equal(bv[s], v)
    batch.close()


def test_material_field_and_table_errors():
    import paper_2308_01629_gb300 as gs
    sc = scenes.cube(n_side=6)
    n = len(sc["lr_pos"])
    ctx = gs.Context(sc)
    ids = (np.arange(n) % 3).astype(np.uint32)
    with pytest.raises(gs.GsError) as e:   # no table yet
        ctx.write(gs.GS_FIELD_LR_MATERIAL, ids)
    assert e.value.code == gs.GS_ERR_STATE
    for bad in (np.zeros((gs.GS_MAX_MATERIALS + 1, 2)), [[0.3, -0.1]], [[np.nan, 0.2]]):
        with pytest.raises(gs.GsError) as e:
            ctx.set_materials(bad)
        assert e.value.code == gs.GS_ERR_ARG
    ctx.set_materials(scenes.MATERIALS, ids)
    np.testing.assert_array_equal(ctx.read(gs.GS_FIELD_LR_MATERIAL), ids)
    with pytest.raises(gs.GsError) as e:   # id 3 with three materials: refused, field unchanged
        ctx.write(gs.GS_FIELD_LR_MATERIAL, np.full(n, 3, np.uint32))
    assert e.value.code == gs.GS_ERR_ARG
    np.testing.assert_array_equal(ctx.read(gs.GS_FIELD_LR_MATERIAL), ids)
    with pytest.raises(gs.GsError) as e:   # a smaller table would orphan id 2
        ctx.set_materials(scenes.MATERIALS[:2])
    assert e.value.code == gs.GS_ERR_ARG
    ctx.step_low(1.0 / 240.0, 2)   # the context stays usable
    ctx.set_materials([])          # off: ids back to 0
    np.testing.assert_array_equal(ctx.read(gs.GS_FIELD_LR_MATERIAL), 0)
    ctx.set_materials(scenes.MATERIALS[:1])
    ctx.sync()
    ctx.close()


def test_step_reverse_mode_refuses_materials():
    import torch

    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300 import diff
    sc = scenes.cube(n_side=6)
    ctx = gs.Context(sc, stream="torch")
    ctx.set_materials(scenes.MATERIALS[:1])
    x = torch.tensor(sc["lr_pos"], device="cuda", requires_grad=True)
    v = torch.tensor(sc["lr_vel"], device="cuda", requires_grad=True)
    ox, ov = diff.StepLowFn.apply(ctx, 1.0 / 240.0, 2, x, v)
    with pytest.raises(gs.GsError) as e:
        (ox[:, :3].sum() + ov[:, :3].sum()).backward()
    assert e.value.code == gs.GS_ERR_STATE
    ctx.close()
