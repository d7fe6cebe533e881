"""The batched pattern: many independent scenes in one context stepped by the
same kernels (one upsampling launch over all scenes, optionally persistent,
optionally replayed as a CUDA graph).  Every scene's result must equal, bit
for bit, the result of the same scene in its own context, and match the
oracle."""
import numpy as np
import pytest

import scenes
from gs_testutil import check_hr, up_prm

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0


def _scenes(n=16, seed=scenes.SEED_BASE + 4):
    return scenes.batch(seed=seed, n_scenes=n, lo_count=300, hi_count=3000)


def _frames(ctx, nframes, n_sub=4, iters=8, use_frame=False):
    for _ in range(nframes):
        if use_frame:
            ctx.frame(DT, n_sub, iters)
        else:
            for _ in range(n_sub):
                ctx.step_low(DT / n_sub, iters)
            ctx.upsample(DT)


def _state(gs, ctx):
    return {k: ctx.read(f) for k, f in (("lr_x", gs.GS_FIELD_LR_POS), ("lr_v", gs.GS_FIELD_LR_VEL),
                                        ("hr_x", gs.GS_FIELD_HR_POS), ("hr_v", gs.GS_FIELD_HR_VEL))}


@pytest.mark.parametrize("shape", [(8, 0), (8, 2), (4, 4), (16, 1)])
def test_batch_equals_separate_contexts_bitwise(shape):
    import paper_2308_01629_gb300 as gs
    sl = _scenes()
    batch = gs.Context(sl)
    batch.set_tuning(*shape)
    _frames(batch, 9)
    got = _state(gs, batch)
    for k, sc in enumerate(sl):
        one = gs.Context(sc)
        _frames(one, 9)
        ref = _state(gs, one)
        one.close()
        for name in ("lr_x", "lr_v"):
            np.testing.assert_array_equal(got[name][batch.scene_slice(k, gs.GS_FIELD_LR_POS)], ref[name])
        for name in ("hr_x", "hr_v"):
            part = got[name][batch.scene_slice(k, gs.GS_FIELD_HR_POS)].copy()
            if name == "hr_x":   # ids are global in the batch, local in the single context
                part[:, 3] = ref[name][:, 3]
            np.testing.assert_array_equal(part, ref[name])
    batch.close()


def test_graph_replay_equals_direct_launches():
    import paper_2308_01629_gb300 as gs
    sl = _scenes(8, seed=scenes.SEED_BASE + 40)
    a = gs.Context(sl)
    b = gs.Context(sl)
    b.set_graphs(True)
    b.set_tuning(8, 2)
    a.set_tuning(8, 2)
    _frames(a, 11, use_frame=True)
    _frames(b, 11, use_frame=True)
    sa, sb = _state(gs, a), _state(gs, b)
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k])
    assert b.launches() > 0
    a.close()
    b.close()


def test_autotune_keeps_state_and_results():
    import paper_2308_01629_gb300 as gs
    sl = _scenes(8, seed=scenes.SEED_BASE + 41)
    a = gs.Context(sl)
    _frames(a, 2)
    before = _state(gs, a)
    w, bps, us = a.autotune(DT, reps=2)
    assert w in (4, 8, 16) and 0 <= bps <= 32 and us > 0
    after = _state(gs, a)
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    b = gs.Context(sl)
    _frames(b, 2)
    _frames(a, 3)
    _frames(b, 3)
    sa, sb = _state(gs, a), _state(gs, b)
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k])
    a.close()
    b.close()


def test_batch_upsample_matches_oracle(orc):
    import paper_2308_01629_gb300 as gs
    sl = [scenes.stir(s, seed=50 + k) for k, s in enumerate(_scenes(6, seed=scenes.SEED_BASE + 42))]
    ctx = gs.Context(sl)
    ctx.set_tuning(8, 2)
    ctx.upsample(DT)
    hx, hv = ctx.read(gs.GS_FIELD_HR_POS), ctx.read(gs.GS_FIELD_HR_VEL)
    for k, sc in enumerate(sl):
        sl_k = ctx.scene_slice(k, gs.GS_FIELD_HR_POS)
        m = len(sc["hr_pos"])
        sub = np.sort(np.random.default_rng(k).choice(m, size=min(m, 3000), replace=False))
        ref = orc.upsample(sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["hr_pos"][:, :3], sc["hr_vel"][:, :3],
                           scenes.sdf_table(sc["sdfs"]), up_prm(sc, DT), sub=sub, mode=1)
        check_hr(sc, DT, hx[sl_k][sub], hv[sl_k][sub], ref)
    ctx.close()


def test_full_size_batch_in_the_benchmark_configuration_matches_oracle(orc):
    """The 256-scene batch the benchmark times (about 19M HR particles) in
    its launch configuration (graph-replayed pipelined frames, persistent
    gather of 8 warps x 4 blocks per SM): one frame without LR steps, so its
    HR frame is the upsampling of the initial state, against the oracle on
    sampled particles of sampled scenes."""
    import paper_2308_01629_gb300 as gs
    sl = [scenes.stir(s, seed=70 + k, spread=0.1) for k, s in enumerate(scenes.batch())]
    ctx = gs.Context(sl)
    ctx.set_graphs(True)
    ctx.set_pipeline(True, 8, 4)
    ctx.frame(DT, 0, 8)
    hx, hv = ctx.read(gs.GS_FIELD_HR_POS), ctx.read(gs.GS_FIELD_HR_VEL)
    assert len(hx) == sum(len(s["hr_pos"]) for s in sl) > 15_000_000
    rng = np.random.default_rng(71)
    for k in sorted(rng.choice(len(sl), size=8, replace=False)):
        sc = sl[k]
        sl_k = ctx.scene_slice(k, gs.GS_FIELD_HR_POS)
        m = len(sc["hr_pos"])
        sub = np.sort(rng.choice(m, size=min(m, 2000), replace=False))
        ref = orc.upsample(sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["hr_pos"][:, :3], sc["hr_vel"][:, :3],
                           scenes.sdf_table(sc["sdfs"]), up_prm(sc, DT), sub=sub, mode=1)
        check_hr(sc, DT, hx[sl_k][sub], hv[sl_k][sub], ref)
    ctx.close()


def _empty_like(sc):
    """The same scene with no particles at all (no LR, hence no HR)."""
    e = dict(sc)
    for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel"):
        e[k] = np.zeros((0, 4), np.float32)
    return e


def test_context_without_particles():
    import paper_2308_01629_gb300 as gs
    ctx = gs.Context(_empty_like(scenes.cube(n_side=4)))
    ctx.set_graphs(True)
    for _ in range(3):
        ctx.frame(DT, 4, 8)
    ctx.step_low(DT, 8)
    ctx.upsample(DT)
    assert ctx.read(gs.GS_FIELD_LR_POS).shape == (0, 4)
    assert ctx.read(gs.GS_FIELD_HR_VEL).shape == (0, 4)
    ctx.sync()
    ctx.close()


@pytest.mark.parametrize("pipelined", [False, True])
def test_batch_with_an_empty_scene_equals_separate_contexts(pipelined):
    """A scene without particles between two others changes nothing for them
    (slot and cell layouts, graph replay, pipelined frames)."""
    import paper_2308_01629_gb300 as gs
    a, b = _scenes(2, seed=scenes.SEED_BASE + 60)
    sl = [a, _empty_like(scenes.cube(n_side=3)), b]
    batch = gs.Context(sl)
    batch.set_graphs(True)
    if pipelined:
        batch.set_pipeline(True, 8, 2)
    _frames(batch, 9, use_frame=True)
    got = _state(gs, batch)
    assert batch.layouts[1].n_low == 0 and batch.layouts[1].n_high == 0
    for k, sc in ((0, a), (2, b)):
        one = gs.Context(sc)
        _frames(one, 9, use_frame=True)
        ref = _state(gs, one)
        one.close()
        for name in ("lr_x", "lr_v"):
            np.testing.assert_array_equal(got[name][batch.scene_slice(k, gs.GS_FIELD_LR_POS)], ref[name])
        for name in ("hr_x", "hr_v"):
            part = got[name][batch.scene_slice(k, gs.GS_FIELD_HR_POS)].copy()
            if name == "hr_x":
                part[:, 3] = ref[name][:, 3]
            np.testing.assert_array_equal(part, ref[name])
    batch.close()
