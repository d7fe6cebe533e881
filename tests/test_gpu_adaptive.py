"""CFL-limited LR substeps (gs_frame_adaptive; Sec. 5.2: a default LR time
step shortened by the CFL condition, one HR frame over several LR steps).

The device-side loop (a conditional while node in the frame's CUDA graph)
must give the same bits as the host-driven loop and as explicit LR steps of
the lengths it reports; every reported length must be the oracle's float32
decision for the GPU's own velocities at that point; free fall and the step
cap are checked in closed form."""
import numpy as np
import pytest

import scenes
from test_gpu_step_low import CASES

pytestmark = pytest.mark.gpu
T = np.float32(1.0 / 60.0)


def _state(gs, ctx):
    out = tuple(ctx.read(f) for f in (gs.GS_FIELD_LR_POS, gs.GS_FIELD_LR_VEL, gs.GS_FIELD_HR_POS, gs.GS_FIELD_HR_VEL))
    ctx.sync()
    return out


def _free_grains(n_side=4, r=0.01, v=(0.0, 0.0, -3.0), g=(0.0, 0.0, -9.81)):
    """Grains far apart in mid-air (no contacts during a frame)."""
    sc = scenes.cube(n_side=n_side, r_low=r)
    sc = dict(sc)
    lr = sc["lr_pos"].copy()
    c = lr[:, :3].mean(0)
    lr[:, :3] = c + (lr[:, :3] - c) * 4.0 + np.array([0.0, 0.0, 0.1], np.float32)
    hr = sc["hr_pos"].copy()
    hr[:, :3] = np.repeat(lr[:, :3], sc["ratio"], axis=0) + (hr[:, :3] - np.repeat(sc["lr_pos"][:, :3], sc["ratio"],
                                                                                       axis=0))
    vel = np.zeros_like(sc["lr_vel"])
    vel[:, :3] = v
    sc.update(lr_pos=lr, hr_pos=hr, lr_vel=vel, gravity=g)
    return sc


@pytest.mark.parametrize("case", ["cube_stir", "funnel"])
def test_device_loop_equals_host_loop_and_explicit_steps(case):
    import paper_2308_01629_gb300 as gs
    sc = CASES[case]()
    iters = sc["iters"]
    got = {}
    for mode in ("graph", "host"):
        ctx = gs.Context(sc)
        ctx.set_graphs(mode == "graph")
        for _ in range(3):
            ctx.frame_adaptive(T, iters)
        dts = ctx.substeps()
        got[mode] = (_state(gs, ctx), dts)
        ctx.close()
    np.testing.assert_array_equal(got["graph"][1], got["host"][1])
    for a, b in zip(got["graph"][0], got["host"][0]):
        np.testing.assert_array_equal(a, b)
    # the third frame again as explicit steps of the reported lengths
    ctx = gs.Context(sc)
    for _ in range(2):
        ctx.frame_adaptive(T, iters)
    for dt in got["graph"][1]:
        ctx.step_low(float(dt), iters)
    ctx.upsample(float(T))
    ref = _state(gs, ctx)
    ctx.close()
    for a, b in zip(got["graph"][0], ref):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("case,vscale", [("cube_stir", 1.0), ("funnel", 1.0), ("cube_stir", 6.0)])
def test_reported_steps_are_the_oracle_decisions(orc, case, vscale):
    """Replay the frame step by step and re-decide every length with the
    oracle's float32 rule from the velocities the GPU holds at that point."""
    import paper_2308_01629_gb300 as gs
    sc = dict(CASES[case]())
    sc["lr_vel"] = sc["lr_vel"] * np.float32(vscale)
    ctx = gs.Context(sc)
    ctx.set_graphs(True)
    ctx.frame_adaptive(T, sc["iters"])
    dts = ctx.substeps()
    ctx.close()
    assert len(dts) >= 4
    ctx = gs.Context(sc)
    r = np.float32(sc["r_low"])
    t_rem = T
    for k, dt in enumerate(dts):
        v = ctx.read(gs.GS_FIELD_LR_VEL)
        want, more = orc.cfl_substep(t_rem, orc.cfl_rate(v, r), 0.005, 0.4, 64 - k)
        assert want == dt, (k, want, dt)
        assert more == (k + 1 < len(dts))
        ctx.step_low(float(dt), sc["iters"])
        t_rem = np.float32(t_rem - dt)
    ctx.close()


def test_slow_frame_takes_four_default_steps():
    import paper_2308_01629_gb300 as gs
    sc = scenes.cube()   # at rest
    ctx = gs.Context(sc)
    ctx.set_graphs(True)
    ctx.frame_adaptive(T, sc["iters"])
    dts = ctx.substeps()
    ctx.close()
    assert len(dts) == 4
    np.testing.assert_allclose(dts, 1.0 / 240.0, rtol=1e-6)


def test_free_fall_matches_the_oracle_and_the_closed_form(orc):
    """No contacts: v = v0 + g (sum of steps), the steps as the oracle's."""
    import paper_2308_01629_gb300 as gs
    sc = _free_grains(r=0.005)
    ctx = gs.Context(sc)
    ctx.set_graphs(True)
    ctx.frame_adaptive(T, 4)
    dts = ctx.substeps()
    x, v = ctx.read(gs.GS_FIELD_LR_POS), ctx.read(gs.GS_FIELD_LR_VEL)
    ctx.sync()
    ctx.close()
    from gs_testutil import pb_prm
    prm = pb_prm(sc, T, 2, 4)
    rx, rv, rdts = orc.frame_adaptive(sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["lr_pos"][:, 3],
                                      scenes.sdf_table(sc["sdfs"]), prm, T, 0.005, 0.4, 64)
    np.testing.assert_array_equal(dts, rdts)
    s = dts.astype(float).sum()
    assert abs(s - float(T)) <= len(dts) * float(np.spacing(T))
    np.testing.assert_allclose(v[:, 2], -3.0 - 9.81 * s, rtol=1e-5)
    np.testing.assert_allclose(v[:, :3], rv, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(x[:, :3], rx, rtol=1e-6, atol=1e-6)


def test_step_count_is_capped():
    import paper_2308_01629_gb300 as gs
    # 10 m/s with r = 0.005: limit 0.0004 s, 42 steps wanted; the grains stay
    # clear of the walls during the frame
    sc = _free_grains(r=0.005, v=(10.0, 0.0, 0.0), g=(0.0, 0.0, 0.0))
    for graphs in (True, False):
        ctx = gs.Context(sc)
        ctx.set_graphs(graphs)
        ctx.frame_adaptive(T, 2, max_sub=16)
        dts = ctx.substeps()
        ctx.close()
        assert len(dts) == 16
        assert abs(dts.astype(float).sum() - float(T)) <= 16 * float(np.spacing(T))


def test_batch_rate_uses_each_scenes_radius(orc):
    import paper_2308_01629_gb300 as gs
    sl = scenes.batch(seed=scenes.SEED_BASE + 70, n_scenes=5, lo_count=300, hi_count=2000)
    sl = [scenes.stir(sc, seed=k, v_scale=0.4) for k, sc in enumerate(sl)]
    ctx = gs.Context(sl)
    ctx.set_graphs(True)
    ctx.frame_adaptive(T, 4)
    dts = ctx.substeps()
    ctx.close()
    r = np.concatenate([np.full(len(sc["lr_pos"]), sc["r_low"], np.float32) for sc in sl])
    v = np.concatenate([sc["lr_vel"] for sc in sl])
    want, _ = orc.cfl_substep(T, orc.cfl_rate(v, r), 0.005, 0.4, 64)
    assert dts[0] == want


def test_launch_count_includes_the_device_loop():
    import paper_2308_01629_gb300 as gs
    sc = CASES["cube_stir"]()
    counts = {}
    for graphs in (False, True):
        ctx = gs.Context(sc)
        ctx.set_graphs(graphs)
        ctx.frame_adaptive(T, 4)   # the first graph frame is captured, not counted twice
        ctx.sync()
        l0 = ctx.launches()
        ctx.frame_adaptive(T, 4)
        ctx.sync()
        counts[graphs] = (ctx.launches() - l0, len(ctx.substeps()))
        ctx.close()
    assert counts[True] == counts[False]


def test_invalid_arguments_are_refused():
    import paper_2308_01629_gb300 as gs
    ctx = gs.Context(scenes.cube(n_side=4))
    for kw in (dict(dt=0.0), dict(dt_max=-1.0), dict(cfl=float("nan")), dict(max_sub=0),
               dict(max_sub=gs.GS_MAX_SUBSTEPS + 1)):
        args = dict(dt=T, dt_max=0.005, cfl=0.4, max_sub=64)
        args.update(kw)
        with pytest.raises(gs.GsError) as e:
            ctx.frame_adaptive(args["dt"], 4, dt_max=args["dt_max"], cfl=args["cfl"], max_sub=args["max_sub"])
        assert e.value.code == gs.GS_ERR_ARG
    ctx.frame_adaptive(T, 4)
    ctx.sync()
    ctx.close()
