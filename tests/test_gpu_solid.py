"""Particle-sampled boundaries and rigid bodies (Sec. 3: LR particles of
inverse mass 0 under the same contact constraints; Sec. 4: they count in the
HR weights except where no grain reaches the HR particle).  GPU against the
FP64 oracle on a cube standing on a particle floor and on the digging bed
with a particle bucket, plus the bitwise agreements that must hold."""
import numpy as np
import pytest

import scenes
from gs_testutil import ATOL_L, RTOL, box_size, check_hr, up_prm, within
from test_gpu_step_low import pb_prm

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0

SCENES = {"cube_floor": scenes.cube_on_particle_floor, "digging_bucket": scenes.digging_particle_bucket}


def _lr(gs, ctx):
    x, v = ctx.read(gs.GS_FIELD_LR_POS), ctx.read(gs.GS_FIELD_LR_VEL)
    ctx.sync()
    return x, v


def _elementwise(sc, dt, x, v, rx, rv, mask):
    L = box_size(sc)
    ok = within(x[:, :3], rx, RTOL, ATOL_L * L) & within(v[:, :3], rv, RTOL, ATOL_L * L / dt)
    bad = np.nonzero(mask & ~ok)[0]
    assert len(bad) == 0, f"{len(bad)} of {mask.sum()} outside tolerance; first {bad[0]}: {x[bad[0]]} {rx[bad[0]]}"


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("passes", [(0, 1), (1, 0), (2, 8)])
def test_lr_step_with_solid_particles_matches_oracle(orc, name, passes):
    import paper_2308_01629_gb300 as gs
    sc = SCENES[name]()
    dt = 1.0 / 240.0
    ctx = gs.Context(sc, n_stab=passes[0])
    ctx.step_low(dt, passes[1])
    x, v = _lr(gs, ctx)
    ctx.close()
    rx, rv, sus, st = orc.pbd_step(sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["lr_pos"][:, 3],
                                   scenes.sdf_table(sc["sdfs"]), pb_prm(sc, dt, *passes), mode=1)
    full = passes[0] + passes[1] > 1
    # a single pass: marks are rare.  A whole step of a resting pile: resolved
    # contacts sit at exactly 2 r_LR, so marks spread to (nearly) every grain
    # and the comparison is statistical, as for the steps without solids
    assert st["active"] > 0 and (full or sus.mean() < 0.02), st
    _elementwise(sc, dt, x, v, rx, rv, ~sus)
    if full:
        dx = np.linalg.norm(x[:, :3] - rx, axis=1)
        assert np.quantile(dx, 0.99) < 0.05 * sc["r_low"] and dx.max() < 2 * sc["r_low"]
        for a, b in ((x[:, :3], rx), (v[:, :3], rv)):
            np.testing.assert_allclose(a.mean(0), b.mean(0), rtol=1e-3, atol=1e-3 * np.abs(b).mean() + 1e-9)
            np.testing.assert_allclose(a.std(0), b.std(0), rtol=1e-2, atol=1e-9)
    solid = sc["lr_pos"][:, 3] == 0
    # solid particles move with their prescribed velocity and keep w = 0
    np.testing.assert_array_equal(x[solid, 3], 0.0)
    np.testing.assert_allclose(x[solid, :3], sc["lr_pos"][solid, :3] + dt * sc["lr_vel"][solid, :3], rtol=0,
                               atol=1e-6)
    if name == "cube_floor":   # a floor at rest does not move at all
        np.testing.assert_array_equal(x[solid], sc["lr_pos"][solid])
        np.testing.assert_array_equal(v[solid], 0.0)


def _ref_up(orc, sc, sub=None):
    return orc.upsample(sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["hr_pos"][:, :3], sc["hr_vel"][:, :3],
                        scenes.sdf_table(sc["sdfs"]), up_prm(sc, DT), sub=sub, mode=1,
                        solid=sc["lr_pos"][:, 3] == 0)


def _beside_the_floor(sc, n=64):
    """HR particles moved next to floor particles at the floor's rim, beyond
    every grain's reach (the rule's case)."""
    sc = dict(sc)
    hr = sc["hr_pos"].copy()
    solid = sc["lr_pos"][sc["lr_pos"][:, 3] == 0, :3]
    grains = sc["lr_pos"][sc["lr_pos"][:, 3] > 0, :3]
    far = solid[np.linalg.norm(solid[:, None, :2] - grains[None, :, :2], axis=2).min(1) > 3.5 * sc["r_low"]]
    assert len(far) >= n
    hr[:n, :3] = far[:n] + np.array([0.0, 0.0, 0.5 * sc["r_low"]], np.float32)
    sc["hr_pos"] = hr
    return sc


def test_gather_with_solid_particles_matches_oracle(orc):
    import paper_2308_01629_gb300 as gs
    sc = _beside_the_floor(scenes.cube_on_particle_floor())
    ctx = gs.Context(sc)
    ctx.upsample(DT)
    x, v = ctx.read(gs.GS_FIELD_HR_POS), ctx.read(gs.GS_FIELD_HR_VEL)
    ctx.sync()
    ctx.close()
    ref = _ref_up(orc, sc)
    check_hr(sc, DT, x, v, ref)
    # beside the floor with no grain in reach: ballistic (the rule)
    g = np.array(sc["gravity"], np.float32)
    want_v = sc["hr_vel"][:64, :3] + np.float32(DT) * g
    np.testing.assert_allclose(v[:64, :3], want_v, rtol=1e-6, atol=1e-7)
    assert np.all(ref["diag"][:64, 0] == 0.0)


def test_gather_with_a_particle_bucket_sampled(orc):
    import paper_2308_01629_gb300 as gs
    sc = scenes.stir(scenes.digging_particle_bucket(), seed=9, spread=0.2)
    ctx = gs.Context(sc)
    ctx.upsample(DT)
    x, v = ctx.read(gs.GS_FIELD_HR_POS), ctx.read(gs.GS_FIELD_HR_VEL)
    ctx.sync()
    ctx.close()
    sub = np.sort(np.random.default_rng(10).choice(len(sc["hr_pos"]), size=20000, replace=False))
    check_hr(sc, DT, x[sub], v[sub], _ref_up(orc, sc, sub=sub))


def test_frames_with_solid_particles_graphs_and_batch_agree_bitwise():
    import paper_2308_01629_gb300 as gs
    sc = scenes.cube_on_particle_floor()
    out = {}
    for graphs in (False, True):
        ctx = gs.Context(sc)
        ctx.set_graphs(graphs)
        for _ in range(5):
            ctx.frame(DT, 4, sc["iters"])
        out[graphs] = (*_lr(gs, ctx), ctx.read(gs.GS_FIELD_HR_POS), ctx.read(gs.GS_FIELD_HR_VEL))
        ctx.close()
    for a, b in zip(out[False], out[True]):
        np.testing.assert_array_equal(a, b)
    sl = [sc, scenes.stir(scenes.cube(seed=scenes.SEED_BASE + 90), seed=3)]
    batch = gs.Context(sl)
    for _ in range(5):
        batch.frame(DT, 4, sc["iters"])
    bx, bv = _lr(gs, batch)
    s = batch.scene_slice(0, gs.GS_FIELD_LR_POS)
    np.testing.assert_array_equal(bx[s], out[False][0])
    np.testing.assert_array_equal(bv[s], out[False][1])
    batch.close()


def test_particle_bucket_keeps_its_velocity():
    import paper_2308_01629_gb300 as gs
    sc = scenes.digging_particle_bucket()
    solid = sc["lr_pos"][:, 3] == 0
    ctx = gs.Context(sc)
    ctx.set_graphs(True)
    for _ in range(6):
        ctx.frame(DT, 4, sc["iters"])
    x, v = _lr(gs, ctx)
    ctx.close()
    u = sc["lr_vel"][solid, :3]
    # v = ((x + dt v) - x) / dt each step: float32 rounding of about 1e-5 m/s
    np.testing.assert_allclose(v[solid, :3], u, rtol=0, atol=2e-4)
    np.testing.assert_allclose(x[solid, :3], sc["lr_pos"][solid, :3] + 6 * DT * u, rtol=0, atol=1e-5)


def test_reverse_modes_refuse_solid_particles():
    import torch

    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300 import diff
    sc = scenes.cube_on_particle_floor()
    ctx = gs.Context(sc, stream="torch")
    x = torch.tensor(sc["lr_pos"], device="cuda", requires_grad=True)
    v = torch.tensor(sc["lr_vel"], device="cuda", requires_grad=True)
    # the refusal is a device-side check, reported by the next blocking call
    ox, ov = diff.StepLowFn.apply(ctx, 1.0 / 240.0, 2, x, v)
    (ox[:, :3].sum() + ov[:, :3].sum()).backward()
    with pytest.raises(gs.GsError) as e:
        ctx.sync()
    assert e.value.code == gs.GS_ERR_STATE
    hx = torch.tensor(sc["hr_pos"], device="cuda", requires_grad=True)
    hv = torch.tensor(sc["hr_vel"], device="cuda", requires_grad=True)
    px, pv = diff.UpsampleFn.apply(ctx, DT, x.detach(), v.detach(), hx, hv)
    (px[:, :3].sum() + pv[:, :3].sum()).backward()
    with pytest.raises(gs.GsError) as e:
        ctx.sync()
    assert e.value.code == gs.GS_ERR_STATE
    ctx.sync()   # reported once; the context stays usable
    ctx.close()
