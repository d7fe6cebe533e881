"""Parity of the GPU upsampling frame (Sec. 4 gather, blend, advection and the
SDF rule) with the FP64 oracle on the same float32 inputs."""
import numpy as np
import pytest

import scenes
from gs_testutil import check_hr, up_prm

pytestmark = pytest.mark.gpu

DT = 1.0 / 60.0


def _run(sc, frames=1, **kw):
    import paper_2308_01629_gb300 as gs
    ctx = gs.Context(sc, **kw)
    for _ in range(frames):
        ctx.upsample(DT)
    x = ctx.read(gs.GS_FIELD_HR_POS)
    v = ctx.read(gs.GS_FIELD_HR_VEL)
    ctx.close()
    return x, v


def _ref(orc, sc, sub=None, mode=1):
    return orc.upsample(sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["hr_pos"][:, :3], sc["hr_vel"][:, :3],
                        scenes.sdf_table(sc["sdfs"]), up_prm(sc, DT), sub=sub, mode=mode)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_cube_every_particle(orc, seed):
    sc = scenes.stir(scenes.cube(), seed=seed)
    x, v = _run(sc)
    st = check_hr(sc, DT, x, v, _ref(orc, sc, mode=0))
    assert st["n"] == 8000
    np.testing.assert_array_equal(x[:, 3], sc["hr_pos"][:, 3])   # ids travel with the particle


def test_scene_straddling_the_origin(orc):
    """The stirred cube translated by -0.25 m on every axis (box [-0.25,
    0.25]^3): HR positions of both signs and near zero, a negative grid
    origin; the warp groups' bounding boxes (integer reductions over an
    order-preserving map of the floats) and the grid contract hold there."""
    sc = scenes.translated(scenes.stir(scenes.cube(), seed=13), (-0.25, -0.25, -0.25))
    assert (sc["hr_pos"][:, :3] < 0).any() and (sc["hr_pos"][:, :3] > 0).any()
    x, v = _run(sc)
    check_hr(sc, DT, x, v, _ref(orc, sc, mode=0))


def test_cube_without_reorder(orc):
    sc = scenes.stir(scenes.cube(), seed=4)
    x, v = _run(sc, resort_every=0)
    check_hr(sc, DT, x, v, _ref(orc, sc))


def _castle():
    """The grains of the sand castle seeded by the library's volume sampler."""
    import paper_2308_01629_gb300 as gs
    return scenes.castle_scene(gs.sample_volume, boulder=False)


@pytest.mark.parametrize("make,nsub", [(scenes.funnel, 20000), (scenes.digging, 20000), (_castle, 20000)])
def test_full_size_sampled(orc, make, nsub):
    sc = scenes.stir(make(), seed=5, spread=0.2)
    x, v = _run(sc)
    sub = np.sort(np.random.default_rng(6).choice(len(sc["hr_pos"]), size=nsub, replace=False))
    ref = _ref(orc, sc, sub=sub)
    check_hr(sc, DT, x[sub], v[sub], ref)


def test_lr_piles_many_particles_per_cell(orc):
    """LR particles piled on points (cells of 40, 100 and 300, ordered by a
    warp or the whole block) with distinct velocities: the binning's copies
    of position and velocity into cell order must be those of the ordered
    cells."""
    sc = scenes.stir(scenes.cube(), seed=7)
    rng = np.random.default_rng(8)
    lr = sc["lr_pos"].copy()
    pts = rng.uniform(0.15, 0.35, size=(6, 3)).astype(np.float32)
    lr[:120, :3] = np.repeat(pts[:3], 40, axis=0)
    lr[120:320, :3] = np.repeat(pts[3:5], 100, axis=0)
    lr[320:620, :3] = pts[5]
    sc["lr_pos"] = lr
    sc["lr_vel"] = sc["lr_vel"].copy()
    sc["lr_vel"][:, :3] = rng.normal(scale=0.3, size=(len(lr), 3)).astype(np.float32)
    x, v = _run(sc)
    check_hr(sc, DT, x, v, _ref(orc, sc, mode=0))


def test_uniform_field_and_isolated_particles(orc):
    sc = scenes.cube()
    u = np.array([0.3, -0.2, 0.1], np.float32)
    sc["lr_vel"] = np.zeros_like(sc["lr_vel"])
    sc["lr_vel"][:, :3] = u
    hr = sc["hr_pos"].copy()
    hr[:50, :3] = [[0.05 + 0.002 * k, 0.05, 0.45] for k in range(50)]   # far from every LR particle
    sc["hr_pos"] = hr
    sc["hr_vel"] = np.zeros_like(sc["hr_vel"])
    x, v = _run(sc)
    ref = _ref(orc, sc)
    check_hr(sc, DT, x, v, ref)
    inner = (ref["diag"][:, 2] == 0) & (ref["flag"] == 0)
    np.testing.assert_allclose(v[inner, :3], np.broadcast_to(u, (inner.sum(), 3)), rtol=0, atol=2e-7)
    free = v[:50, :3]
    np.testing.assert_allclose(free, np.broadcast_to([0, 0, -9.81 * DT], (50, 3)), rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("m", [1, 31, 33, 1000, 4097])
def test_ragged_sizes(orc, m):
    sc = scenes.stir(scenes.cube(n_side=17, ratio=1), seed=m)
    for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel"):
        sc[k] = sc[k][:m].copy()
    sc["hr_pos"][:, 3] = scenes.hr_ids(m)
    x, v = _run(sc)
    check_hr(sc, DT, x, v, _ref(orc, sc, mode=0))


def test_moving_bucket_and_cone(orc):
    # digging bed with the bucket placed inside the sand and a cone in the funnel
    sc = scenes.stir(scenes.digging(), seed=8, spread=0.5)
    sc = dict(sc)
    sc["sdfs"] = [sc["sdfs"][0], scenes.solid_box((0.5, 0.5, 0.25), (0.125, 0.075, 0.075), vel=(0.3, 0.0, -0.2))]
    x, v = _run(sc)
    c = np.array([0.5, 0.5, 0.25])
    near = np.nonzero(np.all(np.abs(sc["hr_pos"][:, :3] - c) < [0.14, 0.09, 0.09], axis=1))[0]
    sub = np.sort(np.random.default_rng(9).choice(near, size=min(20000, len(near)), replace=False))
    check_hr(sc, DT, x[sub], v[sub], _ref(orc, sc, sub=sub))
    sf = scenes.stir(scenes.funnel(), seed=10, spread=0.5)
    sf["hr_pos"][:, 2] -= 0.2   # into the cone shell region
    x, v = _run(sf)
    sub = np.sort(np.random.default_rng(11).choice(len(sf["hr_pos"]), size=20000, replace=False))
    check_hr(sf, DT, x[sub], v[sub], _ref(orc, sf, sub=sub))


def test_several_frames_with_reorders_match_unordered(orc):
    # the reorder changes only the internal order: several frames with and
    # without it agree within float32 rounding (summation order differs)
    sc = scenes.stir(scenes.cube(), seed=12)
    xa, va = _run(sc, frames=9, resort_every=2)
    xb, vb = _run(sc, frames=9, resort_every=0)
    np.testing.assert_array_equal(xa[:, 3], xb[:, 3])
    assert np.abs(xa[:, :3] - xb[:, :3]).max() < 1e-5


def test_gather_timer_in_graph_replayed_frames():
    """The gather timer records inside replayed frame graphs: a positive time
    for every frame, below the whole frame's."""
    import torch

    import paper_2308_01629_gb300 as gs
    sc = scenes.cube(n_side=10)
    s = torch.cuda.Stream()
    ctx = gs.Context(sc, stream=s.cuda_stream)
    assert gs.gs_gather_timer_ms(ctx.ctx)[0] == gs.GS_ERR_STATE
    ctx.set_gather_timer(True)
    ctx.set_graphs(True)
    for f in range(4):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        ctx.frame(1 / 60, 4, 4)
        b.record(s)
        g = ctx.gather_timer_ms()
        b.synchronize()
        assert 0.0 < g < a.elapsed_time(b)
    ctx.set_gather_timer(False)
    ctx.frame(1 / 60, 4, 4)
    ctx.sync()
    ctx.close()
