"""The library's volume sampler (Sec. 4 initial sampling, gs_sample_volume)
against the oracle's: the same inside decisions and the same chosen
candidates in the same order, bit for bit, on a sphere, the castle union
at the LR and the HR radius, and edge cases; then a castle scene seeded by
it (LR and HR particles, and a rigid boulder sampled from an icosphere)
runs frames."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def _both(orc, V, T, cand, r):
    import paper_2308_01629_gb300 as gs
    rc, sel, inside = gs.gs_sample_volume(V, T, cand, r)
    assert rc == gs.GS_OK
    ref_sel, ref_inside = orc.sample_volume(V, T, cand, r)
    np.testing.assert_array_equal(inside, ref_inside)
    np.testing.assert_array_equal(sel, ref_sel)
    return sel


@pytest.mark.parametrize("r, per_cell", [(0.012, 5.0), (0.004, 4.0)])
def test_sphere_samples_equal_the_oracle(orc, r, per_cell):
    V, T = scenes.icosphere((0.3, 0.2, 0.1), 0.15, 2)
    cand = scenes.volume_candidates(V, r, per_cell=per_cell, seed=21)
    sel = _both(orc, V, T, cand, r)
    assert len(sel) > 100


@pytest.mark.parametrize("r", [0.02, 0.0075])
def test_castle_samples_equal_the_oracle(orc, r):
    orc.set_threads(orc.max_threads())
    V, T = scenes.castle_mesh()
    cand = scenes.volume_candidates(V, r, per_cell=3.0, seed=22)
    sel = _both(orc, V, T, cand, r)
    orc.set_threads(1)
    P = cand[sel]
    # spot check of the spacing on a random subset (the oracle's pins cover the rest)
    rng = np.random.default_rng(0)
    sub = P[rng.choice(len(P), size=min(len(P), 1500), replace=False)]
    d2 = ((sub[:, None] - sub[None]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    assert d2.min() >= 4 * r * r


def test_sampler_edge_cases_on_the_gpu(orc):
    import paper_2308_01629_gb300 as gs
    V, T = scenes.box_mesh((0, 0, 0), (0.1, 0.1, 0.1))
    for cand in (np.zeros((0, 3)), [[0.05, 0.05, 0.05]], [[0.5, 0.5, 0.5], [-1, 0, 0]],
                 [[0.05, 0.05, 0.05], [0.0501, 0.05, 0.05]]):
        _both(orc, V, T, np.asarray(cand, float).reshape(-1, 3), 0.01)
    cand = scenes.volume_candidates(V, 0.01, seed=3)
    rc, sel, _ = gs.gs_sample_volume(V, T, cand, 0.01, capacity=3)
    assert rc == gs.GS_ERR_CAPACITY and len(sel) == 3
    rc, sel, inside = gs.gs_sample_volume(V, np.zeros((0, 3), np.int32), cand, 0.01)   # no triangles: nothing inside
    assert rc == gs.GS_OK and len(sel) == 0 and not inside.any()


def test_castle_scene_seeded_by_the_sampler_runs():
    import paper_2308_01629_gb300 as gs
    sc = scenes.castle_scene(gs.sample_volume, size=0.6, height=0.2, r_low=0.02, r_high=0.0075)
    assert sc["ratio"] >= 15 and len(sc["hr_pos"]) > 10 * len(sc["lr_pos"])
    ctx = gs.Context(sc)
    x0 = ctx.read(gs.GS_FIELD_HR_POS)
    for _ in range(6):
        ctx.frame(1.0 / 60.0, 4, sc["iters"])
    x1 = ctx.read(gs.GS_FIELD_HR_POS)
    lr = ctx.read(gs.GS_FIELD_LR_POS)
    assert np.isfinite(x1).all() and np.isfinite(lr).all()
    body = sc["lr_body"] > 0
    assert np.abs(lr[body, :3] - sc["lr_pos"][body, :3]).max() > 0.05    # the boulder flew
    assert np.abs(x1[:, :3] - x0[:, :3]).max() > 0.0
    ctx.close()


def test_surface_samples_equal_the_oracle_and_the_mesh_bucket_runs(orc):
    import paper_2308_01629_gb300 as gs
    for V, T, r in [(*scenes.box_mesh((0.1, 0.2, 0.05), (0.35, 0.3, 0.2)), 0.01),
                    (*scenes.icosphere((0.0, 0.0, 0.0), 0.2, 3), 0.006)]:
        cand = scenes.surface_candidates(V, T, r, seed=9)
        rc, sel = gs.gs_sample_surface(V, cand, r)
        assert rc == gs.GS_OK
        np.testing.assert_array_equal(sel, orc.sample_surface(V, cand, r))
    sc = scenes.digging_mesh_bucket(gs.sample_surface, size=0.5)
    ctx = gs.Context(sc)
    n_g = len(sc["lr_pos"]) - sc["n_solid"]
    x0 = ctx.read(gs.GS_FIELD_LR_POS)
    for _ in range(4):
        ctx.frame(1.0 / 60.0, 4, sc["iters"])
    x1 = ctx.read(gs.GS_FIELD_LR_POS)
    assert np.isfinite(x1).all() and np.isfinite(ctx.read(gs.GS_FIELD_HR_POS)).all()
    # the boundary particles move with their prescribed velocity
    u = sc["lr_vel"][n_g:, :3]
    np.testing.assert_allclose(x1[n_g:, :3] - x0[n_g:, :3], 4 / 60.0 * u, atol=1e-5)
    ctx.close()
