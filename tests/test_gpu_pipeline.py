"""Pipelined frames: the HR frame of frame f runs on a second stream while the
LR steps of frame f + 1 run.  The results must equal those of sequential
frames bit for bit: with and without CUDA graphs, with a boundary that moves
every frame (the deferred frame keeps the SDF table as of its frame), across
an HR reorder, with reads in between (each completes the deferred frame), and
for a batched context."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0


def _state(gs, ctx):
    return {k: ctx.read(f) for k, f in (("lr_x", gs.GS_FIELD_LR_POS), ("lr_v", gs.GS_FIELD_LR_VEL),
                                        ("hr_x", gs.GS_FIELD_HR_POS), ("hr_v", gs.GS_FIELD_HR_VEL))}


def _run(sc, nframes, pipeline, graphs, read_every=0, bucket=True, shape=(8, 1)):
    import paper_2308_01629_gb300 as gs
    ctx = gs.Context(sc)
    if pipeline:
        ctx.set_pipeline(True, *shape)
    ctx.set_graphs(graphs)
    mid = []
    for f in range(nframes):
        if bucket:
            ctx.set_sdf(1, scenes.bucket_sdf(f * DT))
        ctx.frame(DT, 4, 8)
        if read_every and (f + 1) % read_every == 0:
            mid.append(ctx.read(gs.GS_FIELD_HR_POS))
    out = _state(gs, ctx)
    ctx.sync()
    ctx.close()
    return out, mid


def _bucket_scene():
    sc = dict(scenes.digging(size=0.5))
    sc["sdfs"] = [sc["sdfs"][0], scenes.bucket_sdf(0.0)]
    return sc


@pytest.mark.parametrize("graphs", [False, True])
def test_pipelined_frames_equal_sequential_frames(graphs):
    sc = _bucket_scene()
    ref, _ = _run(sc, 10, pipeline=False, graphs=False)
    got, _ = _run(sc, 10, pipeline=True, graphs=graphs)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_pipelined_frames_with_reads_in_between():
    sc = _bucket_scene()
    ref, ref_mid = _run(sc, 9, pipeline=False, graphs=True, read_every=3)
    got, got_mid = _run(sc, 9, pipeline=True, graphs=True, read_every=3)
    for a, b in zip(got_mid, ref_mid):
        np.testing.assert_array_equal(a, b)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


@pytest.mark.parametrize("shape", [(8, 0), (16, 2), (4, 1)])
def test_pipelined_batch_equals_sequential_batch(shape):
    sl = scenes.batch(n_scenes=12, lo_count=300, hi_count=1500)
    ref, _ = _run(sl, 9, pipeline=False, graphs=True, bucket=False)
    got, _ = _run(sl, 9, pipeline=True, graphs=True, bucket=False, shape=shape)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_pipeline_rejects_unknown_launch_shape():
    import paper_2308_01629_gb300 as gs
    ctx = gs.Context(scenes.cube(n_side=4))
    assert gs.gs_set_pipeline(ctx.ctx, 1, 7, 1) == gs.GS_ERR_ARG
    ctx.close()
