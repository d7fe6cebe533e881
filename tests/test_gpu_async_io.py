"""Asynchronous field transfers: gs_write_async / gs_read_async give the same
results as gs_write / gs_read, in the order the calls were made, with and
without graph replay, across HR reorders; a non-finite asynchronous write is
reported at the next sync."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0
FIELDS = ("lr_pos", "lr_vel", "hr_pos", "hr_vel")


def _fields(gs):
    return dict(zip(FIELDS, (gs.GS_FIELD_LR_POS, gs.GS_FIELD_LR_VEL, gs.GS_FIELD_HR_POS, gs.GS_FIELD_HR_VEL)))


def _perturbed(sc, k):
    """A different state for round k (shifted positions, scaled velocities)."""
    st = {n: np.ascontiguousarray(sc[n]).copy() for n in FIELDS}
    st["lr_pos"][:, :3] += 1e-4 * k
    st["hr_pos"][:, :3] -= 1e-4 * k
    st["lr_vel"][:, :3] *= 1.0 + 0.1 * k
    st["hr_vel"][:, :3] += 0.01 * k
    return st


@pytest.mark.parametrize("graphs", [False, True])
def test_async_transfers_equal_synchronous_ones(graphs):
    import paper_2308_01629_gb300 as gs
    F = _fields(gs)
    sc = scenes.stir(scenes.cube(), seed=3, v_scale=0.3)
    states = [_perturbed(sc, k) for k in range(4)]
    # synchronous reference
    ref_ctx = gs.Context(sc)
    ref_ctx.set_graphs(graphs)
    ref = []
    for k, st in enumerate(states):
        for n in FIELDS:
            ref_ctx.write(F[n], st[n])
        for _ in range(k + 1):   # several frames, so some rounds start after an HR reorder
            ref_ctx.frame(DT, 4, 8)
        ref.append({n: ref_ctx.read(F[n]) for n in FIELDS})
    ref_ctx.close()
    # asynchronous
    ctx = gs.Context(sc)
    ctx.set_graphs(graphs)
    outs = []
    for k, st in enumerate(states):
        for n in FIELDS:
            ctx.write_async(F[n], st[n])
        for _ in range(k + 1):
            ctx.frame(DT, 4, 8)
        o = {n: np.zeros_like(st[n]) for n in FIELDS}
        for n in FIELDS:
            ctx.read_async(F[n], o[n])
        outs.append(o)
    ctx.sync()
    ctx.close()
    for k in range(len(states)):
        for n in FIELDS:
            np.testing.assert_array_equal(outs[k][n], ref[k][n], err_msg=f"round {k} {n}")


def test_async_transfers_at_full_size():
    """The 2M-particle digging bed, graphs on, as a caller streams it: every
    round writes all four fields asynchronously, runs frames and reads the HR
    fields asynchronously, without a sync in between (copies in flight on
    their own streams while frames run): the results equal the synchronous
    calls' bit for bit."""
    import paper_2308_01629_gb300 as gs
    F = _fields(gs)
    sc = scenes.stir(scenes.digging(), seed=9, v_scale=0.1)
    states = [_perturbed(sc, k) for k in range(3)]
    ref_ctx = gs.Context(sc)
    ref_ctx.set_graphs(True)
    ref = []
    for k, st in enumerate(states):
        for n in FIELDS:
            ref_ctx.write(F[n], st[n])
        for _ in range(2):
            ref_ctx.frame(DT, 4, 8)
        ref.append({n: ref_ctx.read(F[n]) for n in ("hr_pos", "hr_vel")})
    ref_ctx.close()
    ctx = gs.Context(sc)
    ctx.set_graphs(True)
    outs = []
    for k, st in enumerate(states):
        for n in FIELDS:
            ctx.write_async(F[n], st[n])
        for _ in range(2):
            ctx.frame(DT, 4, 8)
        o = {n: np.zeros_like(st[n]) for n in ("hr_pos", "hr_vel")}
        for n in ("hr_pos", "hr_vel"):
            ctx.read_async(F[n], o[n])
        outs.append(o)
    ctx.sync()
    ctx.close()
    for k in range(len(states)):
        for n in ("hr_pos", "hr_vel"):
            np.testing.assert_array_equal(outs[k][n], ref[k][n], err_msg=f"round {k} {n}")


def test_async_read_is_a_snapshot_and_last_write_wins():
    import paper_2308_01629_gb300 as gs
    F = _fields(gs)
    sc = scenes.stir(scenes.cube(n_side=5), seed=4, v_scale=0.3)
    a, b = _perturbed(sc, 1), _perturbed(sc, 2)
    ctx = gs.Context(sc)
    ctx.write_async(F["hr_vel"], a["hr_vel"])
    ctx.write_async(F["hr_vel"], b["hr_vel"])           # supersedes the first before any commit
    snap = np.zeros_like(b["hr_vel"])
    ctx.read_async(F["hr_vel"], snap)                   # the value at this point ...
    ctx.frame(DT, 4, 8)                                 # ... not after this frame
    ctx.sync()
    np.testing.assert_array_equal(snap, b["hr_vel"])
    assert not np.array_equal(ctx.read(F["hr_vel"]), snap)
    ctx.close()


def test_hr_reads_share_one_snapshot_only_while_nothing_ran():
    """An asynchronous read of one HR field snapshots both; the other's read
    uses that snapshot only if no kernel ran in between (a frame, a write),
    in either order, and a field read twice is snapshotted twice."""
    import paper_2308_01629_gb300 as gs
    F = _fields(gs)
    sc = scenes.stir(scenes.cube(n_side=6), seed=5, v_scale=0.3)
    ctx = gs.Context(sc)
    ctx.set_graphs(True)
    ctx.frame(DT, 4, 8)
    for first, second in (("hr_pos", "hr_vel"), ("hr_vel", "hr_pos")):
        a = np.zeros_like(sc[first])
        b = np.zeros_like(sc[second])
        ctx.read_async(F[first], a)
        ctx.frame(DT, 4, 8)                  # between the two reads
        ctx.read_async(F[second], b)
        ctx.sync()
        want_b = ctx.read(F[second])         # the state after the frame
        np.testing.assert_array_equal(b, want_b, err_msg=f"{first} then frame then {second}")
        # back to back: the pair, then the same field again
        a2, b2, a3 = np.zeros_like(a), np.zeros_like(b), np.zeros_like(a)
        ctx.read_async(F[first], a2)
        ctx.read_async(F[second], b2)
        ctx.read_async(F[first], a3)
        ctx.sync()
        np.testing.assert_array_equal(a2, ctx.read(F[first]))
        np.testing.assert_array_equal(b2, want_b)
        np.testing.assert_array_equal(a3, a2)
    # a write between the two reads is seen by the second one
    v = np.ascontiguousarray(sc["hr_vel"]).copy()
    v[:, :3] += 0.25
    x = np.zeros_like(sc["hr_pos"])
    got = np.zeros_like(v)
    ctx.read_async(F["hr_pos"], x)
    ctx.write_async(F["hr_vel"], v)
    ctx.read_async(F["hr_vel"], got)
    ctx.sync()
    np.testing.assert_array_equal(got, v)
    ctx.close()


def test_non_finite_async_write_is_reported_at_sync():
    import paper_2308_01629_gb300 as gs
    F = _fields(gs)
    sc = scenes.cube(n_side=4)
    bad = np.ascontiguousarray(sc["lr_vel"]).copy()
    bad[3, 2] = np.inf
    ctx = gs.Context(sc)
    ctx.write_async(F["lr_vel"], bad)
    ctx.frame(DT, 4, 8)
    with pytest.raises(gs.GsError) as e:
        ctx.sync()
    assert e.value.code == gs.GS_ERR_DOMAIN
    ctx.close()
