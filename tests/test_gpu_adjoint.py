"""The differentiable pattern on the GPU: reverse modes of the HR frame and of
the LR step against the oracle's analytic reverse modes, autograd wiring, and
checkpointed rollouts."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / max(np.linalg.norm(b), 1e-30))


def small_upsample_state(seed):
    """A stirred 6^3 cube inside planar walls, a few HR particles just
    outside a wall and moving outwards (the wall rule is active for them)."""
    sc = dict(scenes.stir(scenes.cube(n_side=6, ratio=6), seed=seed, spread=0.6))
    sc["sdfs"] = [scenes.box_interior((0.19, 0.19, 0.14), (0.31, 0.31, 0.40))]
    hr = sc["hr_pos"].copy()
    rng = np.random.default_rng(seed)
    hr[:8, 0] = 0.19 + rng.uniform(-0.004, 0.001, 8)
    sc["hr_pos"] = hr
    return sc


def up_prm(sc):
    return dict(r_low=float(np.float32(sc["r_low"])), r_high=float(np.float32(sc["r_high"])),
                dt=float(np.float32(DT)), gx=0.0, gy=0.0, gz=float(np.float32(-9.81)), c1=512 / 729, c2=0.6,
                eps_w=1e-4, eps_x=1e-6)


@pytest.mark.parametrize("seed", [1, 2])
def test_upsample_backward_matches_oracle(orc, seed):
    import torch

    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300.diff import UpsampleFn
    sc = small_upsample_state(seed)
    g = gs.Context(sc, stream="torch")
    ref = orc.upsample(sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["hr_pos"][:, :3], sc["hr_vel"][:, :3],
                       scenes.sdf_table(sc["sdfs"]), up_prm(sc))
    keep = (ref["flag"] == 0)[:, None]
    rng = np.random.default_rng(seed)
    a = (rng.normal(size=(len(keep), 3)) * keep).astype(np.float32)
    b = (rng.normal(size=(len(keep), 3)) * keep).astype(np.float32)
    X, V, x, v = (_t(sc[k]).requires_grad_(True) for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel"))
    ox, ov = UpsampleFn.apply(g, DT, X, V, x, v)
    np.testing.assert_allclose(ox.detach().cpu().numpy()[:, :3][keep[:, 0]], ref["x"][keep[:, 0]], rtol=1e-5,
                               atol=1e-6)
    loss = (ox[:, :3] * _t(a)).sum() + (ov[:, :3] * _t(b)).sum()
    loss.backward()
    gX, gV, gx, gv = orc.upsample_vjp(sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["hr_pos"][:, :3],
                                      sc["hr_vel"][:, :3], scenes.sdf_table(sc["sdfs"]), up_prm(sc), a, b)
    for got, want in ((X.grad, gX), (V.grad, gV), (x.grad, gx), (v.grad, gv)):
        got = got.cpu().numpy()
        assert np.all(got[:, 3] == 0)
        assert _rel(got[:, :3], want) < 2e-4
    g.close()


def _lr_case(name):
    rng = np.random.default_rng(7)
    r = 0.01
    box = scenes.box_interior((-1, -1, 0), (1, 1, 1))
    if name == "cluster":
        grid = np.stack(np.meshgrid(*[np.arange(3)] * 3, indexing="ij"), -1).reshape(-1, 3) * 1.9 * r
        x = grid + [0.3, 0.3, 0.3] + rng.uniform(-0.1 * r, 0.1 * r, grid.shape)
        v = rng.normal(0, 0.2, x.shape)
    else:
        x = np.array([[0.1, 0.1, r * 0.97], [0.3, 0.1, r * 0.98], [0.5, 0.1, r * 0.99], [0.52, 0.1, r * 2.9]])
        v = np.array([[1.2, 0.3, 0.0], [0.05, -0.02, 0.0], [0.6, 0.0, -0.1], [-0.4, 0.2, 0.0]])
    n = len(x)
    sc = dict(name=name, box_lo=[-1.0, -1.0, 0.0], box_hi=[1.0, 1.0, 1.0], r_low=r, r_high=0.004, ratio=1,
              sdfs=[box], gravity=(0.0, 0.0, -9.81), mu_s=0.35, mu_k=0.30,
              lr_pos=np.column_stack([x, np.ones(n)]).astype(np.float32),
              lr_vel=np.column_stack([v, np.zeros(n)]).astype(np.float32))
    sc["hr_pos"] = sc["lr_pos"].copy()
    sc["hr_vel"] = sc["lr_vel"].copy()
    return sc


@pytest.mark.parametrize("name,mass_k,mode", [("cluster", 2.0, 0), ("floor", 0.0, 0), ("floor", 0.0, 1)])
def test_step_low_backward_matches_oracle(orc, name, mass_k, mode):
    import torch

    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300.diff import StepLowFn
    sc = _lr_case(name)
    dt = 1.0 / 240.0
    g = gs.Context(sc, stream="torch", mass_scale_k=mass_k, friction_mode=mode, n_stab=2)
    x32 = sc["lr_pos"][:, :3].astype(float)
    v32 = sc["lr_vel"][:, :3].astype(float)
    prm = dict(r=float(np.float32(0.01)), dt=float(np.float32(dt)), gx=0.0, gy=0.0, gz=float(np.float32(-9.81)),
               mu_s=float(np.float32(0.35)), mu_k=float(np.float32(0.30)), n_stab=2, iters=4, mass_k=mass_k,
               ground_z=0.0, rc=float(np.float32(3 * np.float32(0.01))), friction_mode=mode, eps_x=1e-6,
               eps_impact=0.0)
    _, _, _, st = orc.pbd_step(x32, v32, np.ones(len(x32)), scenes.sdf_table(sc["sdfs"]), prm)
    assert st["significant"] == 0
    rng = np.random.default_rng(5)
    a = rng.normal(size=x32.shape).astype(np.float32)
    b = rng.normal(size=x32.shape).astype(np.float32)
    X, V = _t(sc["lr_pos"]).requires_grad_(True), _t(sc["lr_vel"]).requires_grad_(True)
    ox, ov = StepLowFn.apply(g, dt, 4, X, V)
    loss = (ox[:, :3] * _t(a)).sum() + (ov[:, :3] * _t(b)).sum()
    loss.backward()
    gx, gv = orc.pbd_step_vjp(x32, v32, np.ones(len(x32)), scenes.sdf_table(sc["sdfs"]), prm, a, b)
    assert _rel(X.grad.cpu().numpy()[:, :3], gx) < 1e-3
    assert _rel(V.grad.cpu().numpy()[:, :3], gv) < 1e-3
    g.close()


def test_checkpointed_rollout_equals_plain_rollout():
    import torch

    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300.diff import rollout
    sc = scenes.column(n_low=400, ratio=8)
    g = gs.Context(sc, stream="torch")
    grads = []
    for every in (0, 5):
        X, V, x, v = (_t(sc[k]) for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel"))
        V.requires_grad_(True)
        out = rollout(g, X, V, x, v, DT, frames=12, n_sub=2, iters=4, checkpoint_every=every)
        target = torch.zeros_like(out[2][:, :3])
        loss = ((out[2][:, :3] - target) ** 2).sum()
        loss.backward()
        grads.append(V.grad.cpu().numpy()[:, :3].copy())
    assert np.abs(grads[0]).max() > 0
    assert _rel(grads[1], grads[0]) < 1e-5
    g.close()


def test_graph_replayed_functional_steps_equal_direct_launches():
    """With graphs enabled on a stream that can be captured, the functional
    LR step entry points replay their fixed sequence as a CUDA graph; the
    forward outputs must be the same bits as direct launches, also on the
    second and later calls (replays), and the gradients the same up to the
    order of the reverse kernels' atomic accumulations (which varies from run
    to run with or without graphs)."""
    import torch

    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300.diff import rollout
    sc = scenes.column(n_low=400, ratio=8)
    s = torch.cuda.Stream()
    grads = {}
    with torch.cuda.stream(s):
        for graphs in (False, True):
            g = gs.Context(sc, stream=s.cuda_stream)
            g.set_graphs(graphs)
            out = []
            for rep in range(3):
                X, V, x, v = (_t(sc[k]) for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel"))
                V.requires_grad_(True)
                res = rollout(g, X, V, x, v, DT, frames=6, n_sub=2, iters=4, checkpoint_every=3)
                loss = (res[2][:, :3] ** 2).sum()
                loss.backward()
                out.append((res[0].detach().cpu().numpy(), V.grad.cpu().numpy()))
            torch.cuda.synchronize()
            g.close()
            grads[graphs] = out
    for a, b in zip(grads[False], grads[True]):
        np.testing.assert_array_equal(a[0], b[0])
        assert _rel(b[1], a[1]) < 1e-5
    assert np.abs(grads[True][0][1]).max() > 0


def _gpu_forward_states(g, sc):
    """The GPU forward of the differentiation workload, step by step, with the
    inputs of every operation kept as float32 tensors."""
    import torch

    from paper_2308_01629_gb300.diff import StepLowFn, UpsampleFn
    X, V, x, v = (_t(sc[k]) for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel"))
    ops = []
    with torch.no_grad():
        for _ in range(sc["steps"]):
            ops.append(("lr", X.clone(), V.clone()))
            X, V = StepLowFn.apply(g, sc["dt"], sc["iters"], X, V)
            ops.append(("hr", X.clone(), V.clone(), x.clone(), v.clone()))
            x, v = UpsampleFn.apply(g, sc["dt"], X, V, x, v)
    return ops, X, V, x


def _f64(t):
    return t.cpu().numpy()[:, :3].astype(np.float64)


def _lr_tape(cand, pair, sdfb, n):
    """The oracle's LR-step tape (pbd_step_tape's layout) from the decision
    record of one GPU reverse step: every candidate pair once (i < j) with
    its per-pass bits, then the per-pass SDF bits."""
    k, i = np.nonzero(cand >= 0)
    j = cand[k, i].astype(np.int64)
    sel = i < j
    k, i, j = k[sel], i[sel], j[sel]
    order = np.lexsort((j, i))
    k, i, j = k[order], i[order], j[order]
    passes, ncomp = pair.shape[0], sdfb.shape[2]
    head = np.array([len(i), n, ncomp, passes], np.int64)
    parts = [head.view(np.uint8), np.stack([i, j], 1).astype(np.int64).ravel().view(np.uint8)]
    for q in range(passes):
        parts.append(np.ascontiguousarray(pair[q][k, i]))
        parts.append(np.ascontiguousarray(sdfb[q]).ravel())
    return np.concatenate(parts)


def _gpu_decision_tapes(gs, g, sc, ops, iters, n_stab=2):
    """Oracle tapes of the decisions the GPU's reverse modes take at every
    operation of its own rollout (gs_set_decision_record)."""
    import torch
    n, m = len(sc["lr_pos"]), len(sc["hr_pos"])
    cap, passes = 64, n_stab + iters
    ncomp = sum(6 if s["kind"] == scenes.SDF_BOX_INTERIOR else 1 for s in sc["sdfs"])
    hr = torch.zeros((m, 4), dtype=torch.int32, device="cuda")
    cand = torch.zeros((cap, n), dtype=torch.int32, device="cuda")
    pair = torch.zeros((passes, cap, n), dtype=torch.uint8, device="cuda")
    sdfb = torch.zeros((passes, n, max(ncomp, 1)), dtype=torch.uint8, device="cuda")
    rc = gs.gs_set_decision_record(g.ctx, hr.data_ptr(), cand.data_ptr(), pair.data_ptr(), sdfb.data_ptr(), passes)
    assert rc == gs.GS_OK, gs.gs_last_error(g.ctx)
    zl, zh = torch.zeros((n, 4), device="cuda"), torch.zeros((m, 4), device="cuda")
    o1, o2 = torch.empty((n, 4), device="cuda"), torch.empty((n, 4), device="cuda")
    h1, h2 = torch.empty((m, 4), device="cuda"), torch.empty((m, 4), device="cuda")
    dt = float(np.float32(sc["dt"]))
    tapes = []
    for op in ops:
        if op[0] == "lr":
            _, X, V = op
            rc = gs.gs_step_low_backward(g.ctx, X.data_ptr(), V.data_ptr(), zl.data_ptr(), zl.data_ptr(),
                                         o1.data_ptr(), o2.data_ptr(), dt, iters)
            assert rc == gs.GS_OK, gs.gs_last_error(g.ctx)
            g.sync()
            tapes.append(_lr_tape(cand.cpu().numpy(), pair.cpu().numpy(), sdfb.cpu().numpy()[:, :, :ncomp], n))
        else:
            _, X, V, x, v = op
            rc = gs.gs_upsample_backward(g.ctx, X.data_ptr(), V.data_ptr(), x.data_ptr(), v.data_ptr(), zh.data_ptr(),
                                         zh.data_ptr(), o1.data_ptr(), o2.data_ptr(), h1.data_ptr(), h2.data_ptr(), dt)
            assert rc == gs.GS_OK, gs.gs_last_error(g.ctx)
            g.sync()
            tapes.append(hr.cpu().numpy().view(np.uint32).copy())
    assert gs.gs_set_decision_record(g.ctx, None, None, None, None, 0) == gs.GS_OK
    return tapes


def test_rollout_gradient_config4_matches_oracle(orc):
    """Falling column, 4k LR / 64k HR, 30 steps, checkpoints every 5: the GPU
    gradient of the loss w.r.t. the initial LR velocities against the
    oracle's analytic gradient on the same smooth piece of the method.

    The method is piecewise smooth: resting contacts sit at |x_ij| = 2 r_LR,
    where the contact test is decided by rounding, and an active contact at
    zero penetration still contributes the rank-one Jacobian -u u^T and
    changes n_i.  The float32 rollout and the FP64 one therefore take some
    of these decisions differently and differentiate different pieces
    (measured: 2.4e-2 apart on the directional derivative, 8e-2 in L2).  The
    GPU's reverse modes record the decisions they differentiate at every
    operation of the GPU's own rollout; the oracle replays them in its FP64
    rollout and in its reverse modes, and the GPU gradient must equal that
    analytic gradient within 1e-3, which central differences (eps 1e-4) of
    the replayed oracle rollout confirm."""
    import torch

    import paper_2308_01629_gb300 as gs
    from gs_testutil import diff_prms
    from paper_2308_01629_gb300.diff import rollout
    sc = scenes.diff_column()
    assert len(sc["lr_pos"]) == 4000 and len(sc["hr_pos"]) == 64000
    pb, up = diff_prms(sc)
    T32 = sc["target"]
    g = gs.Context(sc, stream="torch")
    X, V, x, v = (_t(sc[k]) for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel"))
    V.requires_grad_(True)
    out = rollout(g, X, V, x, v, sc["dt"], frames=sc["steps"], n_sub=1, iters=sc["iters"],
                  checkpoint_every=sc["checkpoint_every"])
    loss = ((out[2][:, :3] - _t(T32)) ** 2).sum()
    loss.backward()
    gv_gpu = V.grad.cpu().numpy()[:, :3].astype(np.float64)
    assert np.all(V.grad.cpu().numpy()[:, 3] == 0)

    im = sc["lr_pos"][:, 3].astype(float)
    sdf = scenes.sdf_table(sc["sdfs"])
    T = T32.astype(float)
    X0, V0, x0, v0 = (sc[k][:, :3].astype(float) for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel"))
    rng = np.random.default_rng(23)
    d = rng.normal(size=V0.shape)
    eps = 1e-4

    def fd_of(tapes):
        lp = orc.rollout(X0, V0 + eps * d, im, x0, v0, sdf, pb, up, sc["steps"], tapes=tapes)["hr_x"]
        lm = orc.rollout(X0, V0 - eps * d, im, x0, v0, sdf, pb, up, sc["steps"], tapes=tapes)["hr_x"]
        return (((lp - T) ** 2).sum() - ((lm - T) ** 2).sum()) / (2 * eps)

    # the oracle's own piece (its FP64 decisions), for the record
    ro = orc.rollout(X0, V0, im, x0, v0, sdf, pb, up, sc["steps"])
    _, gv_or, _, _ = orc.rollout_vjp(ro, im, sdf, pb, up, 2.0 * (ro["hr_x"] - T), np.zeros_like(T))
    fd_own = fd_of(ro["tapes"])
    # the GPU's piece: its reverse modes' decisions along its own rollout
    ops, Xg, Vg, xg = _gpu_forward_states(g, sc)
    tapes = _gpu_decision_tapes(gs, g, sc, ops, sc["iters"])
    rg = orc.rollout(X0, V0, im, x0, v0, sdf, pb, up, sc["steps"], tapes=tapes)
    _, gv_piece, _, _ = orc.rollout_vjp(rg, im, sdf, pb, up, 2.0 * (rg["hr_x"] - T), np.zeros_like(T), replay=True)
    fd_piece = fd_of(tapes)
    dir_gpu, dir_piece = float((gv_gpu * d).sum()), float((gv_piece * d).sum())
    report = dict(dir_gpu=dir_gpu, dir_piece=dir_piece, fd_piece=fd_piece,
                  rel_l2_piece=_rel(gv_gpu, gv_piece), rel_dir_piece=abs(dir_gpu - dir_piece) / abs(dir_piece),
                  rel_piece_fd=abs(dir_piece - fd_piece) / abs(fd_piece),
                  rel_oracle_fd=abs(float((gv_or * d).sum()) - fd_own) / abs(fd_own),
                  rel_l2_own_piece=_rel(gv_gpu, gv_or), rel_dir_own_fd=abs(dir_gpu - fd_own) / abs(fd_own),
                  norm=float(np.linalg.norm(gv_piece)))
    # the replayed FP64 rollout follows the GPU's float32 one: float32
    # rounding accumulates to about 1e-3 r_LR over the 30 steps (measured:
    # 99th percentile 1.1e-5 m, r_LR = 0.01 m), and a rare HR particle moves
    # further where the upsampling forward and its reverse, which evaluate
    # the weights in different float32 forms, decide a threshold differently
    gap = np.linalg.norm(rg["hr_x"] - _f64(xg), axis=1)
    lgap = np.linalg.norm(rg["lr_x"] - _f64(Xg), axis=1)
    report.update(hr_gap_q=[float(q) for q in np.quantile(gap, [0.5, 0.99, 0.999, 1.0])],
                  lr_gap_q=[float(q) for q in np.quantile(lgap, [0.5, 0.99, 0.999, 1.0])],
                  hr_gap_frac=float((gap > 1e-5).mean()), lr_gap_max=float(lgap.max()))
    r = sc["r_low"]
    print("config4", report)
    g.close()
    # the oracle's analytic gradient is the derivative of its replayed rollout
    assert report["rel_oracle_fd"] <= 1e-6, report
    assert report["rel_piece_fd"] <= 1e-6, report
    assert report["hr_gap_q"][1] <= 5e-3 * r and report["hr_gap_q"][3] <= 5e-2 * r, report
    assert report["lr_gap_max"] <= 5e-3 * r, report
    # the GPU gradient on its own smooth piece
    assert report["rel_l2_piece"] <= 1e-3, report
    assert report["rel_dir_piece"] <= 1e-3, report


def _lr_reverse_case(orc, sc, g, X, V, n_stab, iters, eps_x, rng):
    """GPU and oracle reverse of one LR step at a float32 state, upstream
    zeroed on the oracle's suspects; returns (rel gx, rel gv, suspect frac)."""
    from gs_testutil import pb_prm
    from paper_2308_01629_gb300.diff import StepLowFn
    pb = pb_prm(sc, sc["dt"], n_stab, iters, eps_x=eps_x, eps_impact=0.0)
    im = sc["lr_pos"][:, 3].astype(float)
    sdf = scenes.sdf_table(sc["sdfs"])
    _, _, sus, _ = orc.pbd_step(_f64(X), _f64(V), im, sdf, pb, mode=1)
    keep = ~sus
    a = (rng.normal(size=(len(keep), 3)) * keep[:, None]).astype(np.float32)
    b = (rng.normal(size=(len(keep), 3)) * keep[:, None]).astype(np.float32)
    Xr, Vr = X.clone().requires_grad_(True), V.clone().requires_grad_(True)
    ox, ov = StepLowFn.apply(g, sc["dt"], iters, Xr, Vr)
    ((ox[:, :3] * _t(a)).sum() + (ov[:, :3] * _t(b)).sum()).backward()
    gx, gv = orc.pbd_step_vjp(_f64(X), _f64(V), im, sdf, pb, a, b)
    return _rel(Xr.grad.cpu().numpy()[:, :3], gx), _rel(Vr.grad.cpu().numpy()[:, :3], gv), float(sus.mean())


@pytest.mark.parametrize("step", [0, 9, 19, 29])
def test_stepwise_reverse_along_config4_trajectory(orc, step):
    """Per-operation reverse modes at states of the GPU's own config-4
    rollout, against the oracle's at the same float32 states.  Upstream
    gradients are zeroed on the particles whose result the oracle finds to
    hang on a decision within float32 reach of its threshold, so both sides
    differentiate the same smooth piece.  In the packed column most LR
    particles carry a resting contact at |x_ij| = 2 r_LR, and over the six
    passes of a step the ambiguity spreads to nearly all of them; single
    passes (solver, stabilization) are therefore compared as well, where it
    does not spread."""
    import paper_2308_01629_gb300 as gs
    from gs_testutil import diff_prms
    from paper_2308_01629_gb300.diff import UpsampleFn
    sc = scenes.diff_column()
    _, up = diff_prms(sc)
    g = gs.Context(sc, stream="torch")
    g_solve = gs.Context(sc, stream="torch", n_stab=0)
    g_stab = gs.Context(sc, stream="torch", n_stab=1)
    ops, _, _, _ = _gpu_forward_states(g, sc)
    sdf = scenes.sdf_table(sc["sdfs"])
    rng = np.random.default_rng(1000 + step)
    res = {}
    _, X, V = ops[2 * step]
    for name, ctx, n_stab, iters, eps_x in (("step", g, 2, 4, 1e-7), ("solve1", g_solve, 0, 1, 2e-8),
                                            ("stab1", g_stab, 1, 0, 2e-8)):
        res[name + "_gx"], res[name + "_gv"], res[name + "_suspect_frac"] = _lr_reverse_case(
            orc, sc, ctx, X, V, n_stab, iters, eps_x, rng)
    # HR frame
    _, X, V, x, v = ops[2 * step + 1]
    ref = orc.upsample(_f64(X), _f64(V), _f64(x), _f64(v), sdf, up, mode=1)
    keep = ref["flag"] == 0
    a = (rng.normal(size=(len(keep), 3)) * keep[:, None]).astype(np.float32)
    b = (rng.normal(size=(len(keep), 3)) * keep[:, None]).astype(np.float32)
    ins = [t.clone().requires_grad_(True) for t in (X, V, x, v)]
    oxh, ovh = UpsampleFn.apply(g, sc["dt"], *ins)
    ((oxh[:, :3] * _t(a)).sum() + (ovh[:, :3] * _t(b)).sum()).backward()
    want = orc.upsample_vjp(_f64(X), _f64(V), _f64(x), _f64(v), sdf, up, a, b)
    for name, t, w in zip(("hr_gX", "hr_gV", "hr_gx", "hr_gv"), ins, want):
        res[name] = _rel(t.grad.cpu().numpy()[:, :3], w)
    res["hr_flag_frac"] = float((~keep).mean())
    print("step", step, res)
    for c in (g, g_solve, g_stab):
        c.close()
    for k, val in res.items():
        if not k.endswith("frac"):
            assert val <= 1e-4, (k, res)
    # single passes compare most of the column
    assert res["solve1_suspect_frac"] <= 0.5 and res["stab1_suspect_frac"] <= 0.5, res


def test_taped_steps_equal_recording_steps_bitwise():
    """A taped LR step (the forward keeps its recorded passes under a tag)
    gives the forward outputs and the gradients of the plain functional
    forms bit for bit; a record that was overwritten is refused
    (GS_ERR_STATE), and the checkpointed rollout with tapes gives the
    gradient of the rollout without them."""
    torch = pytest.importorskip("torch")
    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300.diff import rollout
    sc = scenes.diff_column()
    dev = torch.device("cuda")
    g = gs.Context(sc, stream="torch")
    g.set_graphs(True)
    X = torch.from_numpy(sc["lr_pos"]).to(dev)
    V = torch.from_numpy(sc["lr_vel"]).to(dev)
    dt, iters = sc["dt"], sc["iters"]
    ref_x, ref_v = torch.empty_like(X), torch.empty_like(V)
    assert gs.gs_step_low_forward(g.ctx, X.data_ptr(), V.data_ptr(), ref_x.data_ptr(), ref_v.data_ptr(), dt,
                                  iters) == 0
    g.set_step_tapes(2)
    tapes, outs = [7, 8, 9], []
    x, v = X, V
    for k in range(3):   # three taped steps in two slots: the first record is overwritten
        ox, ov = torch.empty_like(X), torch.empty_like(V)
        assert gs.gs_step_low_forward_taped(g.ctx, x.data_ptr(), v.data_ptr(), ox.data_ptr(), ov.data_ptr(), dt,
                                            iters, tapes[k]) == 0
        outs.append((x, v, ox, ov))
        x, v = ox, ov
    torch.cuda.synchronize()
    assert torch.equal(outs[0][2], ref_x) and torch.equal(outs[0][3], ref_v)
    gx_o = torch.randn_like(X)
    gx_o[:, 3] = 0
    gv_o = torch.randn_like(V)
    gv_o[:, 3] = 0
    a = [torch.empty_like(X) for _ in range(4)]
    assert gs.gs_step_low_backward_taped(g.ctx, tapes[0], gx_o.data_ptr(), gv_o.data_ptr(), a[0].data_ptr(),
                                         a[1].data_ptr()) == gs.GS_ERR_STATE
    for k in (2, 1):
        xi, vi = outs[k][0], outs[k][1]
        assert gs.gs_step_low_backward_taped(g.ctx, tapes[k], gx_o.data_ptr(), gv_o.data_ptr(), a[0].data_ptr(),
                                             a[1].data_ptr()) == 0
        assert gs.gs_step_low_backward(g.ctx, xi.data_ptr(), vi.data_ptr(), gx_o.data_ptr(), gv_o.data_ptr(),
                                       a[2].data_ptr(), a[3].data_ptr(), dt, iters) == 0
        torch.cuda.synchronize()
        assert torch.equal(a[0], a[2]) and torch.equal(a[1], a[3]), k
    # the rollout: with tapes and without (the HR backward's atomics make the
    # gradient vary in the last bits from run to run, so compare closely)
    target = torch.from_numpy(sc["target"]).to(dev)
    hx, hv = (torch.from_numpy(np.ascontiguousarray(sc[n])).to(dev) for n in ("hr_pos", "hr_vel"))

    def grad(tapes):
        Vr = V.clone().requires_grad_(True)
        out = rollout(g, X, Vr, hx, hv, dt, frames=10, n_sub=1, iters=iters, checkpoint_every=5, tapes=tapes)
        ((out[2][:, :3] - target) ** 2).sum().backward()
        return Vr.grad
    g0, g1 = grad(False), grad(True)
    rel = float((g1 - g0).norm() / g0.norm())
    assert rel < 1e-5, rel
    g.close()


@pytest.mark.parametrize("frames, every, n_sub", [(7, 3, 2), (6, 6, 1), (5, 1, 1)])
def test_native_rollout_equals_the_torch_driven_rollout(frames, every, n_sub):
    """The rollout run by the library (gs_rollout_forward / _backward) gives
    the final state of the torch-driven checkpointed rollout bit for bit and
    its gradients with respect to all four initial fields (up to the order
    of the HR backward's atomic sums); a backward after another rollout's
    forward is refused."""
    import torch

    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300.diff import rollout
    sc = scenes.column(n_low=400, ratio=8)
    g = gs.Context(sc, stream="torch")
    g.set_graphs(True)
    res = {}
    for native in (False, True):
        ins = [_t(sc[k]).requires_grad_(True) for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel")]
        out = rollout(g, *ins, DT, frames=frames, n_sub=n_sub, iters=4, checkpoint_every=every, native=native)
        loss = ((out[2][:, :3] - 0.1) ** 2).sum() + (out[1][:, :3] ** 2).sum() + (out[3][:, :3] ** 2).sum()
        loss.backward()
        res[native] = ([o.detach().cpu().numpy() for o in out], [t.grad.cpu().numpy()[:, :3] for t in ins])
    for a, b in zip(res[False][0], res[True][0]):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(res[False][1], res[True][1]):
        assert np.abs(a).max() > 0
        assert _rel(b, a) < 1e-5
    # two forwards, then the first one's backward
    ins = [_t(sc[k]).requires_grad_(True) for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel")]
    o1 = rollout(g, *ins, DT, frames=2, n_sub=1, iters=4, checkpoint_every=1)
    rollout(g, *[t.detach() for t in ins], DT, frames=2, n_sub=1, iters=4, checkpoint_every=1)
    with pytest.raises(RuntimeError):
        o1[2].sum().backward()
    g.close()


def test_native_rollout_of_zero_frames_is_the_identity():
    import torch

    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300.diff import rollout
    sc = scenes.column(n_low=400, ratio=8)
    g = gs.Context(sc, stream="torch")
    ins = [_t(sc[k]).requires_grad_(True) for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel")]
    out = rollout(g, *ins, DT, frames=0, n_sub=1, iters=4, checkpoint_every=3)
    for a, b in zip(out, ins):
        assert torch.equal(a, b.detach())
    sum(o[:, :3].sum() for o in out).backward()
    for t in ins:
        assert torch.equal(t.grad[:, :3], torch.ones_like(t.grad[:, :3]))
    g.close()


def test_deterministic_hr_backward_repeats_bitwise_and_matches_the_atomic_sums():
    """The HR frame's reverse mode with the LR side gathered per LR particle
    gives the same bits on every call, also in a rollout; with float atomics
    (the default) the LR gradients agree within the rounding of a different
    summation order."""
    torch = pytest.importorskip("torch")
    import paper_2308_01629_gb300 as gs
    sc = scenes.stir(scenes.column(n_low=2000, ratio=16), seed=5)
    dev = torch.device("cuda")
    g = gs.Context(sc, stream="torch")
    g.set_deterministic_backward(True)
    X, V, x, v = (torch.from_numpy(np.ascontiguousarray(sc[k])).to(dev) for k in ("lr_pos", "lr_vel", "hr_pos",
                                                                                     "hr_vel"))
    gen = torch.Generator(device="cpu").manual_seed(3)
    gxo = torch.randn(x.shape, generator=gen).to(dev)
    gvo = torch.randn(v.shape, generator=gen).to(dev)

    def backward():
        out = [torch.empty_like(t) for t in (X, V, x, v)]
        assert gs.gs_upsample_backward(g.ctx, X.data_ptr(), V.data_ptr(), x.data_ptr(), v.data_ptr(),
                                       gxo.data_ptr(), gvo.data_ptr(), *[t.data_ptr() for t in out], DT) == 0
        torch.cuda.synchronize()
        return [t.cpu().numpy()[:, :3] for t in out]
    det = [backward() for _ in range(3)]
    for r in det[1:]:
        for a, b in zip(det[0], r):
            np.testing.assert_array_equal(a, b)
    g.set_deterministic_backward(False)
    atom = backward()
    for a, b in zip(det[0], atom):
        assert np.abs(a).max() > 0
        assert _rel(b, a) < 1e-5
    # a whole rollout's gradient repeats bitwise
    from paper_2308_01629_gb300.diff import rollout
    g.set_deterministic_backward(True)
    grads = []
    for _ in range(2):
        Vr = V.clone().requires_grad_(True)
        out = rollout(g, X, Vr, x, v, DT, frames=4, n_sub=1, iters=4, checkpoint_every=2)
        (out[2][:, :3] ** 2).sum().backward()
        grads.append(Vr.grad.cpu().numpy())
    np.testing.assert_array_equal(grads[0], grads[1])
    g.close()
