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


def test_rollout_gradient_config4_matches_oracle(orc):
    """Falling column, 4k LR / 64k HR, 30 steps, checkpoints every 5: the GPU
    gradient of the loss w.r.t. the initial LR velocities against the oracle.

    The oracle's analytic gradient equals central differences (eps 1e-4) of
    its decision-replayed rollout to 1e-6.  The float32 rollout follows a
    different smooth piece of the method: resting contacts sit at
    |x_ij| = 2 r_LR, where the contact test is decided by rounding, and an
    active contact at zero penetration still contributes the rank-one
    Jacobian -u u^T and changes n_i.  The end-to-end difference is therefore
    bounded by what those decisions move (measured: 2.4e-2 on the directional
    derivative, 8e-2 in L2), not by the kernels, which match the oracle per
    operation at the same states (test_stepwise_reverse_along_config4_trajectory)."""
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
    ro = orc.rollout(X0, V0, im, x0, v0, sdf, pb, up, sc["steps"])
    _, gv_or, _, _ = orc.rollout_vjp(ro, im, sdf, pb, up, 2.0 * (ro["hr_x"] - T), np.zeros_like(T))
    rng = np.random.default_rng(23)
    d = rng.normal(size=V0.shape)
    eps = 1e-4
    lp = ((orc.rollout(X0, V0 + eps * d, im, x0, v0, sdf, pb, up, sc["steps"], tapes=ro["tapes"])["hr_x"] - T) ** 2)
    lm = ((orc.rollout(X0, V0 - eps * d, im, x0, v0, sdf, pb, up, sc["steps"], tapes=ro["tapes"])["hr_x"] - T) ** 2)
    fd = (lp.sum() - lm.sum()) / (2 * eps)
    # the oracle's own reverse mode along the GPU's float32 trajectory
    ops, Xg, Vg, xg = _gpu_forward_states(g, sc)
    ops = [(o[0],) + tuple(_f64(t) for t in o[1:]) for o in ops]
    _, gv_along, _, _ = orc.rollout_vjp(dict(ops=ops, lr_x=_f64(Xg), lr_v=_f64(Vg)), im, sdf, pb, up,
                                        2.0 * (_f64(xg) - T), np.zeros_like(T))
    dir_gpu = float((gv_gpu * d).sum())
    report = dict(fd=fd, dir_gpu=dir_gpu, dir_oracle=float((gv_or * d).sum()),
                  rel_dir_fd=abs(dir_gpu - fd) / abs(fd), rel_l2_oracle=_rel(gv_gpu, gv_or),
                  rel_l2_along=_rel(gv_gpu, gv_along), norm=float(np.linalg.norm(gv_or)))
    report["rel_oracle_fd"] = abs(report["dir_oracle"] - fd) / abs(fd)
    print("config4", report)
    g.close()
    assert report["rel_oracle_fd"] <= 1e-6, report
    assert report["rel_dir_fd"] <= 5e-2, report
    assert report["rel_l2_along"] <= 8e-2, report
    assert report["rel_l2_oracle"] <= 0.15, report


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
