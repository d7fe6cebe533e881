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
