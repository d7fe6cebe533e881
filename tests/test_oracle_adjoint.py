"""Pins of the oracle's reverse-mode HR frame against central finite
differences of its own forward map (double precision).  Inputs are drawn so
no branch decision (blend case, largest weight, wall contact) lies within the
finite-difference step of its threshold; walls are planar, where the fixed-
normal derivative of the SDF rule is exact."""
import numpy as np
import pytest

import scenes
from gs_testutil import diff_prms

EPS = 1e-7


def small_state(seed):
    sc = scenes.stir(scenes.cube(n_side=4, ratio=6), seed=seed, spread=0.6)
    box = scenes.box_interior((0.2, 0.2, 0.15), (0.4, 0.4, 0.45))
    hr = sc["hr_pos"][:, :3].astype(float)
    rng = np.random.default_rng(seed)
    # a few HR particles just outside the walls, moving outwards
    hr[:8, 0] = 0.2 + rng.uniform(-0.004, 0.001, 8)
    prm = dict(r_low=sc["r_low"], r_high=0.004, dt=1.0 / 60.0, gx=0.0, gy=0.0, gz=-9.81, c1=512.0 / 729.0,
               c2=0.6, eps_w=1e-4, eps_x=1e-6)
    return (sc["lr_pos"][:, :3].astype(float), sc["lr_vel"][:, :3].astype(float), hr,
            sc["hr_vel"][:, :3].astype(float), scenes.sdf_table([box]), prm)


@pytest.mark.parametrize("seed", [1, 2])
def test_upsample_vjp_matches_central_differences(orc, seed):
    X, V, x, v, sdf, prm = small_state(seed)
    rng = np.random.default_rng(100 + seed)
    base = orc.upsample(X, V, x, v, sdf, prm)
    keep = base["flag"] == 0
    a = rng.normal(size=x.shape) * keep[:, None]
    b = rng.normal(size=v.shape) * keep[:, None]

    def loss(X_, V_, x_, v_):
        o = orc.upsample(X_, V_, x_, v_, sdf, prm)
        assert np.array_equal(o["flag"] == 0, keep)
        return float((a * o["x"]).sum() + (b * o["v"]).sum())

    gX, gV, gx, gv = orc.upsample_vjp(X, V, x, v, sdf, prm, a, b)
    assert np.abs(gX).max() > 0 and np.abs(gV).max() > 0
    for arr, grad, which in ((X, gX, 0), (V, gV, 1), (x, gx, 2), (v, gv, 3)):
        idx = rng.choice(arr.size, size=min(arr.size, 120), replace=False)
        fd = np.zeros(len(idx))
        for n, k in enumerate(idx):
            args_p = [X.copy(), V.copy(), x.copy(), v.copy()]
            args_m = [X.copy(), V.copy(), x.copy(), v.copy()]
            args_p[which].flat[k] += EPS
            args_m[which].flat[k] -= EPS
            fd[n] = (loss(*args_p) - loss(*args_m)) / (2 * EPS)
        an = grad.flat[idx]
        scale = np.abs(fd).max() + 1e-12
        assert np.abs(an - fd).max() <= 2e-6 * scale + 1e-9, (which, np.abs(an - fd).max(), scale)


def test_vjp_of_isolated_particle_is_ballistic(orc):
    # alpha = 1 and no LR in reach: x' = x + dt (v + dt g) -> dL/dx = a, dL/dv = dt a + b
    X = np.array([[5.0, 5.0, 5.0]])
    V = np.zeros((1, 3))
    x = np.array([[0.1, 0.2, 0.3]])
    v = np.array([[0.3, -0.2, 0.1]])
    prm = dict(r_low=0.01, r_high=0.004, dt=0.02, gx=0, gy=0, gz=-9.81, c1=512 / 729, c2=0.6, eps_w=1e-4,
               eps_x=1e-6)
    a, b = np.array([[1.0, 2.0, 3.0]]), np.array([[-1.0, 0.5, 0.25]])
    gX, gV, gx, gv = orc.upsample_vjp(X, V, x, v, None, prm, a, b)
    np.testing.assert_allclose(gx, a, atol=1e-15)
    np.testing.assert_allclose(gv, 0.02 * a + b, atol=1e-15)
    np.testing.assert_array_equal(gX, 0)
    np.testing.assert_array_equal(gV, 0)


def _pb(r, dt=1.0 / 240.0, g=(0.0, 0.0, -9.81), mu=(0.35, 0.30), n_stab=2, iters=4, mass_k=0.0, mode=0):
    return dict(r=r, dt=dt, gx=g[0], gy=g[1], gz=g[2], mu_s=mu[0], mu_k=mu[1], n_stab=n_stab, iters=iters,
                mass_k=mass_k, ground_z=0.0, rc=3.0 * r, friction_mode=mode, eps_x=1e-6, eps_impact=0.0)


def _lr_cases():
    rng = np.random.default_rng(7)
    r = 0.01
    floor = scenes.sdf_table([scenes.box_interior((-1, -1, 0), (1, 1, 1))])
    cases = []
    # a small jittered cluster, falling, with overlaps in both phases
    g = np.stack(np.meshgrid(*[np.arange(3)] * 3, indexing="ij"), -1).reshape(-1, 3) * 1.9 * r
    x = g + [0.3, 0.3, 0.3] + rng.uniform(-0.1 * r, 0.1 * r, g.shape)
    v = rng.normal(0, 0.2, x.shape)
    cases.append(("cluster", x, v, floor, _pb(r, mass_k=2.0)))
    # grains on the floor sliding: kinetic (fast) and static (slow), both friction modes
    x = np.array([[0.1, 0.1, r * 0.97], [0.3, 0.1, r * 0.98], [0.5, 0.1, r * 0.99], [0.52, 0.1, r * 2.9]])
    v = np.array([[1.2, 0.3, 0.0], [0.05, -0.02, 0.0], [0.6, 0.0, -0.1], [-0.4, 0.2, 0.0]])
    cases.append(("floor_mode0", x, v, floor, _pb(r, mu=(0.35, 0.30))))
    cases.append(("floor_mode1", x, v, floor, _pb(r, mu=(0.35, 0.30), mode=1)))
    return cases


@pytest.mark.parametrize("case", [c[0] for c in _lr_cases()])
def test_pbd_step_vjp_matches_central_differences(orc, case):
    name, x, v, sdf, prm = [c for c in _lr_cases() if c[0] == case][0]
    eps = 1e-8
    im = np.ones(len(x))
    _, _, _, st = orc.pbd_step(x, v, im, sdf, prm)
    assert st["significant"] == 0, st   # no decision within reach of its threshold changes the result
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=x.shape), rng.normal(size=v.shape)

    def loss(x_, v_):
        x1, v1, _, _ = orc.pbd_step(x_, v_, im, sdf, prm)
        return float((a * x1).sum() + (b * v1).sum())

    gx, gv = orc.pbd_step_vjp(x, v, im, sdf, prm, a, b)
    for arr, grad, which in ((x, gx, 0), (v, gv, 1)):
        fd = np.zeros(arr.size)
        for k in range(arr.size):
            ap, am = [x.copy(), v.copy()], [x.copy(), v.copy()]
            ap[which].flat[k] += eps
            am[which].flat[k] -= eps
            fd[k] = (loss(*ap) - loss(*am)) / (2 * eps)
        scale = np.abs(fd).max()
        assert scale > 0
        np.testing.assert_allclose(grad.ravel(), fd, rtol=0, atol=2e-5 * scale, err_msg=f"{name} arg {which}")


def _rollout_inputs(sc):
    return (sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["lr_pos"][:, 3].astype(float), sc["hr_pos"][:, :3],
            sc["hr_vel"][:, :3], scenes.sdf_table(sc["sdfs"]))


def test_rollout_replay_reproduces_recording(orc):
    sc = scenes.diff_column(n_low=300, ratio=8)
    pb, up = diff_prms(sc)
    X, V, im, x, v, sdf = _rollout_inputs(sc)
    ro = orc.rollout(X, V, im, x, v, sdf, pb, up, 12)
    rr = orc.rollout(X, V, im, x, v, sdf, pb, up, 12, tapes=ro["tapes"])
    for k in ("lr_x", "lr_v", "hr_x", "hr_v"):
        np.testing.assert_array_equal(rr[k], ro[k])
    # the plain (untaped) step is the same function
    x1, v1, _, _ = orc.pbd_step(X, V, im, sdf, pb)
    np.testing.assert_array_equal(x1, ro["ops"][1][1])


def test_rollout_vjp_matches_frozen_central_differences(orc):
    """Gradient of a 30-step rollout loss w.r.t. every initial quantity
    against central differences (eps 1e-4) of the rollout with its decisions
    replayed from the unperturbed run."""
    sc = scenes.diff_column(n_low=400, ratio=8)
    pb, up = diff_prms(sc)
    X, V, im, x, v, sdf = _rollout_inputs(sc)
    T = sc["target"].astype(float)
    F = sc["steps"]
    ro = orc.rollout(X, V, im, x, v, sdf, pb, up, F)
    # the column lands: floor contacts are active in the last LR steps
    assert ro["lr_x"][:, 2].min() < pb["r"]
    gX, gV, gx, gv = orc.rollout_vjp(ro, im, sdf, pb, up, 2.0 * (ro["hr_x"] - T), np.zeros_like(T))
    rng = np.random.default_rng(17)
    base = [np.asarray(a, float) for a in (X, V, x, v)]
    for which, grad in enumerate((gX, gV, gx, gv)):
        d = rng.normal(size=base[which].shape)
        # velocities: the step of the differentiation workload (1e-4 m/s,
        # about 1e-5 m of displacement over the rollout); positions: a step
        # on the same displacement scale
        eps = 1e-4 if which in (1, 3) else 1e-6

        def loss(s):
            args = [a.copy() for a in base]
            args[which] = args[which] + s * d
            out = orc.rollout(args[0], args[1], im, args[2], args[3], sdf, pb, up, F, tapes=ro["tapes"])
            return float(((out["hr_x"] - T) ** 2).sum())

        fd = (loss(eps) - loss(-eps)) / (2 * eps)
        an = float((grad * d).sum())
        assert abs(an - fd) <= 1e-3 * abs(fd), (which, an, fd)


def test_rollout_vjp_with_foreign_tapes_matches_their_replay(orc):
    """Reverse modes that take every decision from a tape recorded at another
    state (the GPU's decisions, in the end-to-end check) are the derivative
    of the rollout replayed from that tape: pinned against central
    differences of the replay.  The tapes come from a run whose initial
    velocities differ by 1e-2 m/s, so many of their decisions differ from
    the replayed run's own, and the untaped reverse mode gives another
    gradient."""
    sc = scenes.diff_column(n_low=400, ratio=8)
    pb, up = diff_prms(sc)
    X, V, im, x, v, sdf = _rollout_inputs(sc)
    T = sc["target"].astype(float)
    F = 12
    rng = np.random.default_rng(29)
    V0 = np.asarray(V, float)
    Vb = V0 + rng.normal(0.0, 1e-2, V0.shape)
    ro_a = orc.rollout(X, V0, im, x, v, sdf, pb, up, F)
    ro_b = orc.rollout(X, Vb, im, x, v, sdf, pb, up, F, tapes=ro_a["tapes"])
    own_b = orc.rollout(X, Vb, im, x, v, sdf, pb, up, F)
    differ = sum(int(np.count_nonzero(np.asarray(p) != np.asarray(q))) for p, q in
                 zip(ro_a["tapes"], own_b["tapes"]) if np.asarray(p).shape == np.asarray(q).shape)
    assert differ > 0
    g = 2.0 * (ro_b["hr_x"] - T)
    _, gV, _, _ = orc.rollout_vjp(ro_b, im, sdf, pb, up, g, np.zeros_like(T), replay=True)
    _, gV_own, _, _ = orc.rollout_vjp(ro_b, im, sdf, pb, up, g, np.zeros_like(T))
    assert np.linalg.norm(gV - gV_own) > 1e-6 * np.linalg.norm(gV)
    for trial in range(2):
        d = rng.normal(size=V0.shape)
        eps = 1e-4

        def loss(s):
            out = orc.rollout(X, Vb + s * d, im, x, v, sdf, pb, up, F, tapes=ro_a["tapes"])
            return float(((out["hr_x"] - T) ** 2).sum())

        fd = (loss(eps) - loss(-eps)) / (2 * eps)
        an = float((gV * d).sum())
        assert abs(an - fd) <= 1e-5 * abs(fd), (trial, an, fd)
