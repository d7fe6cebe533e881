"""The oracle's plain definitions of the LR step (Algorithm 1) and the HR
frame (Sec. 4) -- written as the paper states them, without decision margins
or tapes, each particle gathering its own sums -- equal the instrumented
oracle functions bit for bit (which carry the closed-form pins), on scenes
with every SDF kind (box interior, cone shell, moving solid box), both
friction threshold readings, several chained steps, and any thread count."""
import numpy as np
import pytest

import scenes


def _pb(sc, dt, friction_mode=0, iters=None):
    r, g = sc["r_low"], sc["gravity"]
    return dict(r=r, dt=dt, gx=g[0], gy=g[1], gz=g[2], mu_s=sc["mu_s"], mu_k=sc["mu_k"], n_stab=2,
                iters=sc["iters"] if iters is None else iters, mass_k=1.0, ground_z=sc["box_lo"][2], rc=3 * r,
                friction_mode=friction_mode, eps_x=1e-7, eps_impact=1e-9)


def _up(sc, dt):
    g = sc["gravity"]
    return dict(r_low=sc["r_low"], r_high=sc["r_high"], dt=dt, gx=g[0], gy=g[1], gz=g[2], c1=512 / 729, c2=0.6,
                eps_w=1e-4, eps_x=2e-6)


def _cases():
    dig = scenes.digging(size=0.3)
    fun = scenes.funnel(n_low=3000)
    cube = scenes.cube(n_side=8)
    return [("digging+bucket", dig, scenes.sdf_table(dig["sdfs"] + [scenes.bucket_sdf(0.2)])),
            ("funnel", fun, scenes.sdf_table(fun["sdfs"])),
            ("cube", cube, scenes.sdf_table(cube["sdfs"]))]


@pytest.mark.parametrize("friction_mode", [0, 1])
def test_plain_lr_steps_equal_the_instrumented_step(orc, friction_mode):
    for name, sc, sdf in _cases():
        x, v, im = sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["lr_pos"][:, 3]
        prm = _pb(sc, 1.0 / 240.0, friction_mode)
        xa, va, xb, vb = x, v, x, v
        for step in range(3):
            xa, va, _, _ = orc.pbd_step(xa, va, im, sdf, prm, mode=1)
            xb, vb = orc.pbd_step_plain(xb, vb, im, sdf, prm)
            np.testing.assert_array_equal(xb, xa, err_msg=f"{name} step {step}")
            np.testing.assert_array_equal(vb, va, err_msg=f"{name} step {step}")
        assert not np.array_equal(xa, x)   # the steps moved the particles


def test_plain_lr_step_equals_the_brute_force_pairs(orc):
    sc = scenes.cube(n_side=8)
    sdf = scenes.sdf_table(sc["sdfs"])
    x, v, im = sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["lr_pos"][:, 3]
    prm = _pb(sc, 1.0 / 60.0)
    xa, va, _, _ = orc.pbd_step(x, v, im, sdf, prm, mode=0)
    xb, vb = orc.pbd_step_plain(x, v, im, sdf, prm)
    np.testing.assert_array_equal(xb, xa)
    np.testing.assert_array_equal(vb, va)


def test_plain_hr_frame_equals_the_instrumented_frame(orc):
    for name, sc, sdf in _cases():
        lr_x, lr_v = sc["lr_pos"][:, :3], sc["lr_vel"][:, :3] + np.array([0.03, -0.02, 0.05])
        n = min(len(sc["hr_pos"]), 30000)
        hr_x, hr_v = sc["hr_pos"][:n, :3], sc["hr_vel"][:n, :3]
        prm = _up(sc, 1.0 / 60.0)
        ref = orc.upsample(lr_x, lr_v, hr_x, hr_v, sdf, prm, mode=1)
        x, v = orc.upsample_plain(lr_x, lr_v, hr_x, hr_v, sdf, prm)
        np.testing.assert_array_equal(x, ref["x"], err_msg=name)
        np.testing.assert_array_equal(v, ref["v"], err_msg=name)
        brute = orc.upsample(lr_x, lr_v, hr_x[:2000], hr_v[:2000], sdf, prm, mode=0)   # the sum over every LR
        np.testing.assert_array_equal(x[:2000], brute["x"], err_msg=name)


def test_plain_definitions_do_not_depend_on_the_thread_count(orc):
    sc = scenes.digging(size=0.3)
    sdf = scenes.sdf_table(sc["sdfs"] + [scenes.bucket_sdf(0.2)])
    x, v, im = sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["lr_pos"][:, 3]
    hr_x, hr_v = sc["hr_pos"][:20000, :3], sc["hr_vel"][:20000, :3]
    out = []
    for threads in (1, 3, max(2, orc.max_threads())):
        orc.set_threads(threads)
        xs, vs = orc.pbd_step_plain(x, v, im, sdf, _pb(sc, 1.0 / 240.0))
        out.append((xs, vs) + orc.upsample_plain(xs, vs, hr_x, hr_v, sdf, _up(sc, 1.0 / 60.0)))
    orc.set_threads(1)
    for o in out[1:]:
        for a, b in zip(o, out[0]):
            np.testing.assert_array_equal(a, b)


def test_plain_definitions_of_empty_sets(orc):
    sc = scenes.cube(n_side=4)
    sdf = scenes.sdf_table(sc["sdfs"])
    x, v = orc.pbd_step_plain(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), sdf, _pb(sc, 0.01))
    assert x.shape == (0, 3) and v.shape == (0, 3)
    hx, hv = sc["hr_pos"][:50, :3], sc["hr_vel"][:50, :3]
    ox, ov = orc.upsample_plain(np.zeros((0, 3)), np.zeros((0, 3)), hx, hv, sdf, _up(sc, 0.01))
    ref = orc.upsample(np.zeros((0, 3)), np.zeros((0, 3)), hx, hv, sdf, _up(sc, 0.01), mode=0)
    np.testing.assert_array_equal(ox, ref["x"])   # no LR in reach: alpha = 1, ballistic + boundary
    np.testing.assert_array_equal(ov, ref["v"])
