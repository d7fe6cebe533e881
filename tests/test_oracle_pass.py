"""Pins of the oracle's single Jacobi pass (Algorithm 1, Sec. 3), the
reference of the pass-by-pass GPU comparison.

The pass is checked against closed forms (one stabilization pass separates
an overlap by the mass ratios; one solver pass of three grains in a row
averages each grain's corrections over its n_i) and against the whole step:
chaining one pass per iteration from the step's predictions reproduces the
step, and its marks are those of this pass's own near-threshold decisions."""
import math

import numpy as np
import pytest

import scenes

BIG_BOX = scenes.sdf_table([scenes.box_interior((-10.0, -10.0, 0.0), (10.0, 10.0, 10.0))])


def pb_prm(r=0.0625, dt=1.0 / 16.0, g=(0.0, 0.0, -8.0), mu_s=0.35, mu_k=0.30, n_stab=2, iters=4, mass_k=0.0,
           ground_z=0.0, eps_x=1e-12, eps_impact=1e-12):
    return dict(r=r, dt=dt, gx=g[0], gy=g[1], gz=g[2], mu_s=mu_s, mu_k=mu_k, n_stab=n_stab, iters=iters,
                mass_k=mass_k, ground_z=ground_z, rc=3.0 * r, friction_mode=0, eps_x=eps_x, eps_impact=eps_impact)


def test_stabilization_pass_separates_by_mass_ratio(orc):
    # Eqs. 1-2 with m^-1 = 1 and 3 (height scaling off): the overlap d is
    # shared 1/4 : 3/4 and applied to x and x~ alike
    r, d = 0.0625, 0.015625
    x = np.array([[1.0, 1.0, 1.0], [1.0 + 2 * r - d, 1.0, 1.0]])
    xt = x + np.array([[0.0, 0.0, -0.001], [0.0, 0.0, -0.001]])
    x1, xt1, sus, st = orc.pbd_pass(x, xt, x, xt, [1.0, 3.0], BIG_BOX, pb_prm(r=r), stab=True)
    assert x1[0, 0] == pytest.approx(1.0 - 0.25 * d, abs=1e-15)
    assert x1[1, 0] == pytest.approx(1.0 + 2 * r - d + 0.75 * d, abs=1e-15)
    np.testing.assert_allclose(xt1 - xt, x1 - x, atol=1e-15)
    assert st["active"] == 1 and not sus.any()


def test_solver_pass_averages_over_constraint_count(orc):
    # three grains in a row on x~ (x at rest): the middle one has two
    # contacts, so its correction is the mean of its two pair terms
    r, d1, d2 = 0.0625, 0.015625, 0.0078125
    xt = np.array([[1.0, 1, 1], [1.0 + 2 * r - d1, 1, 1], [1.0 + 4 * r - d1 - d2, 1, 1]])
    x1, xt1, _, st = orc.pbd_pass(xt, xt, xt, xt, [1.0] * 3, BIG_BOX, pb_prm(r=r), stab=False)
    np.testing.assert_allclose(xt1[:, 0] - xt[:, 0], [-d1 / 2, (d1 / 2 - d2 / 2) / 2, d2 / 2], atol=1e-15)
    np.testing.assert_array_equal(x1, xt)   # a solver pass leaves x alone
    assert st["active"] == 2


def test_height_scaled_masses_come_from_the_step_start(orc):
    # m* = m e^{-k (z - ground)} at x0, the start of the step, not at the
    # pass's input: moving the input up does not change the shares
    r, d, k = 0.0625, 0.015625, 2.0
    x0 = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0 + 2 * r]])
    x = x0.copy()
    x[1, 2] -= d
    x += [0.0, 0.0, 0.5]
    x1, _, _, _ = orc.pbd_pass(x, x, x0, x0, [1.0, 1.0], BIG_BOX, pb_prm(r=r, mass_k=k), stab=True)
    w0, w1 = math.exp(k * x0[0, 2]), math.exp(k * x0[1, 2])
    assert x1[0, 2] - x[0, 2] == pytest.approx(-d * w0 / (w0 + w1), abs=1e-14)
    assert x1[1, 2] - x[1, 2] == pytest.approx(d * w1 / (w0 + w1), abs=1e-14)


@pytest.mark.parametrize("make", [lambda: scenes.stir(scenes.cube(), seed=3, v_scale=0.3),
                                  lambda: scenes.stir(scenes.cube(seed=scenes.SEED_BASE + 77), seed=4, v_scale=0.5)])
def test_chained_passes_are_the_step(orc, make):
    # one pass per iteration from the step's predictions (a step with no
    # pass returns them as x) gives the step's x and v bit for bit
    sc = make()
    r = float(sc["r_low"])
    prm = dict(r=r, dt=1.0 / 240.0, gx=0.0, gy=0.0, gz=-9.81, mu_s=0.35, mu_k=0.30, n_stab=2, iters=6, mass_k=1.0,
               ground_z=float(sc["box_lo"][2]), rc=3.0 * r, friction_mode=0, eps_x=1e-7, eps_impact=1e-9)
    x0, v0, inv_m = sc["lr_pos"][:, :3].astype(float), sc["lr_vel"][:, :3].astype(float), sc["lr_pos"][:, 3]
    sdf = scenes.sdf_table(sc["sdfs"])
    xt0, _, _, _ = orc.pbd_step(x0, v0, inv_m, sdf, dict(prm, n_stab=0, iters=0), mode=1)
    x, xt = x0.copy(), xt0.copy()
    for k in range(prm["n_stab"] + prm["iters"]):
        x, xt, _, _ = orc.pbd_pass(x, xt, x0, xt0, inv_m, sdf, prm, stab=k < prm["n_stab"])
    rx, rv, _, st = orc.pbd_step(x0, v0, inv_m, sdf, prm, mode=1)
    assert st["active"] > 0
    np.testing.assert_array_equal(xt, rx)
    np.testing.assert_array_equal((xt - x) / prm["dt"], rv)


def test_marks_are_this_pass_decisions(orc):
    # a pair 0.5 eps_x beyond contact: the other branch (an active contact)
    # would move both grains by more than eps_impact, so both are marked;
    # an isolated third grain is not
    r, eps = 0.0625, 1e-9
    xt = np.array([[1.0, 1.0, 1.0], [1.0 + 2 * r + 0.5 * eps, 1.0, 1.0], [3.0, 3.0, 3.0]])
    _, xt1, sus, st = orc.pbd_pass(xt, xt, xt, xt, [1.0] * 3, BIG_BOX,
                                   pb_prm(r=r, eps_x=eps, eps_impact=1e-12), stab=False)
    np.testing.assert_array_equal(sus, [True, True, False])
    np.testing.assert_array_equal(xt1, xt)   # the primary branch: no contact
    assert st["active"] == 0 and st["ambiguous"] >= 2
