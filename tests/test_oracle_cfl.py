"""Pins of the CFL-limited LR substeps of a frame (Sec. 5.2: a default LR
time step, shortened by the CFL condition when needed, and one HR frame of
1/60 s over several LR steps): the split of a slow frame, uniform motion and
free fall in closed form, the CFL bound at every step, and the cap on the
number of steps."""
import numpy as np
import pytest

import scenes
from test_oracle_pins import pb_prm

BOX = scenes.sdf_table([scenes.box_interior((-100.0, -100.0, -100.0), (100.0, 100.0, 100.0))])
T = np.float32(1.0 / 60.0)
ULP = float(np.spacing(T))


def _frame(orc, x, v, r, g, dt_max=0.005, cfl=0.4, max_sub=64):
    prm = pb_prm(r=r, g=g, n_stab=2, iters=4)
    return orc.frame_adaptive(x, v, [1.0] * len(x), BOX, prm, T, dt_max, cfl, max_sub)


def test_slow_frame_takes_the_default_step(orc):
    # 1/60 s frame, default 0.005 s (Sec. 5.2): ceil(3.33) = 4 steps of 1/240 s
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    x1, v1, dts = _frame(orc, x, np.zeros((2, 3)), 0.01, (0.0, 0.0, 0.0))
    assert len(dts) == 4
    np.testing.assert_allclose(dts.astype(float), 1.0 / 240.0, rtol=1e-6)
    assert abs(dts.astype(float).sum() - float(T)) <= 4 * ULP
    np.testing.assert_array_equal(x1, x)
    np.testing.assert_array_equal(v1, 0.0)


def test_uniform_motion_closed_form(orc):
    # |v| = 2 m/s, r = 0.01: dt <= 0.4 * 0.02 / 2 = 0.004 s -> ceil(4.17) = 5 steps;
    # without forces or contacts x moves by v * (sum of steps) = v T
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    v = np.array([[2.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    x1, v1, dts = _frame(orc, x, v, 0.01, (0.0, 0.0, 0.0))
    assert len(dts) == 5 and np.all(dts.astype(float) <= 0.004 * (1 + 1e-6))
    s = dts.astype(float).sum()
    assert abs(s - float(T)) <= 5 * ULP
    np.testing.assert_allclose(x1, x + v * s, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(v1, v)


def test_free_fall_obeys_the_bound_and_is_exact_in_total_time(orc):
    # falling at 3 m/s and faster with r = 0.005: the CFL bound decides every
    # step; symplectic Euler gives v = v0 + g (sum of steps) whatever the split
    r, g = 0.005, (0.0, 0.0, -9.81)
    x = np.array([[0.0, 0.0, 0.0]])
    v0 = np.array([[0.0, 0.0, -3.0]])
    x1, v1, dts = _frame(orc, x, v0, r, g)
    d = dts.astype(float)
    assert abs(d.sum() - float(T)) <= len(d) * ULP
    np.testing.assert_allclose(v1[0], [0.0, 0.0, -3.0 - 9.81 * d.sum()], rtol=0, atol=1e-12)
    speed = 3.0 + 9.81 * np.concatenate([[0.0], np.cumsum(d)[:-1]])   # |v| at each step's start
    assert np.all(d <= 0.4 * 2 * r / speed * (1 + 1e-6)) and np.all(d <= 0.005)
    # the fewest steps: one fewer would break the bound at the first decision
    assert len(d) >= np.ceil(float(T) / (0.4 * 2 * r / 3.0) - 1e-6)
    assert 12 <= len(d) <= 20


def test_step_count_is_capped(orc):
    # 1000 m/s asks for thousands of steps; max_sub = 16 caps the frame at 16
    x = np.array([[0.0, 0.0, 0.0]])
    v = np.array([[1000.0, 0.0, 0.0]])
    x1, v1, dts = _frame(orc, x, v, 0.01, (0.0, 0.0, 0.0), max_sub=16)
    assert len(dts) == 16
    assert abs(dts.astype(float).sum() - float(T)) <= 16 * ULP
    np.testing.assert_allclose(x1[0, 0], 1000.0 * dts.astype(float).sum(), rtol=1e-12)


def test_cfl_rate_is_the_largest_speed_over_diameter(orc):
    rng = np.random.default_rng(3)
    v = rng.normal(0.0, 2.0, size=(1000, 3)).astype(np.float32)
    r = rng.uniform(0.005, 0.02, size=1000).astype(np.float32)
    want = (np.linalg.norm(v.astype(float), axis=1) / (2.0 * r.astype(float))).max()
    assert orc.cfl_rate(v, r) == pytest.approx(want, rel=1e-6)
    assert orc.cfl_rate(np.zeros((0, 3)), 0.01) == 0.0


@pytest.mark.parametrize("rate,left,expect_n", [(0.0, 64, 4), (10.0, 64, 4), (500.0, 64, 21), (1e9, 8, 8),
                                                (np.inf, 8, 8), (np.nan, 3, 3), (0.0, 1, 1)])
def test_substep_decision_cases(orc, rate, left, expect_n):
    # n equal steps: 0.005 default -> 4, also when the CFL limit is looser (rate 10/s: 0.04 s);
    # rate 500/s -> limit 0.4/500 = 0.0008 s -> ceil(20.8) = 21;
    # too fast or not finite -> every allowed step; one step left -> the rest of the frame
    dt, more = orc.cfl_substep(T, rate, 0.005, 0.4, left)
    assert more == (expect_n > 1)
    assert float(dt) == pytest.approx(float(T) / expect_n, rel=1e-6)
