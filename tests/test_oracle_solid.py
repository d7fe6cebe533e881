"""Pins of particle-sampled boundaries and rigid bodies (Sec. 3: objects
sampled with particles of inverse mass 0 and handled by the same contact
constraints; Sec. 4: their particles count in the HR weights, except that an
HR particle with no grain in reach ignores them so it does not stick to a
rigid body moved externally)."""
import numpy as np
import pytest

import scenes
from test_oracle_pins import BIG_BOX, pb_prm, up_prm

C1 = 512.0 / 729.0


def _w(d, r):
    return max(0.0, 1.0 - d * d / (9.0 * r * r)) ** 3


def test_solid_and_grain_weights_blend_in_closed_form(orc):
    # a grain at distance r (w = c1) and a solid particle at 0.5 r:
    # max w = (35/36)^3 > c1 and max w / sum w = 0.567 < 0.6 -> alpha = 0
    r, dt = 0.01, 1.0 / 60.0
    hr = np.array([[0.5, 0.5, 0.5]])
    lr = np.array([[0.5 + r, 0.5, 0.5], [0.5, 0.5 - 0.5 * r, 0.5]])
    lv = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 2.0]])
    out = orc.upsample(lr, lv, hr, np.zeros((1, 3)), BIG_BOX, up_prm(r_low=r, r_high=0.004, dt=dt), solid=[0, 1])
    wg, ws = _w(r, r), _w(0.5 * r, r)
    assert wg == pytest.approx(C1, rel=1e-15) and ws > C1 and ws / (wg + ws) < 0.6
    want = (wg * lv[0] + ws * lv[1]) / (wg + ws)
    np.testing.assert_allclose(out["v"][0], want, rtol=1e-13)
    np.testing.assert_allclose(out["x"][0], hr[0] + dt * want, rtol=1e-13)
    assert out["flag"][0] == 0


def test_no_grain_in_reach_ignores_solid_particles(orc):
    # the grain is beyond the 3 r support: the solid particle at 0.5 r is
    # ignored and the HR particle moves ballistically; without the solid flag
    # the same particle would drag it along
    r, dt = 0.01, 1.0 / 60.0
    hr, hv = np.array([[0.5, 0.5, 0.5]]), np.array([[0.1, 0.0, 0.0]])
    lr = np.array([[0.5 + 3.5 * r, 0.5, 0.5], [0.5, 0.5 - 0.5 * r, 0.5]])
    lv = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 2.0]])
    prm = up_prm(r_low=r, r_high=0.004, dt=dt)
    out = orc.upsample(lr, lv, hr, hv, BIG_BOX, prm, solid=[0, 1])
    g = np.array([0.0, 0.0, -9.81])
    np.testing.assert_allclose(out["v"][0], hv[0] + dt * g, rtol=1e-14)
    np.testing.assert_allclose(out["x"][0], hr[0] + dt * (hv[0] + dt * g), rtol=1e-14)
    assert out["diag"][0, 0] == 0.0 and out["flag"][0] == 0
    plain = orc.upsample(lr, lv, hr, hv, BIG_BOX, prm)
    ws = _w(0.5 * r, r)
    alpha = 1.0 - ws   # one LR particle in reach: max w / sum w = 1
    np.testing.assert_allclose(plain["v"][0], (1 - alpha) * lv[1] + alpha * (hv[0] + dt * g), rtol=1e-13)


def test_grain_at_the_edge_of_the_support_is_flagged(orc):
    r = 0.01
    hr = np.array([[0.5, 0.5, 0.5]])
    edge = 3.0 * r * np.sqrt(1.0 - 1e-7)   # t = 1e-7: inside the rule's margin
    lr = np.array([[0.5 + edge, 0.5, 0.5], [0.5, 0.5 - 0.5 * r, 0.5]])
    out = orc.upsample(lr, np.zeros((2, 3)), hr, np.zeros((1, 3)), BIG_BOX, up_prm(r_low=r, r_high=0.004),
                       solid=[0, 1])
    assert out["flag"][0] == 2
    # the primary branch: the grain's weight (1e-21) is positive, so the
    # solid particle still counts
    assert out["diag"][0, 0] == pytest.approx(_w(0.5 * r, r), rel=1e-12)


def _floor(r, n=7, z=0.0, c=(0.5, 0.5)):
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 2).astype(float)
    xy = np.asarray(c) + (g - (n - 1) / 2.0) * 2.0 * r
    return np.column_stack([xy, np.full(len(xy), z)])


def test_grain_rests_on_a_particle_floor(orc):
    # a grain on a square lattice of solid particles (spacing 2 r) under
    # gravity: it settles into the hollow between four floor particles and
    # stays; the floor does not move at all
    r, dt = 0.0625, 1.0 / 64.0
    floor = _floor(r)
    grain = np.array([[0.5 + r, 0.5 + r, np.sqrt(2.0) * r + 0.01]])
    x = np.vstack([floor, grain])
    v = np.zeros_like(x)
    im = np.r_[np.zeros(len(floor)), 1.0]
    prm = pb_prm(r=r, dt=dt, g=(0.0, 0.0, -8.0), n_stab=2, iters=8)
    for _ in range(120):
        x, v, _, _ = orc.pbd_step(x, v, im, np.zeros((0, 20)), prm)
    np.testing.assert_array_equal(x[:-1], floor)
    np.testing.assert_array_equal(v[:-1], 0.0)
    assert abs(v[-1]).max() < 1e-3
    np.testing.assert_allclose(x[-1], [0.5 + r, 0.5 + r, np.sqrt(2.0) * r], atol=2e-3 * r)


def test_moving_solid_pushes_a_grain_with_mass_ratio_one(orc):
    # a solid particle moving at u reaches a grain it touches: the predicted
    # overlap u dt goes entirely to the grain (Eqs. 1-2 with m^-1 = 0), which
    # leaves with the solid's velocity; the solid keeps its prescribed motion
    r, dt, u = 0.0625, 1.0 / 64.0, 0.5
    x = np.array([[1.0, 1.0, 1.0], [1.0 + 2 * r, 1.0, 1.0]])
    v = np.array([[u, 0.0, 0.0], [0.0, 0.0, 0.0]])
    # (no gravity: a falling grain would meet the pusher off its axis)
    x1, v1, _, _ = orc.pbd_step(x, v, [0.0, 1.0], BIG_BOX, pb_prm(r=r, dt=dt, g=(0.0, 0.0, 0.0), n_stab=2, iters=4))
    np.testing.assert_allclose(v1[0], [u, 0.0, 0.0], atol=1e-13)
    np.testing.assert_allclose(v1[1], [u, 0.0, 0.0], atol=1e-12)
    np.testing.assert_allclose(x1[1, 0] - x1[0, 0], 2 * r, atol=1e-13)


def test_solid_particles_feel_no_gravity(orc):
    x = np.array([[1.0, 1.0, 1.0]])
    x1, v1, _, _ = orc.pbd_step(x, np.zeros((1, 3)), [0.0], BIG_BOX, pb_prm())
    np.testing.assert_array_equal(x1, x)
    np.testing.assert_array_equal(v1, 0.0)
