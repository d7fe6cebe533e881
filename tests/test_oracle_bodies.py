"""Pins of shape matching (Sec. 3: a rigid body's particles are treated as
free particles, then a shape-matching constraint moves each towards the
rigidly transformed rest shape, R xo + c, with R from the polar decomposition
of C = sum m (xt - c) xo^T and c the centre of mass; counted once in the
Jacobi average)."""
import numpy as np
import pytest

from test_oracle_pins import BIG_BOX, pb_prm


def _svd_rotation(C):
    U, _, Vt = np.linalg.svd(C)
    d = np.sign(np.linalg.det(U @ Vt))
    return U @ np.diag([1.0, 1.0, d]) @ Vt


def _rot(axis, angle):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def test_polar_rotation_is_the_closest_rotation(orc):
    rng = np.random.default_rng(11)
    for _ in range(50):
        C = rng.normal(size=(3, 3))
        R = orc.polar_rotation(C)
        np.testing.assert_allclose(R, _svd_rotation(C), atol=1e-10)   # errors scale with 1 / sigma_min
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-10)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-10)
    # C = R0 S with S symmetric positive definite gives R0
    R0 = _rot((1.0, 2.0, -0.5), 0.7)
    S = np.array([[2.0, 0.3, 0.1], [0.3, 1.0, -0.2], [0.1, -0.2, 0.5]])
    np.testing.assert_allclose(orc.polar_rotation(R0 @ S), R0, atol=1e-13)


def _body(r, n=3, spacing=3.0):
    """A 3 x 3 x 3 cluster of particles 3 r apart (no contacts) around 1 m."""
    g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(float)
    return 1.0 + (g - (n - 1) / 2.0) * spacing * r


def test_shape_matching_makes_a_deformed_body_rigid(orc):
    # rest shape xr, unequal masses; the predicted positions are a rotated,
    # moved and noisily deformed copy; one solver pass with no other
    # constraint moves every particle onto R xo + c
    r, dt = 0.0625, 1.0 / 64.0
    rng = np.random.default_rng(12)
    xr = _body(r)
    n = len(xr)
    im = rng.uniform(0.5, 2.0, n)
    body = np.ones(n, np.int32)
    xo = orc.body_rest_offsets(xr, im, body)
    R0 = _rot((0.3, -1.0, 0.4), 0.5)
    target = (xr - xr.mean(0)) @ R0.T + np.array([1.1, 0.9, 1.05]) + rng.normal(0, 0.1 * r, (n, 3))
    v = (target - xr) / dt
    x1, v1, _, _ = orc.pbd_step(xr, v, im, BIG_BOX, pb_prm(r=r, dt=dt, g=(0, 0, 0), n_stab=0, iters=1),
                                bodies=(body, xo))
    xt = xr + dt * v   # the predicted positions the pass starts from
    m = 1.0 / im
    c = (m[:, None] * xt).sum(0) / m.sum()
    R = _svd_rotation(((xt - c) * m[:, None]).T @ xo)
    np.testing.assert_allclose(x1, xo @ R.T + c, atol=1e-12)
    # rigid: every pairwise distance is the rest distance
    d1 = np.linalg.norm(x1[:, None] - x1[None], axis=2)
    d0 = np.linalg.norm(xr[:, None] - xr[None], axis=2)
    np.testing.assert_allclose(d1, d0, atol=1e-12)
    # the mass-weighted centre is that of the predicted positions
    np.testing.assert_allclose((m[:, None] * x1).sum(0) / m.sum(), c, atol=1e-13)


def test_rigidly_moved_body_is_a_fixed_point(orc):
    r, dt = 0.0625, 1.0 / 64.0
    xr = _body(r)
    n = len(xr)
    im = np.linspace(0.5, 2.0, n)
    body = np.ones(n, np.int32)
    xo = orc.body_rest_offsets(xr, im, body)
    m = 1.0 / im
    cr = (m[:, None] * xr).sum(0) / m.sum()
    R0 = _rot((1.0, 1.0, 0.0), 0.9)
    target = (xr - cr) @ R0.T + cr + np.array([0.01, -0.02, 0.03])
    v = (target - xr) / dt
    x1, v1, _, _ = orc.pbd_step(xr, v, im, BIG_BOX, pb_prm(r=r, dt=dt, g=(0, 0, 0), n_stab=0, iters=3),
                                bodies=(body, xo))
    np.testing.assert_allclose(x1, xr + dt * v, atol=1e-13)
    np.testing.assert_allclose(v1, v, atol=1e-10)


def test_grain_pushes_a_body_which_stays_rigid(orc):
    # two-way coupling: a grain sliding into a resting body moves it, and the
    # body keeps its shape
    r, dt = 0.0625, 1.0 / 64.0
    xr = _body(r, spacing=2.0)   # touching particles: contacts inside the body too
    n = len(xr)
    grain = np.array([[xr[:, 0].min() - 2 * r + 0.2 * r, 1.0, 1.0]])
    x = np.vstack([xr, grain])
    v = np.zeros_like(x)
    v[-1, 0] = 2.0
    im = np.r_[np.full(n, 1.0), 1.0]
    body = np.r_[np.ones(n, np.int32), 0]
    xo = orc.body_rest_offsets(x, im, body)
    for _ in range(3):
        x, v, _, _ = orc.pbd_step(x, v, im, BIG_BOX, pb_prm(r=r, dt=dt, g=(0, 0, 0), n_stab=2, iters=6),
                                  bodies=(body, xo))
    vb = v[:n].mean(0)
    assert vb[0] > 0.01 and v[-1, 0] < 2.0
    d1 = np.linalg.norm(x[:n, None] - x[None, :n], axis=2)
    d0 = np.linalg.norm(xr[:, None] - xr[None], axis=2)
    assert np.abs(d1 - d0).max() < 0.05 * r
