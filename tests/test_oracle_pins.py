"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: constants
the paper prints, closed forms, textbook definitions, brute force on tiny
inputs, or invariants.  They are chosen so that a plausible slip (a dropped
term, a wrong sign, a swapped index, a missing 1/n_i) fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest

import scenes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
C1 = GOLD["c1"]["value_num"] / GOLD["c1"]["value_den"]
C2 = GOLD["c2"]["value"]


def up_prm(r_low=0.01, r_high=0.004, dt=1.0 / 60.0, g=(0.0, 0.0, -9.81), c1=C1, c2=C2, eps_w=1e-4, eps_x=1e-9):
    return dict(r_low=r_low, r_high=r_high, dt=dt, gx=g[0], gy=g[1], gz=g[2], c1=c1, c2=c2, eps_w=eps_w,
                eps_x=eps_x)


def pb_prm(r=0.0625, dt=1.0 / 16.0, g=(0.0, 0.0, -8.0), mu_s=0.35, mu_k=0.30, n_stab=2, iters=4, mass_k=0.0,
           ground_z=0.0, rc=None, friction_mode=0, eps_x=1e-12, eps_impact=1e-12):
    return dict(r=r, dt=dt, gx=g[0], gy=g[1], gz=g[2], mu_s=mu_s, mu_k=mu_k, n_stab=n_stab, iters=iters,
                mass_k=mass_k, ground_z=ground_z, rc=3.0 * r if rc is None else rc, friction_mode=friction_mode,
                eps_x=eps_x, eps_impact=eps_impact)


BIG_BOX = scenes.sdf_table([scenes.box_interior((-10.0, -10.0, 0.0), (10.0, 10.0, 10.0))])


# ------------------------------------------------------------- weights ---
def test_weight_at_r_low_is_c1(orc):
    # Sec. 4: c1 = 512/729 is the weight at a distance equal to r_LR
    for r in (0.005, 0.0089, 0.013, 0.05):
        assert orc.weight(r * r, r) == pytest.approx(C1, rel=1e-14, abs=0)


def test_weight_closed_forms(orc):
    r = 0.013
    s = GOLD["support_factor"]["value"]
    assert orc.weight(0.0, r) == 1.0
    assert orc.weight((s * r) ** 2, r) == 0.0
    assert orc.weight((s * r * 1.001) ** 2, r) == 0.0
    assert orc.weight((2 * r) ** 2, r) == pytest.approx((5.0 / 9.0) ** 3, rel=1e-14)
    d = np.linspace(0, 3 * r, 200)
    w = [orc.weight(x * x, r) for x in d]
    assert all(a > b for a, b in zip(w[:-1], w[1:]))


# ------------------------------------------------------- HR upsampling ---
def test_isolated_hr_follows_discrete_parabola(orc):
    # no LR within 3 r_LR: sum w = 0, max w = 0 <= c1, so alpha = 1 and the
    # particle moves ballistically under symplectic Euler
    dt = 1.0 / 60.0
    g = np.array([0.0, 0.0, -9.81])
    lr_x, lr_v = np.array([[10.0, 10.0, 10.0]]), np.array([[1.0, 2.0, 3.0]])
    x0, v0 = np.array([0.1, 0.2, 0.3]), np.array([0.5, -0.25, 1.0])
    x, v = x0.copy(), v0.copy()
    for n in range(1, 31):
        out = orc.upsample(lr_x, lr_v, x[None], v[None], None, up_prm(dt=dt))
        x, v = out["x"][0], out["v"][0]
        assert out["diag"][0, 2] == 1.0
        np.testing.assert_allclose(v, v0 + n * dt * g, rtol=0, atol=1e-12)
        np.testing.assert_allclose(x, x0 + n * dt * v0 + dt * dt * g * n * (n + 1) / 2, rtol=0, atol=1e-12)
        # and within dt^2 |g| n / 2 of the continuous parabola
        t = n * dt
        cont = x0 + t * v0 + 0.5 * g * t * t
        assert np.abs(x - cont).max() <= dt * dt * 9.81 * n / 2 + 1e-12


def test_lattice_site_weight_sum_and_alpha(orc):
    # HR at a site of a perfect 2r lattice: neighbours at 2r (6), 2r*sqrt2 (12),
    # 2r*sqrt3 (8, outside the support) -> closed-form sum of weights
    r = 0.01
    g = np.stack(np.meshgrid(*[np.arange(-3, 4)] * 3, indexing="ij"), -1).reshape(-1, 3) * 2 * r
    lr_v = np.tile([0.3, -0.1, 0.2], (len(g), 1))
    out = orc.upsample(g, lr_v, np.zeros((1, 3)), np.zeros((1, 3)), None, up_prm(r_low=r))
    S_ref = 1.0 + 6 * (5.0 / 9.0) ** 3 + 12 * (1.0 / 9.0) ** 3
    assert out["diag"][0, 0] == pytest.approx(S_ref, rel=1e-13)
    assert out["diag"][0, 1] == 1.0
    assert out["diag"][0, 1] / out["diag"][0, 0] < C2        # dense interior: alpha = 0
    assert out["diag"][0, 2] == 0.0
    np.testing.assert_allclose(out["v"][0], [0.3, -0.1, 0.2], rtol=0, atol=1e-14)


def test_uniform_lr_velocity_is_reproduced(orc):
    # partition of unity: a uniform LR field u gives vtilde = u wherever sum w > 0
    sc = scenes.stir(scenes.cube(), seed=7)
    r = sc["r_low"]
    lr_x = sc["lr_pos"][:, :3]
    u = np.array([0.21, -0.37, 0.05])
    lr_v = np.tile(u, (len(lr_x), 1))
    hr_x, hr_v = sc["hr_pos"][:2000, :3], sc["hr_vel"][:2000, :3]
    prm = up_prm(r_low=r)
    out = orc.upsample(lr_x, lr_v, hr_x, hr_v, None, prm)
    a = out["diag"][:, 2:3]
    dt, g = prm["dt"], np.array([0.0, 0.0, -9.81])
    expect_v = (1 - a) * u + a * (hr_v + dt * g)
    has = out["diag"][:, 0] > 0
    assert has.sum() > 1000 and (a[:, 0] == 0).sum() > 500 and ((a[:, 0] > 0) & has).sum() > 10
    np.testing.assert_allclose(out["v"][has], expect_v[has], rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["x"], hr_x + dt * out["v"], rtol=0, atol=1e-13)


def _one(orc, lr_x, lr_v, x, v, **kw):
    out = orc.upsample(np.asarray(lr_x, float), np.asarray(lr_v, float), np.asarray([x], float),
                       np.asarray([v], float), None, up_prm(**kw))
    return out


def test_alpha_single_close_lr(orc):
    r, dt = 0.01, 1.0 / 60.0
    vl, v0 = np.array([0.4, 0.1, -0.2]), np.array([0.0, 0.3, 0.0])
    out = _one(orc, [[0.5 * r, 0, 0]], [vl], [0, 0, 0], v0, r_low=r, dt=dt)
    w = (1 - 0.25 / 9) ** 3                      # max w / sum w = 1 >= c2
    a = 1 - w
    assert out["diag"][0, 2] == pytest.approx(a, rel=1e-14)
    np.testing.assert_allclose(out["v"][0], (1 - a) * vl + a * (v0 + dt * np.array([0, 0, -9.81])), atol=1e-14)


def test_alpha_two_symmetric_close(orc):
    r = 0.01
    out = _one(orc, [[0.5 * r, 0, 0], [-0.5 * r, 0, 0]], [[1.0, 0, 0], [0, 1.0, 0]], [0, 0, 0], [0, 0, 0], r_low=r)
    # ratio 1/2 < c2 and max w > c1: alpha = 0, plain average
    assert out["diag"][0, 2] == 0.0
    np.testing.assert_allclose(out["v"][0], [0.5, 0.5, 0.0], atol=1e-15)


def test_alpha_two_symmetric_far(orc):
    r = 0.01
    out = _one(orc, [[1.2 * r, 0, 0], [-1.2 * r, 0, 0]], [[1.0, 0, 0], [0, 1.0, 0]], [0, 0, 0], [0, 0, 0], r_low=r)
    w = (1 - 1.44 / 9) ** 3                      # below c1
    assert w < C1
    assert out["diag"][0, 2] == pytest.approx(1 - w, rel=1e-14)


def test_alpha_dominant_neighbour(orc):
    r = 0.01
    out = _one(orc, [[0.5 * r, 0, 0], [-2.5 * r, 0, 0]], [[1.0, 0, 0], [0, 1.0, 0]], [0, 0, 0], [0, 0, 0], r_low=r)
    w1, w2 = (1 - 0.25 / 9) ** 3, (1 - 6.25 / 9) ** 3
    assert w1 > C1 and w1 / (w1 + w2) >= C2
    assert out["diag"][0, 2] == pytest.approx(1 - w1, rel=1e-14)


def test_ambiguous_alpha_reports_other_branch(orc):
    r = 0.01
    # two LR at (almost exactly) r_LR: max w within eps of c1, ratio 1/2
    d = r * (1 + 1e-9)
    vl = [[1.0, 0, 0], [0, 1.0, 0]]
    out = _one(orc, [[d, 0, 0], [-d, 0, 0]], vl, [0, 0, 0], [0, 0, 0], r_low=r)
    assert out["flag"][0] == 1
    wm = out["diag"][0, 1]
    assert abs(wm - C1) < 1e-6
    a = out["diag"][0, 2]
    v_avg = np.array([0.5, 0.5, 0.0])
    other = v_avg if a > 0 else (1 - wm) * np.array([0, 0, -9.81]) / 60.0 + wm * v_avg
    np.testing.assert_allclose(out["alt_v"][0], other, atol=1e-12)
    clear = _one(orc, [[0.5 * r, 0, 0], [-0.5 * r, 0, 0]], vl, [0, 0, 0], [0, 0, 0], r_low=r)
    assert clear["flag"][0] == 0


def test_hr_floor_contact_rule(orc):
    rh, dt = 0.004, 1.0 / 60.0
    x0, v0 = np.array([0.5, 0.5, rh + 0.001]), np.array([0.3, -0.2, -1.0])
    out = orc.upsample(np.array([[5.0, 5, 5]]), np.zeros((1, 3)), x0[None], v0[None],
                       scenes.sdf_table([scenes.box_interior((0, 0, 0), (1, 1, 1))]), up_prm(r_high=rh, dt=dt))
    v1 = v0 + dt * np.array([0, 0, -9.81])
    x1 = x0 + dt * v1
    assert x1[2] < rh
    np.testing.assert_allclose(out["x"][0], [x1[0], x1[1], rh], atol=1e-15)
    np.testing.assert_allclose(out["v"][0], [v1[0], v1[1], 0.0], atol=1e-15)


def test_hr_outward_velocity_is_kept(orc):
    rh, dt = 0.004, 1.0 / 60.0
    x0, v0 = np.array([0.5, 0.5, 0.001]), np.array([0.1, 0.0, 0.05])   # inside the wall margin, moving out
    out = orc.upsample(np.array([[5.0, 5, 5]]), np.zeros((1, 3)), x0[None], v0[None],
                       scenes.sdf_table([scenes.box_interior((0, 0, 0), (1, 1, 1))]),
                       up_prm(r_high=rh, dt=dt, g=(0, 0, 0)))
    assert out["x"][0, 2] == pytest.approx(rh, abs=1e-15)
    np.testing.assert_allclose(out["v"][0], v0, atol=1e-15)


def test_hr_moving_bucket_normal_velocity(orc):
    rh, dt = 0.004, 1.0 / 60.0
    ub = (0.0, 0.0, 0.5)
    box = scenes.solid_box((0.5, 0.5, 0.5), (0.1, 0.1, 0.1), vel=ub)
    x0, v0 = np.array([0.52, 0.47, 0.6 + rh + 1e-4]), np.array([0.2, 0.0, -0.3])
    out = orc.upsample(np.array([[5.0, 5, 5]]), np.zeros((1, 3)), x0[None], v0[None], scenes.sdf_table([box]),
                       up_prm(r_high=rh, dt=dt, g=(0, 0, 0)))
    np.testing.assert_allclose(out["x"][0], [x0[0] + dt * 0.2, x0[1], 0.6 + rh], atol=1e-14)
    # the inward relative normal velocity is removed: v_z becomes the bucket's
    np.testing.assert_allclose(out["v"][0], [0.2, 0.0, 0.5], atol=1e-14)


# --------------------------------------------------------------- SDFs ---
def test_solid_box_sdf_matches_clamp_definition(orc):
    rng = np.random.default_rng(1)
    c, h = np.array([0.4, 0.5, 0.3]), np.array([0.1, 0.05, 0.07])
    rec = scenes.sdf_table([scenes.solid_box(c, h)])[0]
    lo, hi = c - h, c + h
    for x in rng.uniform(0.1, 0.7, size=(400, 3)):
        phi, n, tie = orc.sdf_eval(rec, x)
        q = np.clip(x, lo, hi)
        if np.any(x < lo) or np.any(x > hi):
            ref = np.linalg.norm(x - q)
        else:
            ref = -min(np.min(x - lo), np.min(hi - x))
        assert phi[0] == pytest.approx(ref, abs=1e-14)
        if not tie:
            e = 1e-7
            fd = np.array([(orc.sdf_eval(rec, x + e * np.eye(3)[k])[0][0]
                            - orc.sdf_eval(rec, x - e * np.eye(3)[k])[0][0]) / (2 * e) for k in range(3)])
            np.testing.assert_allclose(n[0], fd, atol=1e-5)


def test_cone_shell_sdf_matches_sampled_surface(orc):
    rng = np.random.default_rng(2)
    cx, cy, z0, r0, z1, r1, th = 0.2, 0.2, 0.05, 0.01, 0.25, 0.15, 0.005
    rec = scenes.sdf_table([scenes.cone_shell(cx, cy, z0, r0, z1, r1, th)])[0]
    # dense sampling of the mid-surface (the segment revolved about the axis)
    t = np.linspace(0, 1, 801)
    ang = np.linspace(0, 2 * np.pi, 1441)[:-1]
    R, Z = r0 + t * (r1 - r0), z0 + t * (z1 - z0)
    surf = np.stack([cx + np.outer(R, np.cos(ang)), cy + np.outer(R, np.sin(ang)),
                     np.repeat(Z[:, None], len(ang), 1)], -1).reshape(-1, 3)
    seg = math.hypot(r1 - r0, z1 - z0) / 800
    res = math.sqrt(seg ** 2 + (r1 * 2 * np.pi / 1440) ** 2)
    for x in rng.uniform([0.0, 0.0, 0.0], [0.4, 0.4, 0.35], size=(60, 3)):
        phi, n, tie = orc.sdf_eval(rec, x)
        ref = np.sqrt(((surf - x) ** 2).sum(1)).min() - th
        assert abs(phi[0] - ref) <= res
        e = 1e-7
        fd = np.array([(orc.sdf_eval(rec, x + e * np.eye(3)[k])[0][0]
                        - orc.sdf_eval(rec, x - e * np.eye(3)[k])[0][0]) / (2 * e) for k in range(3)])
        np.testing.assert_allclose(n[0], fd, atol=1e-5)


def test_box_interior_components(orc):
    rec = scenes.sdf_table([scenes.box_interior((0, 0, 0), (1, 2, 3))])[0]
    phi, n, _ = orc.sdf_eval(rec, [0.25, 0.5, 2.0])
    np.testing.assert_allclose(phi, [0.25, 0.75, 0.5, 1.5, 2.0, 1.0])
    np.testing.assert_allclose(n, [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])


# ------------------------------------------------------ binning / grid ---
def test_counting_sort_matches_stable_argsort(orc):
    rng = np.random.default_rng(3)
    for n, nk in ((0, 5), (1, 1), (1000, 7), (5000, 4096), (300, 1)):
        keys = rng.integers(0, nk, size=n).astype(np.uint32)
        idx, start = orc.counting_sort(keys, nk)
        np.testing.assert_array_equal(idx, np.argsort(keys, kind="stable"))
        np.testing.assert_array_equal(start, np.searchsorted(np.sort(keys), np.arange(nk + 1), side="left"))


def test_grid_contract_dims(orc):
    o, h, ih, dims = orc.grid(0.0089, (0, 0, 0), (1.0, 1.0, 0.6))
    assert h >= 3 * 0.0089 and h < 3 * 0.0089 * 1.002
    assert list(dims) == [math.ceil(1.0 / h), math.ceil(1.0 / h), math.ceil(0.6 / h)]
    assert dims[0] * h >= 1.0 and (dims[0] - 1) * h < 1.0


def test_cell_keys_agree_with_geometry(orc):
    rng = np.random.default_rng(4)
    lo, hi = np.array([-0.1, 0.0, 0.2]), np.array([0.5, 0.4, 0.9])
    o, h, ih, dims = orc.grid(0.007, lo, hi)
    pos = np.zeros((20000, 4), np.float32)
    pos[:, :3] = rng.uniform(lo - 0.05, hi + 0.05, size=(20000, 3))
    keys = orc.cell_keys(pos, o, ih, dims, fine=False)
    fkeys = orc.cell_keys(pos, o, ih, dims, fine=True)
    a = (pos[:, :3].astype(np.float64) - lo) / h          # exact geometry in double
    sub = np.clip(np.floor(2 * a), 0, 2 * dims - 1).astype(np.int64)
    near = np.abs(2 * a - np.round(2 * a)) < 1e-4         # within rounding of a sub-cell face
    ok = ~near.any(1)
    c = sub >> 1
    ref = (c[:, 2] * dims[1] + c[:, 1]) * dims[0] + c[:, 0]
    np.testing.assert_array_equal(keys[ok], ref[ok])
    oct_ = (sub[:, 2] & 1) * 4 + (sub[:, 1] & 1) * 2 + (sub[:, 0] & 1)
    np.testing.assert_array_equal(fkeys[ok], (8 * ref + oct_)[ok])
    np.testing.assert_array_equal(fkeys >> 3, keys)
    assert ok.mean() > 0.99


def test_pairs_closer_than_support_are_adjacent_cells(orc):
    rng = np.random.default_rng(5)
    r = 0.0089
    o, h, ih, dims = orc.grid(r, (0, 0, 0), (1, 1, 0.6))
    a = rng.uniform(0.05, 0.55, size=(50000, 3))
    d = rng.normal(size=(50000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    b = a + d * (3 * r) * (1 - 1e-7)
    pa = np.zeros((50000, 4), np.float32)
    pb = np.zeros((50000, 4), np.float32)
    pa[:, :3], pb[:, :3] = a, b
    pa32, pb32 = pa[:, :3].astype(np.float64), pb[:, :3].astype(np.float64)
    keep = np.linalg.norm(pa32 - pb32, axis=1) < 3 * r
    ka, kb = orc.cell_keys(pa, o, ih, dims), orc.cell_keys(pb, o, ih, dims)

    def coords(k):
        return np.stack([k % dims[0], (k // dims[0]) % dims[1], k // (dims[0] * dims[1])], 1).astype(np.int64)
    assert np.abs(coords(ka) - coords(kb))[keep].max() <= 1


def test_pair_search_equals_numpy_brute_force(orc):
    rng = np.random.default_rng(6)
    a = rng.uniform(0, 0.2, size=(300, 3))
    b = rng.uniform(-0.02, 0.22, size=(400, 3))
    R = 0.03
    D = np.sqrt(((a[:, None, :] - b[None, :, :]) ** 2).sum(-1))
    ref_i, ref_j = np.nonzero(D < R)
    for use_grid in (False, True):
        i, j = orc.pairs_within(a, b, R, use_grid=use_grid)
        np.testing.assert_array_equal(i, ref_i)
        np.testing.assert_array_equal(j, ref_j)


def test_upsample_grid_mode_is_bitwise_brute_force(orc):
    sc = scenes.stir(scenes.cube(), seed=11)
    prm = up_prm(r_low=sc["r_low"], r_high=sc["r_high"])
    sdf = scenes.sdf_table(sc["sdfs"])
    args = (sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["hr_pos"][:, :3], sc["hr_vel"][:, :3], sdf, prm)
    a = orc.upsample(*args, mode=0)
    b = orc.upsample(*args, mode=1)
    for k in ("x", "v", "flag", "diag"):
        np.testing.assert_array_equal(a[k], b[k])


# ------------------------------------------------------------- LR step ---
def test_lr_free_fall_parabola(orc):
    p = pb_prm(dt=1.0 / 240.0, g=(0.0, 0.0, -9.81))
    x0, v0 = np.array([[0.3, 0.1, 5.0]]), np.array([[0.2, -0.1, 0.4]])
    x, v = x0.copy(), v0.copy()
    g = np.array([0, 0, -9.81])
    for n in range(1, 21):
        x, v, _, _ = orc.pbd_step(x, v, [1.0], BIG_BOX, p)
        np.testing.assert_allclose(v[0], v0[0] + n * p["dt"] * g, atol=1e-12)
        np.testing.assert_allclose(x[0], x0[0] + n * p["dt"] * v0[0] + p["dt"] ** 2 * g * n * (n + 1) / 2,
                                   atol=1e-12)


def test_stabilization_separates_overlap_without_velocity(orc):
    r = 0.0625
    d = 0.015625
    for im, share in (((1.0, 1.0), (0.5, 0.5)), ((1.0, 3.0), (0.25, 0.75))):
        x = np.array([[1.0, 1.0, 1.0], [1.0 + 2 * r - d, 1.0, 1.0]])
        x1, v1, _, _ = orc.pbd_step(x, np.zeros((2, 3)), im, BIG_BOX, pb_prm(r=r, g=(0, 0, 0), n_stab=1, iters=0))
        assert x1[0, 0] == pytest.approx(1.0 - share[0] * d, abs=1e-15)
        assert x1[1, 0] == pytest.approx(1.0 + 2 * r - d + share[1] * d, abs=1e-15)
        np.testing.assert_array_equal(v1, 0.0)


def test_solver_contact_is_inelastic_and_conserves_momentum(orc):
    r, dt = 0.0625, 1.0 / 16.0
    u = 0.5
    for im in ((1.0, 1.0), (1.0, 3.0)):
        x = np.array([[1.0, 1.0, 1.0], [1.0 + 2 * r, 1.0, 1.0]])
        v = np.array([[u, 0, 0], [-u, 0, 0]])
        x1, v1, _, _ = orc.pbd_step(x, v, im, BIG_BOX, pb_prm(r=r, dt=dt, g=(0, 0, 0), n_stab=2, iters=3))
        m = 1.0 / np.array(im)
        common = (m[0] * u - m[1] * u) / m.sum()
        np.testing.assert_allclose(v1[:, 0], [common, common], atol=1e-14)
        np.testing.assert_allclose(v1[:, 1:], 0.0, atol=1e-15)
        assert x1[1, 0] - x1[0, 0] == pytest.approx(2 * r, abs=1e-14)


def test_boundary_has_infinite_mass(orc):
    r, d = 0.0625, 0.015625
    x = np.array([[0.5, 0.5, r - d]])
    x1, v1, _, _ = orc.pbd_step(x, np.zeros((1, 3)), [1.0], BIG_BOX, pb_prm(r=r, g=(0, 0, 0), n_stab=1, iters=0))
    np.testing.assert_allclose(x1[0], [0.5, 0.5, r], atol=1e-15)
    np.testing.assert_array_equal(v1, 0.0)


@pytest.mark.parametrize("u,expect", [(0.5, 0.0), (1.0, 1.0 - 2 * 0.0625 * 0.30 * 16.0)])
def test_friction_static_and_kinetic_closed_form(orc, u, expect):
    # grain resting on the floor (phi = r exactly) sliding with u; with these
    # binary-exact numbers the floor contact is active in the first solver
    # pass only.  |d_perp| = u dt against 2 r mu_s = 0.04375:
    #   u = 0.5: 0.03125 < 0.04375 -> static, the slide is cancelled
    #   u = 1.0: 0.0625 >= 0.04375 -> kinetic, reduced by 2 r mu_k
    r, dt = 0.0625, 1.0 / 16.0
    x = np.array([[0.5, 0.5, r]])
    v = np.array([[u, 0.0, 0.0]])
    x1, v1, _, _ = orc.pbd_step(x, v, [1.0], BIG_BOX, pb_prm(r=r, dt=dt, g=(0, 0, -8.0), mu_s=0.35, mu_k=0.30))
    assert v1[0, 0] == pytest.approx(expect, abs=1e-12)
    assert v1[0, 2] == 0.0 and v1[0, 1] == 0.0
    assert x1[0, 2] == r


def test_friction_mode_uses_penetration_depth(orc):
    # mode 1 thresholds scale with the penetration depth (here g dt^2 = 1/32)
    r, dt = 0.0625, 1.0 / 16.0
    x = np.array([[0.5, 0.5, r]])
    v = np.array([[0.25, 0.0, 0.0]])   # slide 1/64 >= (1/32) 0.35 -> kinetic
    _, v1, _, _ = orc.pbd_step(x, v, [1.0], BIG_BOX, pb_prm(r=r, dt=dt, friction_mode=1))
    assert v1[0, 0] == pytest.approx(0.25 - (1.0 / 32.0) * 0.30 * 16.0, abs=1e-12)


ROUGH_FLOOR = scenes.sdf_table([scenes.box_interior((-10.0, -10.0, 0.0), (10.0, 10.0, 10.0), mu_s=1.0, mu_k=1.0)])


@pytest.mark.parametrize("u,expect", [(0.75, 0.0), (1.5, 1.5 - 2 * 0.0625 * 0.4 * 16.0)])
def test_boundary_friction_uses_cross_coefficients(orc, u, expect):
    # Sec. 3: mu_ib = sqrt(mu_i mu_b).  Grain (0.25, 0.16) on a floor (1, 1):
    # thresholds 2 r (0.5, 0.4) = (0.0625, 0.05).  The slide u dt is
    #   0.046875 (u = 0.75): static; with the grain's own mu_s it would be
    #   kinetic (0.046875 >= 2 r 0.25 = 0.03125)
    #   0.09375 (u = 1.5): kinetic, reduced by 2 r 0.4 (mean 0.58 or the
    #   floor's own 1.0 would cancel the slide; the grain's 0.16 would leave
    #   1.5 - 0.32)
    r, dt = 0.0625, 1.0 / 16.0
    x = np.array([[0.5, 0.5, r]])
    v = np.array([[u, 0.0, 0.0]])
    x1, v1, _, _ = orc.pbd_step(x, v, [1.0], ROUGH_FLOOR, pb_prm(r=r, dt=dt, g=(0, 0, -8.0)), mu=[[0.25, 0.16]])
    assert v1[0, 0] == pytest.approx(expect, abs=1e-12)
    assert v1[0, 1] == 0.0 and x1[0, 2] == r


@pytest.mark.parametrize("u,expect", [(0.25, 0.0), (0.5, 0.5 - 0.0625 * 0.2 * 16.0)])
def test_pair_friction_uses_cross_coefficients(orc, u, expect):
    # Sec. 3: a pair of grains with coefficients (0.09, 0.04) and (1, 1)
    # uses mu_ij = (sqrt(0.09), sqrt(0.04)) = (0.3, 0.2).  The grains start
    # offset in y and slide past each other at -/+u so that after the
    # prediction they sit side by side along x, overlapping by delta: the
    # contact normal is x and the relative displacement 2 u dt is
    # tangential.  The first solver pass (no stabilization, no gravity):
    #   static (2 u dt = 0.03125 < 2 r 0.3): the slide is cancelled, v_y = 0
    #   kinetic (2 u dt = 0.0625 >= 0.0375): each grain gives back r mu_k,
    #   v_y = +/-(u - r 0.2 / dt) = +/-0.3 (the arithmetic mean or the
    #   maximum would be static, v_y = 0; the minimum 0.46; either grain's
    #   own coefficient, 0.46 or static)
    # and both grains leave contact (|x_ij| > 2 r), so later passes add
    # nothing; the overlap delta is split, v_x = -/+ delta / (2 dt).
    r, dt, delta = 0.0625, 1.0 / 16.0, 1.0 / 64.0
    x = np.array([[1.0, 1.0 - u * dt, 1.0], [1.0 + 2 * r - delta, 1.0 + u * dt, 1.0]])
    v = np.array([[0.0, u, 0.0], [0.0, -u, 0.0]])
    mu = [[0.09, 0.04], [1.0, 1.0]]
    for m in (mu, mu[::-1]):   # the cross coefficient is symmetric
        _, v1, _, _ = orc.pbd_step(x, v, [1.0, 1.0], BIG_BOX, pb_prm(r=r, dt=dt, g=(0, 0, 0), n_stab=0, iters=3),
                                   mu=m)
        np.testing.assert_allclose(v1[:, 1], [expect, -expect], atol=1e-12)
        np.testing.assert_allclose(v1[:, 0], [-delta / (2 * dt), delta / (2 * dt)], atol=1e-12)


def test_uniform_per_particle_friction_equals_the_step_coefficients(orc):
    # sqrt(mu mu) = mu exactly in binary floating point, so per-particle
    # coefficients that all equal the step's give the step bit for bit
    rng = np.random.default_rng(7)
    r = 0.0625
    x = np.array([[0.5 + 0.11 * (k % 4), 0.5 + 0.11 * (k // 4 % 4), r + 0.11 * (k // 16)] for k in range(40)])
    x += rng.uniform(-0.01, 0.01, x.shape)
    v = rng.uniform(-1.0, 1.0, x.shape)
    prm = pb_prm(r=r)
    a = orc.pbd_step(x, v, [1.0] * len(x), BIG_BOX, prm)
    b = orc.pbd_step(x, v, [1.0] * len(x), BIG_BOX, prm, mu=[[prm["mu_s"], prm["mu_k"]]] * len(x))
    assert a[3]["active"] > 0
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_jacobi_averaging_three_in_a_row(orc):
    r, d1, d2 = 0.0625, 0.015625, 0.0078125
    x = np.array([[1.0, 1, 1], [1.0 + 2 * r - d1, 1, 1], [1.0 + 4 * r - d1 - d2, 1, 1]])
    x1, _, _, _ = orc.pbd_step(x, np.zeros((3, 3)), [1.0] * 3, BIG_BOX, pb_prm(r=r, g=(0, 0, 0), n_stab=1,
                                                                                  iters=0))
    np.testing.assert_allclose(x1[:, 0] - x[:, 0], [-d1 / 2, (d1 / 2 - d2 / 2) / 2, d2 / 2], atol=1e-15)


def test_height_scaled_mass(orc):
    # m* = m e^{-h}: the higher grain is lighter and takes the larger share
    r, d, k = 0.0625, 0.015625, 2.0
    z0, z1 = 1.0, 1.0 + 2 * r - d
    x = np.array([[1.0, 1.0, z0], [1.0, 1.0, z1]])
    x1, _, _, _ = orc.pbd_step(x, np.zeros((2, 3)), [1.0, 1.0], BIG_BOX,
                               pb_prm(r=r, g=(0, 0, 0), n_stab=1, iters=0, mass_k=k, ground_z=0.0))
    w0, w1 = math.exp(k * z0), math.exp(k * z1)
    assert x1[0, 2] - z0 == pytest.approx(-d * w0 / (w0 + w1), abs=1e-14)
    assert x1[1, 2] - z1 == pytest.approx(d * w1 / (w0 + w1), abs=1e-14)
    assert x1[1, 2] - z1 > -(x1[0, 2] - z0)


def test_single_grain_rests_exactly(orc):
    r = 0.0625
    x = np.array([[0.5, 0.5, r]])
    v = np.zeros((1, 3))
    for _ in range(20):
        x, v, _, _ = orc.pbd_step(x, v, [1.0], BIG_BOX, pb_prm(r=r))
    np.testing.assert_array_equal(v, 0.0)
    np.testing.assert_array_equal(x, [[0.5, 0.5, r]])


def test_column_comes_to_rest(orc):
    # A 3-grain column on the floor converges to a stationary configuration.
    # Stabilization shifts x and xt together each step, so at the fixed
    # point the reported velocity equals minus the stabilization shift / dt
    # while the positions no longer move; without stabilization the
    # velocity itself vanishes.
    r, dt = 0.01, 1.0 / 240.0
    for n_stab in (2, 0):
        x = np.array([[0.5, 0.5, r + 2 * r * k] for k in range(3)])
        v = np.zeros((3, 3))
        p = pb_prm(r=r, dt=dt, g=(0, 0, -9.81), n_stab=n_stab, iters=4)
        for _ in range(500):
            x, v, _, _ = orc.pbd_step(x, v, [1.0] * 3, BIG_BOX, p)
        x_prev = x.copy()
        for _ in range(100):
            x, v, _, _ = orc.pbd_step(x, v, [1.0] * 3, BIG_BOX, p)
        assert np.abs(x - x_prev).max() < 1e-9 * r
        gaps = np.diff(x[:, 2])
        assert np.all(gaps > 2 * r * 0.97) and x[0, 2] > r * 0.97
        np.testing.assert_allclose(x[:, :2], 0.5, atol=1e-12)
        if n_stab == 0:
            assert np.abs(v).max() < 1e-9
        else:
            assert np.abs(v[:, :2]).max() == 0.0 and np.all(v[:, 2] < 0)


def test_lr_grid_mode_is_bitwise_brute_force(orc):
    sc = scenes.stir(scenes.cube(), seed=12)
    r = sc["r_low"]
    p = pb_prm(r=r, dt=1.0 / 240.0, g=(0, 0, -9.81), mu_s=0.5, mu_k=0.5, iters=4, mass_k=1.0, eps_x=1e-6)
    sdf = scenes.sdf_table(sc["sdfs"])
    x, v, im = sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["lr_pos"][:, 3]
    a = orc.pbd_step(x, v, im, sdf, p, mode=0)
    b = orc.pbd_step(x, v, im, sdf, p, mode=1)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[3] == b[3]


def test_settled_pile_keeps_overlap_small(orc):
    # after one second of settling at the paper's LR step size the residual
    # interpenetration stays a few percent of the contact distance
    sc = scenes.cube()
    r = sc["r_low"]
    p = pb_prm(r=r, dt=1.0 / 240.0, g=(0, 0, -9.81), mu_s=0.5, mu_k=0.5, iters=8, mass_k=1.0, eps_x=1e-6)
    x, v = sc["lr_pos"][:, :3].astype(float), np.zeros((len(sc["lr_pos"]), 3))
    im = sc["lr_pos"][:, 3].astype(float)
    sdf = scenes.sdf_table(sc["sdfs"])
    for _ in range(240):
        x, v, _, st = orc.pbd_step(x, v, im, sdf, p, mode=1)
    i, j = orc.pairs_within(x, x, 2 * r, use_grid=True)
    m = i < j
    ov = (2 * r - np.linalg.norm(x[i[m]] - x[j[m]], axis=1)).max() / (2 * r)
    assert ov < 0.06
    assert x[:, 2].min() > 0.9 * r
    assert np.all(np.isfinite(x))
