"""Pins of the oracle's initial volume sampling (Sec. 4): the generalized
winding number against closed forms, and the sampler against what its
definition fixes -- every pair of samples at least 2 r apart, every sample
inside the mesh (checked by half-spaces, independently of the winding
number), at most one sample per cell of side 2 r / sqrt(3), every unchosen
inside candidate blocked by a sample or behind its cell's pick, the same
samples as a brute-force greedy over the same cell order (also with the
cells of each phase shuffled), and the same samples for the same seed."""
import math

import numpy as np
import pytest

import scenes


def test_winding_number_closed_forms(orc):
    # one octant triangle seen from the origin covers 1/8 of the sphere
    V = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    assert orc.winding_number(V, [[0, 1, 2]], [[0, 0, 0]])[0] == pytest.approx(1 / 8, abs=1e-15)
    assert orc.winding_number(V, [[0, 2, 1]], [[0, 0, 0]])[0] == pytest.approx(-1 / 8, abs=1e-15)
    # a regular tetrahedron seen from its centroid: each face 1/4
    Vt = np.array([[1.0, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]])
    Tt = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]])
    for f in range(4):
        assert abs(orc.winding_number(Vt, Tt[f:f + 1], [[0, 0, 0]])[0]) == pytest.approx(0.25, abs=1e-14)
    w = orc.winding_number(Vt, Tt, [[0, 0, 0], [0.2, 0.1, -0.1], [3, 0, 0], [0, 0, -2.5]])
    np.testing.assert_allclose(np.abs(w), [1, 1, 0, 0], atol=1e-13)
    # closed meshes: 1 inside, 0 outside; the overlap of two parts counts twice
    for V2, T2, inside, outside in [(*scenes.box_mesh((0, 0, 0), (1, 2, 3)), (0.3, 1.9, 0.2), (1.2, 1, 1)),
                                    (*scenes.icosphere((1, 1, 1), 0.5, 2), (1.2, 0.9, 1.3), (1.5, 1.5, 1.5)),
                                    (*scenes.prism_mesh(0, 0, 1, 0, 1, 16, apex=0.5), (0, 0, 1.3), (0, 0, 1.6))]:
        np.testing.assert_allclose(orc.winding_number(V2, T2, [inside, outside]), [1, 0], atol=1e-12)
    V3, T3 = scenes.merge_meshes([scenes.box_mesh((0, 0, 0), (2, 2, 2)), scenes.box_mesh((1, 1, 1), (3, 3, 3))])
    np.testing.assert_allclose(orc.winding_number(V3, T3, [[0.5, 0.5, 0.5], [1.5, 1.5, 1.5], [2.5, 2.5, 2.5]]),
                               [1, 2, 1], atol=1e-12)


def _convex_inside(V, T, p, eps=1e-12):
    """p inside the convex closed mesh (V, T): behind every face plane."""
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(b - a, c - a)
    return np.all(np.einsum("fk,pfk->pf", n, p[:, None, :] - a[None]) < eps, axis=1)


def _castle_parts(size=0.6, height=0.2):
    base = (0.5, 0.5, 0.0)
    cx, cy, z0 = base
    h2 = size / 2
    parts = [scenes.box_mesh((cx - h2, cy - h2, z0), (cx + h2, cy + h2, z0 + height)),
             scenes.box_mesh((cx - 0.2 * size, cy - 0.2 * size, z0 + 0.5 * height),
                             (cx + 0.2 * size, cy + 0.2 * size, z0 + 2.0 * height))]
    for sx in (-1, 1):
        for sy in (-1, 1):
            parts.append(scenes.prism_mesh(cx + sx * 0.8 * h2, cy + sy * 0.8 * h2, 0.12 * size, z0,
                                           z0 + 1.6 * height, n=20, apex=0.6 * height))
    return parts


def _cells(orc, V, r, pts):
    lo, h, dims = orc.sample_grid(V, r)
    c = np.clip(np.floor((pts - lo) / h).astype(np.int64), 0, dims - 1)
    return c, dims, h


def _check_sampling(orc, V, T, cand, r, inside_ref):
    sel, inside = orc.sample_volume(V, T, cand, r)
    P = cand[sel]
    # inside, by an independent test
    assert inside_ref(P).all()
    np.testing.assert_array_equal(inside, inside_ref(cand))   # the classification itself (no point on a face)
    # every pair at least 2 r apart
    d2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    assert d2.min() >= 4 * r * r
    # at most one sample per cell, listed in ascending cell order
    c, dims, h = _cells(orc, V, r, P)
    lin = c[:, 0] + dims[0] * (c[:, 1] + dims[1] * c[:, 2])
    assert len(np.unique(lin)) == len(lin) and np.all(np.diff(lin) > 0)
    assert h == pytest.approx(2 * r / math.sqrt(3), rel=1e-15)
    # maximal: every unchosen inside candidate is blocked by a sample, or its
    # cell's pick comes before it in input order
    ci, _, _ = _cells(orc, V, r, cand)
    lin_c = ci[:, 0] + dims[0] * (ci[:, 1] + dims[1] * ci[:, 2])
    pick_of = dict(zip(lin.tolist(), sel.tolist()))
    chosen = np.zeros(len(cand), bool)
    chosen[sel] = True
    for i in np.flatnonzero(inside & ~chosen):
        blocked = ((P - cand[i]) ** 2).sum(-1).min() < 4 * r * r
        earlier = pick_of.get(int(lin_c[i]), 1 << 62) < i
        assert blocked or earlier, i
    return sel


def test_sampler_on_a_sphere(orc):
    V, T = scenes.icosphere((0.3, 0.2, 0.1), 0.15, 2)
    r = 0.012
    cand = scenes.volume_candidates(V, r, per_cell=5.0, seed=7)
    sel = _check_sampling(orc, V, T, cand, r, lambda p: _convex_inside(V, T, p))
    # the volume is filled: sphere volume fraction of the samples
    vol = abs(float(np.sum(np.einsum("fk,fk->f", V[T[:, 0]], np.cross(V[T[:, 1]], V[T[:, 2]]))) / 6.0))
    frac = len(sel) * 4 / 3 * math.pi * r ** 3 / vol
    assert 0.25 < frac < 0.5, frac


def test_sampler_on_the_castle_union(orc):
    parts = _castle_parts()
    V, T = scenes.merge_meshes(parts)
    r = 0.02
    cand = scenes.volume_candidates(V, r, per_cell=4.0, seed=11)
    _check_sampling(orc, V, T, cand, r, lambda p: np.any([_convex_inside(v, t, p) for v, t in parts], axis=0))


def _greedy_brute(orc, V, r, cand, inside, shuffle_seed=None):
    """The sampler's definition on a tiny input: phases in order, the cells
    of a phase in linear order (or shuffled), candidates in input order,
    distance to every sample so far."""
    c, dims, h = _cells(orc, V, r, cand)
    lin = c[:, 0] + dims[0] * (c[:, 1] + dims[1] * c[:, 2])
    phase = (c[:, 0] % 3) + 3 * (c[:, 1] % 3) + 9 * (c[:, 2] % 3)
    rng = np.random.default_rng(shuffle_seed) if shuffle_seed is not None else None
    samples, picks = [], {}
    for ph in range(27):
        cells = sorted(set(lin[inside & (phase == ph)].tolist()))
        if rng is not None:
            rng.shuffle(cells)
        for cell in cells:
            for i in np.flatnonzero(inside & (lin == cell)):
                if all(((cand[i] - cand[s]) ** 2).sum() >= 4 * r * r for s in samples):
                    samples.append(i)
                    picks[cell] = i
                    break
    return np.array([picks[k] for k in sorted(picks)], np.int64)


@pytest.mark.parametrize("shuffle", [None, 1, 2])
def test_sampler_equals_the_brute_force_greedy(orc, shuffle):
    V, T = scenes.icosphere((0.0, 0.0, 0.0), 0.06, 1)
    r = 0.01
    cand = scenes.volume_candidates(V, r, per_cell=3.0, seed=3)
    sel, inside = orc.sample_volume(V, T, cand, r)
    np.testing.assert_array_equal(sel, _greedy_brute(orc, V, r, cand, inside, shuffle))


def test_sampler_is_deterministic_per_seed(orc):
    V, T = scenes.icosphere((0.0, 0.0, 0.0), 0.1, 2)
    r = 0.01
    a = orc.sample_volume(V, T, scenes.volume_candidates(V, r, seed=5), r)[0]
    b = orc.sample_volume(V, T, scenes.volume_candidates(V, r, seed=5), r)[0]
    c = orc.sample_volume(V, T, scenes.volume_candidates(V, r, seed=6), r)[0]
    np.testing.assert_array_equal(a, b)
    assert len(a) != len(c) or not np.array_equal(a, c)


def test_sampler_edge_cases(orc):
    V, T = scenes.box_mesh((0, 0, 0), (0.1, 0.1, 0.1))
    r = 0.01
    sel, inside = orc.sample_volume(V, T, np.zeros((0, 3)), r)        # no candidates
    assert len(sel) == 0
    sel, inside = orc.sample_volume(V, T, [[0.05, 0.05, 0.05]], r)     # one
    np.testing.assert_array_equal(sel, [0])
    sel, inside = orc.sample_volume(V, T, [[0.5, 0.5, 0.5], [-1, 0, 0]], r)   # all outside
    assert len(sel) == 0 and not inside.any()
    # two candidates in one cell: the first one wins
    sel, _ = orc.sample_volume(V, T, [[0.05, 0.05, 0.05], [0.0501, 0.05, 0.05]], r)
    np.testing.assert_array_equal(sel, [0])


def test_surface_sampler_on_a_box(orc):
    """Surface sampling (Sec. 3's boundary particles): every sample on a face
    of the box, pairs at least 2 r apart, one per cell at most, every
    unchosen candidate blocked by a sample or behind its cell's pick, the
    brute-force greedy's result, the same samples for the same seed."""
    lo, hi = np.array([0.1, 0.2, 0.05]), np.array([0.35, 0.3, 0.2])
    V, T = scenes.box_mesh(lo, hi)
    r = 0.01
    cand = scenes.surface_candidates(V, T, r, per_cell=5.0, seed=4)
    on_face = np.any(np.isclose(cand, lo, atol=1e-12) | np.isclose(cand, hi, atol=1e-12), axis=1)
    assert on_face.all()   # the candidate generator puts points on the faces
    sel = orc.sample_surface(V, cand, r)
    P = cand[sel]
    assert len(sel) > 100
    d2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    assert d2.min() >= 4 * r * r
    c, dims, h = _cells(orc, V, r, P)
    lin = c[:, 0] + dims[0] * (c[:, 1] + dims[1] * c[:, 2])
    assert len(np.unique(lin)) == len(lin) and np.all(np.diff(lin) > 0)
    ci, _, _ = _cells(orc, V, r, cand)
    lin_c = ci[:, 0] + dims[0] * (ci[:, 1] + dims[1] * ci[:, 2])
    pick_of = dict(zip(lin.tolist(), sel.tolist()))
    chosen = np.zeros(len(cand), bool)
    chosen[sel] = True
    for i in np.flatnonzero(~chosen):
        assert ((P - cand[i]) ** 2).sum(-1).min() < 4 * r * r or pick_of.get(int(lin_c[i]), 1 << 62) < i, i
    small = cand[:400]
    np.testing.assert_array_equal(orc.sample_surface(V, small, r),
                                  _greedy_brute(orc, V, r, small, np.ones(len(small), bool)))
    np.testing.assert_array_equal(sel, orc.sample_surface(V, scenes.surface_candidates(V, T, r, 5.0, seed=4), r))
