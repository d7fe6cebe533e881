"""Seeded synthetic scenes shaped like the paper's workloads (Sec. 5.2).

This package only draws inputs: particle positions and velocities, boundary
descriptions and per-frame boundary poses.  It holds none of the method's
arithmetic, so both the CUDA library and the CPU oracle can be fed from it
without sharing code.  The paper's own scenes need triangle meshes and an
interactive excavator; these stand-ins keep their sizes, radii and shapes:

* ``cube``    -- 10x10x10 jittered lattice (r_LR = 0.01 m) in a 0.5 m box,
                 ratio 8 (a sanity scene).
* ``funnel``  -- 20,000 LR (r_LR = 0.005 m) above an analytic cone shell
                 with a 2 cm outlet, ratio 25 -> 500,000 HR (stands in for
                 the hourglass scene, 10k LR / 460k HR).
* ``digging`` -- 1 x 1 m sand bed, 0.3 m deep with seeded value-noise
                 height, r_LR = 0.0089 m (50,527 LR), ratio 40 -> 2,021,080
                 HR, and a kinematic box "bucket" on a piecewise-
                 linear path (stands in for the excavator scenes).
* ``column``  -- a falling column, 4,000 LR / 64,000 HR (differentiation).
* ``batch``   -- many independent small scenes of uneven sizes.

Arrays follow the library's layout: float32 (n, 4) with pos.w = inverse mass
for LR and the HR particle's original index (as uint32 bits) for HR;
vel.w = 0.  Layout of an SDF record: dict(kind, p[12], vel[3], mu_s, mu_k).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2308016290
SDF_BOX_INTERIOR, SDF_CONE_SHELL, SDF_SOLID_BOX = 1, 2, 3
GRAVITY = (0.0, 0.0, -9.81)
RHO = 1600.0                       # Sec. 5.2 granular density
MU_S, MU_K = 0.35, 0.30            # Sec. 5.2 friction coefficients


# ----------------------------------------------------------------- SDFs ---
def _rec(kind, p, vel=(0.0, 0.0, 0.0), mu_s=MU_S, mu_k=MU_K):
    pp = [0.0] * 12
    pp[:len(p)] = [float(a) for a in p]
    return dict(kind=int(kind), p=pp, vel=[float(a) for a in vel], mu_s=float(mu_s), mu_k=float(mu_k))


def box_interior(lo, hi, **kw):
    return _rec(SDF_BOX_INTERIOR, list(lo) + list(hi), **kw)


def cone_shell(cx, cy, z_out, r_out, z_top, r_top, half_thickness, **kw):
    return _rec(SDF_CONE_SHELL, [cx, cy, z_out, r_out, z_top, r_top, half_thickness], **kw)


def solid_box(center, half, vel=(0.0, 0.0, 0.0), **kw):
    return _rec(SDF_SOLID_BOX, list(center) + list(half), vel=vel, **kw)


def sdf_table(sdfs):
    """SDF records as the oracle's float64 (n, 20) table."""
    t = np.zeros((len(sdfs), 20))
    for i, s in enumerate(sdfs):
        t[i, 0] = s["kind"]
        t[i, 1:13] = s["p"]
        t[i, 13:16] = s["vel"]
        t[i, 16] = s["mu_s"]
        t[i, 17] = s["mu_k"]
    return t


# ------------------------------------------------------------ sampling ---
def _ball(rng, n):
    """n points uniform in the unit ball (rejection sampling)."""
    out = np.empty((0, 3))
    while len(out) < n:
        c = rng.uniform(-1.0, 1.0, size=(2 * (n - len(out)) + 16, 3))
        c = c[(c * c).sum(1) <= 1.0]
        out = np.concatenate([out, c])
    return out[:n]


def _hr_in_balls(rng, lr_xyz, r_low, ratio):
    """`ratio` HR per LR particle, uniform inside that LR particle's sphere."""
    n = len(lr_xyz)
    off = _ball(rng, n * ratio) * r_low
    return np.repeat(lr_xyz, ratio, axis=0) + off


def _pack(xyz, w):
    a = np.zeros((len(xyz), 4), np.float32)
    a[:, :3] = xyz
    a[:, 3] = w
    return a


def hr_ids(m):
    return np.arange(m, dtype=np.uint32).view(np.float32)


def _finish(name, seed, box_lo, box_hi, r_low, ratio, lr_xyz, rng, sdfs, dt, iters, mu_s=MU_S, mu_k=MU_K,
            r_high=None, **extra):
    m_lr = RHO * 4.0 / 3.0 * math.pi * r_low ** 3
    n = len(lr_xyz)
    lr_pos = _pack(lr_xyz, np.float32(1.0 / m_lr))
    hr_xyz = _hr_in_balls(rng, lr_xyz, r_low, ratio)
    hr_pos = _pack(hr_xyz, 0.0)
    hr_pos[:, 3] = hr_ids(len(hr_xyz))
    if r_high is None:
        r_high = r_low * ratio ** (-1.0 / 3.0)
    sc = dict(name=name, seed=seed, box_lo=[float(a) for a in box_lo], box_hi=[float(a) for a in box_hi],
              r_low=float(r_low), r_high=float(r_high), ratio=int(ratio), sdfs=sdfs,
              gravity=GRAVITY, mu_s=mu_s, mu_k=mu_k, dt=float(dt), iters=int(iters),
              lr_pos=lr_pos, lr_vel=np.zeros((n, 4), np.float32),
              hr_pos=hr_pos, hr_vel=np.zeros((len(hr_pos), 4), np.float32))
    sc.update(extra)
    return sc


def _lattice(rng, lo, counts, spacing, jitter):
    g = np.stack(np.meshgrid(*[np.arange(c) for c in counts], indexing="ij"), -1).reshape(-1, 3)
    g = g[:, [0, 1, 2]].astype(np.float64)
    xyz = np.asarray(lo, float) + g * spacing
    return xyz + rng.uniform(-jitter, jitter, size=xyz.shape)


# --------------------------------------------------------------- scenes ---
def cube(seed=SEED_BASE + 0, n_side=10, r_low=0.01, ratio=8):
    """Jittered lattice cube (spacing 2r, jitter +-0.1r) in a 0.5 m box."""
    rng = np.random.default_rng(seed)
    box_lo, box_hi = (0.0, 0.0, 0.0), (0.5, 0.5, 0.5)
    sp = 2.0 * r_low
    half = 0.5 * sp * (n_side - 1)
    lo = (0.25 - half, 0.25 - half, 0.15 + r_low)
    xyz = _lattice(rng, lo, (n_side,) * 3, sp, 0.1 * r_low)
    return _finish("cube", seed, box_lo, box_hi, r_low, ratio, xyz, rng,
                   [box_interior(box_lo, box_hi, mu_s=0.5, mu_k=0.5)], dt=1.0 / 60.0, iters=4,
                   mu_s=0.5, mu_k=0.5)


def funnel(seed=SEED_BASE + 1, n_low=20000, r_low=0.005, ratio=25):
    """LR particles released above a cone shell (half-angle 35 deg, top radius
    0.15 m, outlet diameter 0.02 m, wall thickness 2 r_LR) in a 0.4 x 0.4 x
    0.6 m box."""
    rng = np.random.default_rng(seed)
    box_lo, box_hi = (0.0, 0.0, 0.0), (0.4, 0.4, 0.6)
    cx = cy = 0.2
    r_out, r_top = 0.01, 0.15
    height = (r_top - r_out) / math.tan(math.radians(35.0))
    z_out = 0.05
    z_top = z_out + height
    sp = 2.0 * r_low
    rad = r_top - 2.0 * r_low
    nxy = int(2 * rad / sp) + 1
    layers = []
    z = z_top + 2.0 * r_low
    total = 0
    while total < n_low:
        g = np.stack(np.meshgrid(np.arange(nxy), np.arange(nxy), indexing="ij"), -1).reshape(-1, 2)
        xy = np.array([cx - rad, cy - rad]) + g * sp
        keep = ((xy - [cx, cy]) ** 2).sum(1) <= rad * rad
        xy = xy[keep]
        layers.append(np.column_stack([xy, np.full(len(xy), z)]))
        total += len(xy)
        z += sp
    xyz = np.concatenate(layers)[:n_low]
    xyz = xyz + rng.uniform(-0.1 * r_low, 0.1 * r_low, size=xyz.shape)
    sdfs = [box_interior(box_lo, box_hi), cone_shell(cx, cy, z_out, r_out, z_top, r_top, r_low)]
    return _finish("funnel", seed, box_lo, box_hi, r_low, ratio, xyz, rng, sdfs, dt=1.0 / 60.0, iters=6)


def _value_noise(rng, n_ctrl, amp, u, v):
    c = rng.uniform(-amp, amp, size=(n_ctrl, n_ctrl))
    fu = u * (n_ctrl - 1)
    fv = v * (n_ctrl - 1)
    i0 = np.clip(np.floor(fu).astype(int), 0, n_ctrl - 2)
    j0 = np.clip(np.floor(fv).astype(int), 0, n_ctrl - 2)
    a, b = fu - i0, fv - j0
    return ((1 - a) * (1 - b) * c[i0, j0] + a * (1 - b) * c[i0 + 1, j0]
            + (1 - a) * b * c[i0, j0 + 1] + a * b * c[i0 + 1, j0 + 1])


BUCKET_HALF = (0.125, 0.075, 0.075)
BUCKET_PATH = ((0.15, 0.5, 0.42), (0.32, 0.5, 0.27), (0.68, 0.5, 0.27), (0.85, 0.5, 0.42))
BUCKET_SPEED = 0.4


def bucket_pose(t):
    """Centre and velocity of the digging bucket at time t: piecewise-linear
    ping-pong along BUCKET_PATH at BUCKET_SPEED m/s (translation only)."""
    pts = np.asarray(BUCKET_PATH, float)
    seg = np.linalg.norm(np.diff(pts, axis=0), axis=1)
    total = seg.sum()
    period = 2.0 * total / BUCKET_SPEED
    s = (t % period) * BUCKET_SPEED
    direction = 1.0
    if s > total:
        s = 2.0 * total - s
        direction = -1.0
    k = 0
    while k < len(seg) - 1 and s > seg[k]:
        s -= seg[k]
        k += 1
    d = (pts[k + 1] - pts[k]) / seg[k]
    c = pts[k] + d * min(s, seg[k])
    return c, d * BUCKET_SPEED * direction


def bucket_sdf(t):
    c, u = bucket_pose(t)
    return solid_box(c, BUCKET_HALF, vel=u)


def digging(seed=SEED_BASE + 2, r_low=0.0089, ratio=40, size=1.0, depth=0.3):
    """Sand bed with seeded value-noise height (+-0.05 m on 8x8 control
    points, bilinear) and a kinematic box bucket."""
    rng = np.random.default_rng(seed)
    box_lo, box_hi = (0.0, 0.0, 0.0), (size, size, 0.6)
    sp = 2.0 * r_low
    n_xy = int((size - 2 * r_low) / sp) + 1
    g = np.arange(n_xy) * sp + r_low
    X, Y = np.meshgrid(g, g, indexing="ij")
    H = depth + _value_noise(rng, 8, 0.05, X / size, Y / size)
    cols = []
    for k in range(int((depth + 0.05) / sp) + 2):
        z = r_low + k * sp
        m = z <= H - r_low
        cols.append(np.column_stack([X[m], Y[m], np.full(m.sum(), z)]))
    xyz = np.concatenate(cols)
    xyz = xyz + rng.uniform(-0.1 * r_low, 0.1 * r_low, size=xyz.shape)
    sdfs = [box_interior(box_lo, box_hi), bucket_sdf(0.0)]
    return _finish("digging", seed, box_lo, box_hi, r_low, ratio, xyz, rng, sdfs, dt=1.0 / 60.0, iters=8,
                   bucket_index=1)


def translated(sc, shift):
    """A copy of a scene moved by shift (metres, per axis): particles, box and
    its box-interior boundary; other SDFs are dropped."""
    sh = np.asarray(shift, np.float32)
    sc = dict(sc)
    for k in ("lr_pos", "hr_pos"):
        sc[k] = sc[k].copy()
        sc[k][:, :3] += sh
    sc["box_lo"] = tuple(float(np.float32(b) + s) for b, s in zip(sc["box_lo"], sh))
    sc["box_hi"] = tuple(float(np.float32(b) + s) for b, s in zip(sc["box_hi"], sh))
    sc["sdfs"] = [box_interior(sc["box_lo"], sc["box_hi"], mu_s=sc["mu_s"], mu_k=sc["mu_k"])]
    return sc


def column(seed=SEED_BASE + 3, n_low=4000, r_low=0.01, ratio=16, z0=0.1):
    """Falling column (10 x 10 footprint) in a 0.6 m box, lowest layer
    centred z0 above the floor."""
    rng = np.random.default_rng(seed)
    box_lo, box_hi = (0.0, 0.0, 0.0), (0.6, 0.6, 1.2)
    n_xy = 10
    layers = -(-n_low // (n_xy * n_xy))
    sp = 2.0 * r_low
    lo = (0.3 - 0.5 * sp * (n_xy - 1), 0.3 - 0.5 * sp * (n_xy - 1), z0)
    xyz = _lattice(rng, lo, (n_xy, n_xy, layers), sp, 0.1 * r_low)[:n_low]
    return _finish("column", seed, box_lo, box_hi, r_low, ratio, xyz, rng,
                   [box_interior(box_lo, box_hi)], dt=1.0 / 60.0, iters=4)


def diff_column(seed=SEED_BASE + 5, n_low=4000, ratio=16):
    """Workload of the differentiable pattern: the falling column released
    with its lowest layer 1 cm above resting contact, so it lands within the
    rollout; 30 steps of 1/240 s, each one LR step (2 stabilization + 4
    solver passes) and one HR frame; recomputation checkpoints every 5 steps.
    The loss is sum_i |x_i - t_i|^2 over the HR particles after the rollout,
    with targets t = initial HR positions moved by (5, 0, -2) cm plus seeded
    N(0, 1 cm) noise (float32, shared by both sides)."""
    sc = column(n_low=n_low, ratio=ratio, z0=0.02)
    rng = np.random.default_rng(seed)
    m = len(sc["hr_pos"])
    t = sc["hr_pos"][:, :3].astype(np.float64) + np.array([0.05, 0.0, -0.02]) + rng.normal(0.0, 0.01, (m, 3))
    sc.update(name="diff_column", target=t.astype(np.float32), dt=1.0 / 240.0, steps=30, checkpoint_every=5,
              n_stab=2, iters=4)
    return sc


def batch(seed=SEED_BASE + 4, n_scenes=256, lo_count=500, hi_count=8000, ratios=(8, 16, 32)):
    """Independent small scenes with uneven particle counts, box sizes 0.2-1.0
    m and round-robin boundary kinds (box / cone / bucket)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_scenes):
        n_low = int(rng.integers(lo_count, hi_count + 1))
        ratio = int(rng.choice(ratios))
        L = float(rng.uniform(0.2, 1.0))
        r_low = float(0.25 * L / max(2.0, round(n_low ** (1.0 / 3.0))))
        r_low = min(max(r_low, 0.003), 0.02)
        box_lo, box_hi = (0.0, 0.0, 0.0), (L, L, L)
        sp = 2.0 * r_low
        n_side = int(math.ceil(n_low ** (1.0 / 3.0)))
        n_side = min(n_side, int((L - 4 * r_low) / sp))
        layers = -(-n_low // (n_side * n_side))
        lo = (0.5 * L - 0.5 * sp * (n_side - 1), 0.5 * L - 0.5 * sp * (n_side - 1), 2 * r_low)
        xyz = _lattice(rng, lo, (n_side, n_side, layers), sp, 0.1 * r_low)[:n_low]
        sdfs = [box_interior(box_lo, box_hi)]
        kind = s % 3
        if kind == 1:
            sdfs.append(cone_shell(0.5 * L, 0.5 * L, 0.05 * L, 0.05 * L, 0.3 * L, 0.45 * L, r_low))
        elif kind == 2:
            sdfs.append(solid_box((0.5 * L, 0.5 * L, 0.8 * L), (0.1 * L, 0.1 * L, 0.05 * L),
                                  vel=(0.0, 0.0, -0.2)))
        out.append(_finish(f"batch{s}", seed, box_lo, box_hi, r_low, ratio, xyz, rng, sdfs,
                           dt=1.0 / 60.0, iters=4))
    return out


# ------------------------------------------------------ perturbed states ---
def stir(sc, seed, v_scale=0.5, spread=0.5, hr_v_scale=0.3):
    """A copy of a scene with a seeded, non-uniform LR velocity field (affine
    plus noise), random HR velocities, and a fraction of HR particles spread
    out of the LR support so every blending case occurs."""
    rng = np.random.default_rng(seed)
    sc = dict(sc)
    lr_pos = sc["lr_pos"].copy()
    hr_pos = sc["hr_pos"].copy()
    n, m = len(lr_pos), len(hr_pos)
    c = lr_pos[:, :3].mean(0)
    A = rng.normal(0, v_scale, size=(3, 3))
    b = rng.normal(0, v_scale, size=3)
    lr_vel = np.zeros((n, 4), np.float32)
    lr_vel[:, :3] = b + (lr_pos[:, :3] - c) @ A.T * 5.0 + rng.normal(0, 0.1 * v_scale, size=(n, 3))
    hr_vel = np.zeros((m, 4), np.float32)
    hr_vel[:, :3] = rng.normal(0, hr_v_scale, size=(m, 3))
    k = int(spread * 0.2 * m)
    sel = rng.choice(m, size=k, replace=False)
    hr_pos[sel, :3] += rng.normal(0, 3.0 * sc["r_low"], size=(k, 3))
    lo = np.asarray(sc["box_lo"]) + sc["r_high"]
    hi = np.asarray(sc["box_hi"]) - sc["r_high"]
    hr_pos[:, :3] = np.clip(hr_pos[:, :3], lo - 2 * sc["r_high"], hi + 2 * sc["r_high"])
    sc.update(lr_vel=lr_vel, hr_vel=hr_vel, hr_pos=hr_pos)
    return sc


# ------------------------------------------------------- grain materials ---
# Friction coefficient pairs (mu_s, mu_k) of three grain materials, from
# smooth to rough around the paper's default pair (Sec. 5.2).
MATERIALS = np.array([[MU_S, MU_K], [0.8, 0.6], [0.1, 0.05]], np.float32)


def materials(sc, seed, layout="random", table=MATERIALS):
    """(table, ids): a material per LR particle.  "random" draws each
    particle's material independently (every pairing of materials occurs);
    "layers" gives the particles above the median height the second
    material and the rest the first (a bed covered by another grain)."""
    n = len(sc["lr_pos"])
    if layout == "random":
        ids = np.random.default_rng(seed).integers(0, len(table), size=n)
    elif layout == "layers":
        z = sc["lr_pos"][:, 2]
        ids = (z > np.median(z)).astype(np.int64) if n else np.zeros(0, np.int64)
    else:
        raise ValueError(layout)
    return np.asarray(table, np.float32), ids.astype(np.uint32)


# ------------------------------------------ particle-sampled solid bodies ---
# Sec. 3: boundaries and rigid bodies sampled with LR particles of inverse
# mass 0.  Their HR share is drawn around the grains, so a context of
# n_low = grains + solids particles and ratio HR per LR holds only granular
# HR particles.
def _face_lattice(lo, hi, spacing, axes):
    """Points on the face of a box where the coordinates `axes` vary (a
    lattice of the given spacing, centred on the face)."""
    out = []
    for a in axes:
        n = max(int(round((hi[a] - lo[a]) / spacing)) + 1, 1)
        out.append(np.linspace(lo[a], hi[a], n))
    g = np.stack(np.meshgrid(*out, indexing="ij"), -1).reshape(-1, len(axes))
    return g


def box_surface(center, half, spacing):
    """Particles on the surface of an axis-aligned box (each face a lattice,
    shared edges once)."""
    c, h = np.asarray(center, float), np.asarray(half, float)
    lo, hi = c - h, c + h
    pts = []
    for a in range(3):
        b, e = [k for k in range(3) if k != a]
        face = _face_lattice(lo, hi, spacing, (b, e))
        for s in (lo[a], hi[a]):
            p = np.zeros((len(face), 3))
            p[:, a] = s
            p[:, b], p[:, e] = face[:, 0], face[:, 1]
            pts.append(p)
    p = np.unique(np.round(np.concatenate(pts), 12), axis=0)
    return p


def with_solids(sc, solid_xyz, solid_vel, seed):
    """A copy of a scene with LR particles of inverse mass 0 appended at
    solid_xyz (velocities solid_vel) and the HR set redrawn around the
    grains (ratio x all LR particles, each grain's share in turn)."""
    rng = np.random.default_rng(seed)
    sc = dict(sc)
    n_g = len(sc["lr_pos"])
    solid_xyz = np.asarray(solid_xyz, float).reshape(-1, 3)
    lr_pos = np.concatenate([sc["lr_pos"], _pack(solid_xyz, 0.0)])
    lr_vel = np.concatenate([sc["lr_vel"], np.zeros((len(solid_xyz), 4), np.float32)])
    lr_vel[n_g:, :3] = np.broadcast_to(np.asarray(solid_vel, np.float32), (len(solid_xyz), 3))
    m = sc["ratio"] * len(lr_pos)
    owner = np.arange(m) % max(n_g, 1)
    hr_xyz = sc["lr_pos"][owner, :3].astype(np.float64) + _ball(rng, m) * sc["r_low"]
    hr_pos = _pack(hr_xyz, 0.0)
    hr_pos[:, 3] = hr_ids(m)
    hr_vel = np.zeros((m, 4), np.float32)
    hr_vel[:, :3] = sc["hr_vel"][owner % len(sc["hr_vel"]), :3] if len(sc["hr_vel"]) else 0.0
    sc.update(lr_pos=lr_pos, lr_vel=lr_vel, hr_pos=hr_pos, hr_vel=hr_vel, n_solid=len(solid_xyz))
    return sc


def cube_on_particle_floor(seed=SEED_BASE + 6, v_scale=0.3):
    """The cube (stirred) standing on a particle-sampled floor instead of the
    box's floor: a 2 r_LR lattice one radius below the lowest layer, wider
    than the cube by three particles on each side."""
    sc = stir(cube(), seed=seed, v_scale=v_scale)
    r = sc["r_low"]
    lo = sc["lr_pos"][:, :3].min(0) - 3 * 2 * r
    hi = sc["lr_pos"][:, :3].max(0) + 3 * 2 * r
    z = sc["lr_pos"][:, 2].min() - 2 * r
    face = _face_lattice(lo, hi, 2 * r, (0, 1))
    floor = np.column_stack([face, np.full(len(face), z)])
    return with_solids(sc, floor, (0.0, 0.0, 0.0), seed)


def digging_particle_bucket(seed=SEED_BASE + 7, t=0.0, **kw):
    """The digging bed with the bucket sampled as particles (a 2 r_LR lattice
    on the box surface) moving with the bucket's velocity at time t, in place
    of the bucket SDF."""
    sc = digging(**kw)
    c, u = bucket_pose(t)
    pts = box_surface(c, BUCKET_HALF, 2 * sc["r_low"])
    sc = with_solids(sc, pts, u, seed)
    sc["sdfs"] = [sc["sdfs"][0]]
    sc.pop("bucket_index", None)
    return sc


# --------------------------------------------------------- rigid bodies ---
# Sec. 3 / Sec. 5.2: a movable rigid body sampled with LR particles of finite
# mass that collide like grains and are shape-matched to their rest shape
# every solver pass.  "lr_body" holds the body of each LR particle (0: a
# grain).
def cube_with_block(seed=SEED_BASE + 8, v_scale=0.3):
    """The stirred cube whose top three layers' central 4 x 4 columns form a
    rigid block (48 particles)."""
    sc = stir(cube(), seed=seed, v_scale=v_scale)
    p = sc["lr_pos"][:, :3]
    lo, hi = p.min(0), p.max(0)
    r = sc["r_low"]
    mid = 0.5 * (lo + hi)
    sel = (np.abs(p[:, 0] - mid[0]) < 4 * r) & (np.abs(p[:, 1] - mid[1]) < 4 * r) & (p[:, 2] > hi[2] - 5 * r)
    body = np.zeros(len(p), np.uint32)
    body[sel] = 1
    sc = dict(sc)
    sc["lr_body"] = body
    return sc


def digging_with_boulder(seed=SEED_BASE + 9, radius=0.08, density=5000.0, velocity=(0.0, 0.0, -2.0), **kw):
    """The digging bed with a boulder hurled into it: a sphere of radius
    `radius` sampled on a 2 r_LR lattice (density 5000 kg/m^3, the paper's
    rigid body in the sand-castle scene), its lowest particle 2 r_LR above
    the bed's highest grain, moving at `velocity`; the HR set is redrawn
    around the grains."""
    sc = digging(**kw)
    r = sc["r_low"]
    n = int(radius / (2 * r)) + 1
    g = np.stack(np.meshgrid(*[np.arange(-n, n + 1)] * 3, indexing="ij"), -1).reshape(-1, 3) * 2 * r
    g = g[np.linalg.norm(g, axis=1) <= radius]
    top = sc["lr_pos"][:, 2].max()
    c = np.array([0.5 * sc["box_hi"][0], 0.5 * sc["box_hi"][1], top + 4 * r + radius])
    xyz = g + c
    n_g = len(sc["lr_pos"])
    sc = with_solids(sc, xyz, velocity, seed)
    m = density * 4.0 / 3.0 * math.pi * r ** 3
    sc["lr_pos"][n_g:, 3] = np.float32(1.0 / m)
    body = np.zeros(len(sc["lr_pos"]), np.uint32)
    body[n_g:] = 1
    sc["lr_body"] = body
    sc.pop("n_solid", None)
    sc["n_body"] = len(xyz)
    return sc


# --------------------------------------------------- procedural meshes ---
# Closed triangle meshes, counter-clockwise seen from outside (outward
# normals), as vertex array float64 [n][3] and triangle array int32 [m][3].
# They are input geometry for the volume sampler of Sec. 4 (whose particles
# the paper seeds from artists' meshes, not available here).

def box_mesh(lo, hi):
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    V = np.array([[x, y, z] for z in (lo[2], hi[2]) for y in (lo[1], hi[1]) for x in (lo[0], hi[0])])
    # vertex k = x + 2 y + 4 z (bits); faces as quads (a, b, c, d) counter-clockwise from outside
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    T = [(a, b, c) for a, b, c, d in quads] + [(a, c, d) for a, b, c, d in quads]
    return V, np.array(T, np.int32)


def prism_mesh(cx, cy, radius, z0, z1, n=24, apex=None):
    """A closed n-gon prism (a cylinder's stand-in) from z0 to z1; with apex
    (a height above z1) a cone on top instead of the flat cap."""
    ang = 2 * np.pi * np.arange(n) / n
    ring = np.stack([cx + radius * np.cos(ang), cy + radius * np.sin(ang)], 1)
    V = [[x, y, z0] for x, y in ring] + [[x, y, z1] for x, y in ring] + [[cx, cy, z0]]
    bot = 2 * n
    T = []
    for k in range(n):
        k1 = (k + 1) % n
        T += [(k, k1, n + k1), (k, n + k1, n + k)]     # side
        T += [(bot, k1, k)]                             # bottom (normal down)
    if apex is None:
        V.append([cx, cy, z1])
        top = 2 * n + 1
        T += [(top, n + k, n + (k + 1) % n) for k in range(n)]
    else:
        V.append([cx, cy, z1 + apex])
        top = 2 * n + 1
        T += [(top, n + k, n + (k + 1) % n) for k in range(n)]
    return np.array(V, float), np.array(T, np.int32)


def icosphere(center, radius, subdiv=2):
    """A subdivided icosahedron with its vertices on the sphere."""
    t = (1 + 5 ** 0.5) / 2
    V = [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]]
    V = [list(np.array(v) / np.linalg.norm(v)) for v in V]
    T = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        mid = {}

        def m(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = np.array(V[a]) + np.array(V[b])
                V.append(list(p / np.linalg.norm(p)))
                mid[key] = len(V) - 1
            return mid[key]
        T = [t2 for a, b, c in T for t2 in ((a, m(a, b), m(c, a)), (b, m(b, c), m(a, b)), (c, m(c, a), m(b, c)),
                                             (m(a, b), m(b, c), m(c, a)))]
    return np.asarray(center, float) + radius * np.array(V), np.array(T, np.int32)


def merge_meshes(parts):
    """Several closed meshes as one triangle soup (overlaps allowed: their
    union is where the winding number exceeds 1/2)."""
    Vs, Ts, off = [], [], 0
    for V, T in parts:
        Vs.append(V)
        Ts.append(T + off)
        off += len(V)
    return np.concatenate(Vs), np.concatenate(Ts).astype(np.int32)


def castle_mesh(base=(0.5, 0.5, 0.0), size=0.6, height=0.2):
    """A sand castle: a square base, a central keep, four round corner towers
    with cone roofs (overlapping closed parts)."""
    cx, cy, z0 = base
    h2 = size / 2
    parts = [box_mesh((cx - h2, cy - h2, z0), (cx + h2, cy + h2, z0 + height)),
             box_mesh((cx - 0.2 * size, cy - 0.2 * size, z0 + 0.5 * height),
                      (cx + 0.2 * size, cy + 0.2 * size, z0 + 2.0 * height))]
    for sx in (-1, 1):
        for sy in (-1, 1):
            parts.append(prism_mesh(cx + sx * 0.8 * h2, cy + sy * 0.8 * h2, 0.12 * size, z0, z0 + 1.6 * height,
                                    n=20, apex=0.6 * height))
    return merge_meshes(parts)


def volume_candidates(V, r, per_cell=6.0, seed=SEED_BASE + 10):
    """Uniform random candidate positions in the bounding box of the mesh
    vertices for the volume sampler: about per_cell candidates per cell of
    side 2 r / sqrt(3)."""
    lo, hi = V.min(0), V.max(0)
    h = 2 * r / math.sqrt(3)
    n = int(math.ceil(per_cell * float(np.prod(hi - lo)) / h ** 3))
    rng = np.random.default_rng(seed)
    return lo + (hi - lo) * rng.random((n, 3))


def castle_scene(sample, seed=SEED_BASE + 11, size=1.25, height=0.4, r_low=0.02, r_high=0.0075,
                 boulder_radius=0.1, boulder_velocity=(-3.0, 0.0, -1.0), per_cell=4.0, dt=1.0 / 240.0, iters=8,
                 boulder=True):
    """The sand-castle scene of Sec. 5 (a rigid body hurled into a castle):
    LR grains and HR particles sampled from the castle mesh, a boulder's LR
    particles sampled from an icosphere (density 5000 kg/m^3, one rigid
    body) flying at the castle.  `sample(V, T, candidates, r)` is the volume
    sampler (it returns the indices of the chosen candidates); this module
    only draws the candidates.  The paper's castle: 10k LR (r_LR = 0.02) /
    207k HR (r_HR = 0.0075); the defaults give about that."""
    V, T = castle_mesh(base=(0.5 * size + 0.3, 0.5 * size + 0.3, 0.0), size=size, height=height)
    lr = volume_candidates(V, r_low, per_cell, seed)
    lr = lr[sample(V, T, lr, r_low)]
    hr = volume_candidates(V, r_high, per_cell, seed + 1)
    hr = hr[sample(V, T, hr, r_high)]
    c = np.array([V[:, 0].max() + 0.3, 0.5 * (V[:, 1].min() + V[:, 1].max()), 0.6 * V[:, 2].max()])
    Vb, Tb = icosphere(c, boulder_radius, 2)
    bd = volume_candidates(Vb, r_low, per_cell, seed + 2)
    bd = bd[sample(Vb, Tb, bd, r_low)] if boulder else np.zeros((0, 3))
    m_g = RHO * 4.0 / 3.0 * math.pi * r_low ** 3
    m_b = 5000.0 * 4.0 / 3.0 * math.pi * r_low ** 3
    lr_pos = np.concatenate([_pack(lr, np.float32(1.0 / m_g)), _pack(bd, np.float32(1.0 / m_b))])
    lr_vel = np.zeros((len(lr_pos), 4), np.float32)
    lr_vel[len(lr):, :3] = np.asarray(boulder_velocity, np.float32)
    body = np.zeros(len(lr_pos), np.uint32)
    body[len(lr):] = 1
    hr_pos = _pack(hr, 0.0)
    hr_pos[:, 3] = hr_ids(len(hr))
    lo = [0.0, 0.0, 0.0]
    hi = [float(V[:, 0].max() + 1.0), float(V[:, 1].max() + 0.3), float(max(V[:, 2].max(), c[2]) + 0.5)]
    ratio = max(1, int(round(len(hr) / max(len(lr), 1))))
    sc = dict(name="castle", seed=seed, box_lo=lo, box_hi=hi, r_low=float(r_low), r_high=float(r_high),
              ratio=ratio, sdfs=[box_interior(lo, hi)], gravity=GRAVITY, mu_s=MU_S, mu_k=MU_K, dt=float(dt),
              iters=int(iters), lr_pos=lr_pos, lr_vel=lr_vel, hr_pos=hr_pos,
              hr_vel=np.zeros((len(hr_pos), 4), np.float32), n_body=len(bd))
    if len(bd):
        sc["lr_body"] = body
    return sc


def surface_candidates(V, T, r, per_cell=6.0, seed=SEED_BASE + 12):
    """Uniform random candidate positions on the triangles of a mesh (each
    triangle chosen with probability proportional to its area) for the
    surface sampler: about per_cell candidates per area h^2 of a cell of
    side h = 2 r / sqrt(3)."""
    A, B, C = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(B - A, C - A), axis=1)
    h = 2 * r / math.sqrt(3)
    n = int(math.ceil(per_cell * float(area.sum()) / h ** 2))
    rng = np.random.default_rng(seed)
    tri = rng.choice(len(T), size=n, p=area / area.sum())
    u, v = rng.random(n), rng.random(n)
    flip = u + v > 1.0
    u[flip], v[flip] = 1.0 - u[flip], 1.0 - v[flip]
    return A[tri] + u[:, None] * (B[tri] - A[tri]) + v[:, None] * (C[tri] - A[tri])


def digging_mesh_bucket(sample_surface, seed=SEED_BASE + 13, t=0.0, **kw):
    """The digging bed with the bucket as particles of inverse mass 0 sampled
    on the surface of its box mesh by `sample_surface(V, candidates, r)` (the
    surface sampler, returning the chosen candidates' indices), moving with
    the bucket's velocity at time t, in place of the bucket SDF."""
    sc = digging(**kw)
    c, u = bucket_pose(t)
    V, T = box_mesh(np.asarray(c) - BUCKET_HALF, np.asarray(c) + BUCKET_HALF)
    cand = surface_candidates(V, T, sc["r_low"], seed=seed)
    pts = cand[sample_surface(V, cand, sc["r_low"])]
    sc = with_solids(sc, pts, u, seed)
    sc["sdfs"] = [sc["sdfs"][0]]
    sc.pop("bucket_index", None)
    return sc
