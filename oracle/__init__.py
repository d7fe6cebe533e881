"""FP64 CPU oracle for the two-level granular method (arXiv 2308.01629).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product library never
imports this package and this package never imports the product; the two
meet only through the seeded arrays of the ``scenes`` package.

The arithmetic lives in ``gs_oracle.c`` (plain C, double precision, compiled
with ``-ffp-contract=off``); this module compiles it with gcc on first use and
marshals numpy arrays through ctypes.  Each wrapper names the passage of the
paper the C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

SDF_STRIDE = 20
UP_KEYS = ["r_low", "r_high", "dt", "gx", "gy", "gz", "c1", "c2", "eps_w", "eps_x"]
PB_KEYS = ["r", "dt", "gx", "gy", "gz", "mu_s", "mu_k", "n_stab", "iters", "mass_k",
           "ground_z", "rc", "friction_mode", "eps_x", "eps_impact"]

_lib = None


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into _build/liboracle.so (OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_max_threads.restype = ctypes.c_int
        L.or_grid.argtypes = [ctypes.c_double, P, P, P, P, P, P]
        L.or_grid.restype = ctypes.c_int
        L.or_cell_keys.argtypes = [P, ctypes.c_long, P, ctypes.c_float, P, ctypes.c_int, P]
        L.or_counting_sort.argtypes = [P, ctypes.c_long, ctypes.c_long, P, P]
        L.or_counting_sort.restype = ctypes.c_int
        L.or_weight.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_weight.restype = ctypes.c_double
        L.or_sdf_eval.argtypes = [P, P, P, P, P, ctypes.c_double]
        L.or_sdf_eval.restype = ctypes.c_int
        L.or_upsample.argtypes = [P, P, ctypes.c_long, P, P, ctypes.c_long, P, ctypes.c_long,
                                  P, ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, P]
        L.or_upsample.restype = ctypes.c_int
        L.or_upsample_solid.argtypes = [P, P, P, ctypes.c_long, P, P, ctypes.c_long, P, ctypes.c_long,
                                        P, ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, P]
        L.or_upsample_solid.restype = ctypes.c_int
        L.or_pbd_step.argtypes = [P, P, P, ctypes.c_long, P, ctypes.c_int, P, ctypes.c_int, P, P]
        L.or_pbd_step.restype = ctypes.c_int
        L.or_pbd_pass.argtypes = [P, P, P, P, P, ctypes.c_long, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                  P, P]
        L.or_pbd_pass.restype = ctypes.c_int
        L.or_pbd_step_mu.argtypes = [P, P, P, ctypes.c_long, P, ctypes.c_int, P, ctypes.c_int, P, P, P]
        L.or_pbd_step_mu.restype = ctypes.c_int
        L.or_pbd_step_bodies.argtypes = [P, P, P, ctypes.c_long, P, ctypes.c_int, P, ctypes.c_int, P, P, P,
                                         ctypes.c_int, P, P]
        L.or_pbd_step_bodies.restype = ctypes.c_int
        L.or_polar_rotation.argtypes = [P, P]
        L.or_polar_rotation.restype = ctypes.c_int
        L.or_pairs_within.argtypes = [P, ctypes.c_long, P, ctypes.c_long, ctypes.c_double, P, P, ctypes.c_long]
        L.or_pairs_within.restype = ctypes.c_long
        L.or_upsample_vjp.argtypes = [P, P, ctypes.c_long, P, P, ctypes.c_long, P, ctypes.c_int, P, P, P,
                                      P, P, P, P]
        L.or_upsample_vjp.restype = ctypes.c_int
        L.or_upsample_vjp_tape.argtypes = [P, P, ctypes.c_long, P, P, ctypes.c_long, P, ctypes.c_int, P, P, P, P,
                                           P, P, P, P]
        L.or_upsample_vjp_tape.restype = ctypes.c_int
        L.or_pbd_step_vjp_tape.argtypes = [P, P, P, ctypes.c_long, P, ctypes.c_int, P, P, ctypes.c_long, P, P, P,
                                           P]
        L.or_pbd_step_vjp_tape.restype = ctypes.c_int
        L.or_pbd_step_vjp.argtypes = [P, P, P, ctypes.c_long, P, ctypes.c_int, P, P, P, P, P]
        L.or_pbd_step_vjp.restype = ctypes.c_int
        L.or_upsample_tape.argtypes = [P, P, ctypes.c_long, P, P, ctypes.c_long, P, ctypes.c_int, P, ctypes.c_int,
                                       P, P, P]
        L.or_upsample_tape.restype = ctypes.c_int
        L.or_pbd_step_tape.argtypes = [P, P, P, ctypes.c_long, P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_long,
                                       P]
        L.or_pbd_step_tape.restype = ctypes.c_int
        L.or_upsample_plain.argtypes = [P, P, ctypes.c_long, P, P, ctypes.c_long, P, ctypes.c_int, P, P, P]
        L.or_upsample_plain.restype = ctypes.c_int
        L.or_pbd_step_plain.argtypes = [P, P, P, ctypes.c_long, P, ctypes.c_int, P]
        L.or_pbd_step_plain.restype = ctypes.c_int
        L.or_winding_number.argtypes = [P, P, ctypes.c_long, P]
        L.or_winding_number.restype = ctypes.c_double
        L.or_sample_grid.argtypes = [P, ctypes.c_long, ctypes.c_double, P, P, P]
        L.or_sample_volume.argtypes = [P, ctypes.c_long, P, ctypes.c_long, P, ctypes.c_long, ctypes.c_double, P,
                                       ctypes.c_long, P]
        L.or_sample_volume.restype = ctypes.c_long
        L.or_sample_surface.argtypes = [P, ctypes.c_long, P, ctypes.c_long, ctypes.c_double, P, ctypes.c_long]
        L.or_sample_surface.restype = ctypes.c_long
        L.or_pairs_within_grid.argtypes = L.or_pairs_within.argtypes
        L.or_pairs_within_grid.restype = ctypes.c_long
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, cols=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if cols is not None:
        a = np.ascontiguousarray(a.reshape(-1, cols))
    return a


def set_threads(n: int) -> None:
    _L().or_set_threads(int(n))


def max_threads() -> int:
    return int(_L().or_max_threads())


# ---------------------------------------------------------------- grid ---
def grid(r_low, box_lo, box_hi):
    """Cell contract of the neighbour grid: (origin f32[3], h, inv_h, dims)."""
    o = np.zeros(3, np.float32)
    h = np.zeros(1, np.float32)
    ih = np.zeros(1, np.float32)
    dims = np.zeros(3, np.int32)
    rc = _L().or_grid(float(r_low), _ptr(_f64(box_lo)), _ptr(_f64(box_hi)), _ptr(o), _ptr(h),
                      _ptr(ih), _ptr(dims))
    if rc != 0:
        raise ValueError("invalid grid arguments")
    return o, float(h[0]), np.float32(ih[0]), dims


def cell_keys(pos4, o, inv_h, dims, fine=False):
    """Cell id (or 8*cell + octant when fine) of each float4 position."""
    pos4 = np.ascontiguousarray(np.asarray(pos4, dtype=np.float32).reshape(-1, 4))
    keys = np.zeros(len(pos4), np.uint32)
    _L().or_cell_keys(_ptr(pos4), len(pos4), _ptr(np.asarray(o, np.float32)), ctypes.c_float(inv_h),
                      _ptr(np.asarray(dims, np.int32)), int(bool(fine)), _ptr(keys))
    return keys


def counting_sort(keys, nkeys):
    """Stable counting sort: (sorted_idx, start[nkeys+1])."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    idx = np.zeros(len(keys), np.uint32)
    start = np.zeros(int(nkeys) + 1, np.uint32)
    rc = _L().or_counting_sort(_ptr(keys), len(keys), int(nkeys), _ptr(idx), _ptr(start))
    if rc != 0:
        raise ValueError("key out of range")
    return idx, start


# ----------------------------------------------------------- upsampling ---
def weight(d2, r_low):
    """Sec. 4 distance weight w = max(0, (1 - d^2 / (9 r_LR^2))^3)."""
    return _L().or_weight(float(d2), float(r_low))


def sdf_eval(rec, x, eps=0.0):
    rec = _f64(rec)
    phi = np.zeros(6)
    n = np.zeros(18)
    tie = np.zeros(1, np.int32)
    nc = _L().or_sdf_eval(_ptr(rec), _ptr(_f64(x)), _ptr(phi), _ptr(n), _ptr(tie), float(eps))
    return phi[:nc], n[:3 * nc].reshape(nc, 3), bool(tie[0])


def _prm(d, keys):
    return np.array([float(d[k]) for k in keys], dtype=np.float64)


def upsample(lr_x, lr_v, hr_x, hr_v, sdf, prm, sub=None, mode=0, solid=None):
    """One HR frame of Sec. 4 for HR particles ``sub`` (all when None).

    ``prm`` holds r_low, r_high, dt, gx, gy, gz, c1, c2, eps_w, eps_x.
    ``solid`` (optional, one flag per LR particle) marks LR particles of
    infinite mass (sampled boundaries, rigid bodies): they count in the
    weights unless no grain reaches the HR particle.
    Returns dict(x, v, flag, alt_x, alt_v, diag) with diag = (S, wmax, alpha, n,
    sens_x, sens_v).
    """
    lr_x, lr_v = _f64(lr_x, 3), _f64(lr_v, 3)
    hr_x, hr_v = _f64(hr_x, 3), _f64(hr_v, 3)
    sdf = _f64(sdf, SDF_STRIDE) if sdf is not None and len(sdf) else np.zeros((0, SDF_STRIDE))
    p = _prm(prm, UP_KEYS)
    subv = None if sub is None else np.ascontiguousarray(sub, dtype=np.int64)
    n = len(hr_x) if subv is None else len(subv)
    out = dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), flag=np.zeros(n, np.int32),
               alt_x=np.zeros((n, 3)), alt_v=np.zeros((n, 3)), diag=np.zeros((n, 6)))
    args = (_ptr(hr_x), _ptr(hr_v), len(hr_x), _ptr(subv), 0 if subv is None else len(subv), _ptr(sdf), len(sdf),
            _ptr(p), int(mode), _ptr(out["x"]), _ptr(out["v"]), _ptr(out["flag"]), _ptr(out["alt_x"]),
            _ptr(out["alt_v"]), _ptr(out["diag"]))
    if solid is None:
        rc = _L().or_upsample(_ptr(lr_x), _ptr(lr_v), len(lr_x), *args)
    else:
        solid = np.ascontiguousarray(np.asarray(solid).astype(np.uint8))
        if len(solid) != len(lr_x):
            raise ValueError("solid needs one flag per LR particle")
        rc = _L().or_upsample_solid(_ptr(lr_x), _ptr(lr_v), _ptr(solid), len(lr_x), *args)
    if rc != 0:
        raise RuntimeError(f"or_upsample failed ({rc})")
    return out


def upsample_vjp(lr_x, lr_v, hr_x, hr_v, sdf, prm, gx, gv, tape=None):
    """Reverse mode of ``upsample``: given dL/dx^{t+1}, dL/dv^{t+1} returns
    (dL/dX_LR, dL/dV_LR, dL/dx_HR, dL/dv_HR) for the forward branch
    decisions (contact normals held fixed), or for the decisions of a tape
    (``upsample_tape``'s layout) when one is given."""
    lr_x, lr_v = _f64(lr_x, 3), _f64(lr_v, 3)
    hr_x, hr_v = _f64(hr_x, 3), _f64(hr_v, 3)
    sdf = _f64(sdf, SDF_STRIDE) if sdf is not None and len(sdf) else np.zeros((0, SDF_STRIDE))
    gx, gv = _f64(gx, 3), _f64(gv, 3)
    out = [np.zeros_like(lr_x), np.zeros_like(lr_v), np.zeros_like(hr_x), np.zeros_like(hr_v)]
    args = (_ptr(lr_x), _ptr(lr_v), len(lr_x), _ptr(hr_x), _ptr(hr_v), len(hr_x), _ptr(sdf), len(sdf),
            _ptr(_prm(prm, UP_KEYS)))
    if tape is None:
        rc = _L().or_upsample_vjp(*args, _ptr(gx), _ptr(gv), *[_ptr(o) for o in out])
    else:
        tape = np.ascontiguousarray(tape, np.uint32)
        if tape.shape != (len(hr_x), 4):
            raise ValueError("tape does not match the HR count")
        rc = _L().or_upsample_vjp_tape(*args, _ptr(tape), _ptr(gx), _ptr(gv), *[_ptr(o) for o in out])
    if rc != 0:
        raise RuntimeError("or_upsample_vjp failed")
    return tuple(out)


# ------------------------------------------------------------- LR step ---
def polar_rotation(C):
    """Rotation of the polar decomposition of the 3 x 3 matrix C."""
    C = _f64(C).reshape(3, 3).copy()
    R = np.zeros((3, 3))
    if _L().or_polar_rotation(_ptr(C), _ptr(R)) != 0:
        raise ValueError("degenerate matrix")
    return R


def body_rest_offsets(x, inv_m, body):
    """Offsets of every body particle from its body's centre of mass (masses
    1 / inv_m) in the configuration x; 0 for grains (body 0)."""
    x, inv_m, body = _f64(x, 3), _f64(inv_m), np.asarray(body, np.int64)
    xo = np.zeros_like(x)
    for b in np.unique(body[body > 0]):
        sel = body == b
        m = 1.0 / inv_m[sel]
        xo[sel] = x[sel] - (m[:, None] * x[sel]).sum(0) / m.sum()
    return xo


def upsample_plain(lr_x, lr_v, hr_x, hr_v, sdf, prm):
    """One HR frame of Sec. 4 as its plain definition (no decision margins
    or tapes; parallel over HR particles).  Returns (x, v)."""
    lr_x, lr_v = _f64(lr_x, 3), _f64(lr_v, 3)
    hr_x, hr_v = _f64(hr_x, 3), _f64(hr_v, 3)
    sdf = _f64(sdf, SDF_STRIDE) if sdf is not None and len(sdf) else np.zeros((0, SDF_STRIDE))
    p = _prm(prm, UP_KEYS)
    ox, ov = np.zeros_like(hr_x), np.zeros_like(hr_v)
    rc = _L().or_upsample_plain(_ptr(lr_x), _ptr(lr_v), len(lr_x), _ptr(hr_x), _ptr(hr_v), len(hr_x), _ptr(sdf),
                                len(sdf), _ptr(p), _ptr(ox), _ptr(ov))
    if rc != 0:
        raise RuntimeError(f"or_upsample_plain failed ({rc})")
    return ox, ov


def pbd_step_plain(x, v, inv_m, sdf, prm):
    """One LR step of Algorithm 1 as its plain definition (no decision
    margins or tapes; each particle gathers its own corrections, parallel
    over particles).  Returns (x, v)."""
    x, v = _f64(x, 3).copy(), _f64(v, 3).copy()
    inv_m = _f64(inv_m)
    sdf = _f64(sdf, SDF_STRIDE) if sdf is not None and len(sdf) else np.zeros((0, SDF_STRIDE))
    p = _prm(prm, PB_KEYS)
    rc = _L().or_pbd_step_plain(_ptr(x), _ptr(v), _ptr(inv_m), len(x), _ptr(sdf), len(sdf), _ptr(p))
    if rc != 0:
        raise RuntimeError(f"or_pbd_step_plain failed ({rc})")
    return x, v


def pbd_step(x, v, inv_m, sdf, prm, mode=0, mu=None, bodies=None):
    """One LR time step of Algorithm 1.  Returns (x, v, suspect, stats).
    mu (N x 2: mu_s, mu_k per particle), when given, replaces the step's
    friction coefficients; pairs use the cross coefficients of Sec. 3.
    bodies = (body, xo): body id per particle (0: grain, 1..B: rigid body)
    and rest offsets (body_rest_offsets); each body is shape-matched in the
    solver passes (Sec. 3)."""
    x, v = _f64(x, 3).copy(), _f64(v, 3).copy()
    inv_m = _f64(inv_m)
    sdf = _f64(sdf, SDF_STRIDE) if sdf is not None and len(sdf) else np.zeros((0, SDF_STRIDE))
    p = _prm(prm, PB_KEYS)
    sus = np.zeros(len(x), np.int32)
    stats = np.zeros(5, np.int64)
    if bodies is not None:
        body = np.ascontiguousarray(np.asarray(bodies[0], np.int32))
        xo = _f64(bodies[1], 3)
        muv = None if mu is None else _f64(mu, 2)
        rc = _L().or_pbd_step_bodies(_ptr(x), _ptr(v), _ptr(inv_m), len(x), _ptr(sdf), len(sdf), _ptr(p),
                                     int(mode), _ptr(muv), _ptr(body), _ptr(xo), int(body.max(initial=0)),
                                     _ptr(sus), _ptr(stats))
    elif mu is None:
        rc = _L().or_pbd_step(_ptr(x), _ptr(v), _ptr(inv_m), len(x), _ptr(sdf), len(sdf), _ptr(p),
                              int(mode), _ptr(sus), _ptr(stats))
    else:
        mu = _f64(mu, 2)
        if len(mu) != len(x):
            raise ValueError("mu must hold one (mu_s, mu_k) pair per particle")
        rc = _L().or_pbd_step_mu(_ptr(x), _ptr(v), _ptr(inv_m), len(x), _ptr(sdf), len(sdf), _ptr(p),
                                 int(mode), _ptr(mu), _ptr(sus), _ptr(stats))
    if rc != 0:
        raise RuntimeError(f"or_pbd_step failed ({rc})")
    return x, v, sus.astype(bool), dict(pairs=int(stats[0]), significant=int(stats[1]),
                                        max_candidates=int(stats[2]), active=int(stats[3]),
                                        ambiguous=int(stats[4]))


def pbd_pass(x, xt, x0, xt0, inv_m, sdf, prm, stab, mode=1):
    """One Jacobi pass of Algorithm 1 (Sec. 3) from a given state: x (start-
    of-step positions as stabilized so far) and xt (predictions as corrected
    so far) are the pass's input; x0 (step start) fixes the height-scaled
    masses and xt0 (the step's predictions) the candidate pairs; stab selects
    a stabilization pass (contacts on x, applied to x and xt) or a solver pass
    (Eqs. 1-4 on xt).  Returns (x, xt, suspect, stats); suspect marks the
    particles whose result hangs on a decision within this pass's margins."""
    x, xt = _f64(x, 3).copy(), _f64(xt, 3).copy()
    x0, xt0 = _f64(x0, 3), _f64(xt0, 3)
    inv_m = _f64(inv_m)
    sdf = _f64(sdf, SDF_STRIDE) if sdf is not None and len(sdf) else np.zeros((0, SDF_STRIDE))
    sus = np.zeros(len(x), np.int32)
    stats = np.zeros(5, np.int64)
    rc = _L().or_pbd_pass(_ptr(x), _ptr(xt), _ptr(x0), _ptr(xt0), _ptr(inv_m), len(x), _ptr(sdf), len(sdf),
                          _ptr(_prm(prm, PB_KEYS)), int(bool(stab)), int(mode), _ptr(sus), _ptr(stats))
    if rc != 0:
        raise RuntimeError(f"or_pbd_pass failed ({rc})")
    return x, xt, sus.astype(bool), dict(pairs=int(stats[0]), significant=int(stats[1]), active=int(stats[3]),
                                         ambiguous=int(stats[4]))


def pbd_step_vjp(x, v, inv_m, sdf, prm, gx, gv, tape=None):
    """Reverse mode of ``pbd_step`` (brute-force pairs): given dL/dx_out,
    dL/dv_out returns (dL/dx, dL/dv) at the start of the step for the
    forward pass's branch decisions, or, when a tape (``pbd_step_tape``'s
    layout) is given, for its candidate pairs and decisions."""
    x, v = _f64(x, 3), _f64(v, 3)
    inv_m = _f64(inv_m)
    sdf = _f64(sdf, SDF_STRIDE) if sdf is not None and len(sdf) else np.zeros((0, SDF_STRIDE))
    gx, gv = _f64(gx, 3), _f64(gv, 3)
    ox, ov = np.zeros_like(x), np.zeros_like(v)
    if tape is not None:
        tape = np.ascontiguousarray(tape, np.uint8)
        rc = _L().or_pbd_step_vjp_tape(_ptr(x), _ptr(v), _ptr(inv_m), len(x), _ptr(sdf), len(sdf),
                                       _ptr(_prm(prm, PB_KEYS)), _ptr(tape), tape.size, _ptr(gx), _ptr(gv), _ptr(ox),
                                       _ptr(ov))
        if rc != 0:
            raise RuntimeError(f"or_pbd_step_vjp_tape failed ({rc})")
        return ox, ov
    rc = _L().or_pbd_step_vjp(_ptr(x), _ptr(v), _ptr(inv_m), len(x), _ptr(sdf), len(sdf), _ptr(_prm(prm, PB_KEYS)),
                              _ptr(gx), _ptr(gv), _ptr(ox), _ptr(ov))
    if rc != 0:
        raise RuntimeError("or_pbd_step_vjp failed")
    return ox, ov


# ------------------------------------------------------- decision tapes ---
# The method is piecewise smooth (blend branch, largest weight, contact
# activation, static/kinetic friction, SDF active set).  A tape records the
# decisions of one evaluation; replaying it evaluates the recorded branch of
# every decision, i.e. the smooth piece that contains the recording point,
# whose derivative the reverse modes compute.
TAPE_RECORD, TAPE_REPLAY = 1, 2


def upsample_tape(lr_x, lr_v, hr_x, hr_v, sdf, prm, tape=None):
    """One HR frame (Sec. 4) recording its decisions (tape None) or replaying
    them.  Returns (x, v, tape)."""
    lr_x, lr_v = _f64(lr_x, 3), _f64(lr_v, 3)
    hr_x, hr_v = _f64(hr_x, 3), _f64(hr_v, 3)
    sdf = _f64(sdf, SDF_STRIDE) if sdf is not None and len(sdf) else np.zeros((0, SDF_STRIDE))
    mode = TAPE_REPLAY if tape is not None else TAPE_RECORD
    if tape is None:
        tape = np.zeros((len(hr_x), 4), np.uint32)
    elif tape.shape != (len(hr_x), 4):
        raise ValueError("tape does not match the HR count")
    ox, ov = np.zeros_like(hr_x), np.zeros_like(hr_v)
    rc = _L().or_upsample_tape(_ptr(lr_x), _ptr(lr_v), len(lr_x), _ptr(hr_x), _ptr(hr_v), len(hr_x), _ptr(sdf),
                               len(sdf), _ptr(_prm(prm, UP_KEYS)), mode, _ptr(tape), _ptr(ox), _ptr(ov))
    if rc != 0:
        raise RuntimeError(f"or_upsample_tape failed ({rc})")
    return ox, ov, tape


def pbd_step_tape(x, v, inv_m, sdf, prm, tape=None):
    """One LR step (Algorithm 1) recording its decisions (tape None) or
    replaying them.  Returns (x, v, tape)."""
    x0, v0 = _f64(x, 3), _f64(v, 3)
    inv_m = _f64(inv_m)
    sdf = _f64(sdf, SDF_STRIDE) if sdf is not None and len(sdf) else np.zeros((0, SDF_STRIDE))
    p = _prm(prm, PB_KEYS)
    mode = TAPE_REPLAY if tape is not None else TAPE_RECORD
    buf = tape if tape is not None else np.zeros(32 + 64 * len(x0) * 8, np.uint8)
    need = ctypes.c_long(0)
    while True:
        xo, vo = x0.copy(), v0.copy()
        rc = _L().or_pbd_step_tape(_ptr(xo), _ptr(vo), _ptr(inv_m), len(xo), _ptr(sdf), len(sdf), _ptr(p), mode,
                                   _ptr(buf), buf.size, ctypes.byref(need))
        if rc == -3 and mode == TAPE_RECORD and need.value > buf.size:
            buf = np.zeros(need.value, np.uint8)
            continue
        if rc != 0:
            raise RuntimeError(f"or_pbd_step_tape failed ({rc})")
        break
    return xo, vo, (buf[:need.value].copy() if mode == TAPE_RECORD else buf)


# ------------------------------------------- CFL-limited LR substeps ---
# Sec. 5.2: the LR simulation runs with a default time step that the CFL
# condition shortens when the grains move fast, and one HR frame covers many
# LR steps.  Reading used (the paper gives no formula): a step may move no
# grain by more than cfl times its diameter, dt <= cfl 2 r_LR / max |v|, and
# never exceeds the default dt_max; the frame time left is split into the
# fewest equal steps within that limit, decided again after every step from
# the new velocities; at most max_sub steps per frame (the last one takes
# what is left).  The decisions fix an integer (the step count), so they are
# taken in float32 with correctly rounded operations, as the library does.
def cfl_rate(v, r_low):
    """max over particles of |v| / (2 r_LR) in float32 (0 for no particles);
    r_low may be one value or one per particle."""
    v = np.asarray(v, np.float32)
    if len(v) == 0:
        return np.float32(0.0)
    v = v.reshape(len(v), -1)[:, :3]
    s = (v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2]
    d = np.float32(2.0) * np.asarray(r_low, np.float32)
    q = np.sqrt(s) / d
    return np.float32(q.max())


def cfl_substep(t_rem, rate, dt_max, cfl, left):
    """(dt, more): the next substep for t_rem seconds of frame left, the
    current rate max |v| / (2 r_LR) and `left` >= 1 steps allowed; more is
    False for the frame's last step."""
    f = np.float32
    t_rem, rate, dt_max, cfl = f(t_rem), f(rate), f(dt_max), f(cfl)
    if not np.isfinite(rate):
        lim = f(0.0)
    elif rate > 0:
        lim = min(dt_max, f(cfl / rate))
    else:
        lim = dt_max
    with np.errstate(divide="ignore"):
        q = f(t_rem / lim) if lim > 0 else f(np.inf)
    n = left if (left <= 1 or not q < f(left)) else max(1, int(np.ceil(q)))
    return f(t_rem / f(n)), n > 1


def frame_adaptive(x, v, inv_m, sdf, prm, dt_frame, dt_max, cfl, max_sub, mode=1):
    """LR steps of Algorithm 1 covering one frame of dt_frame with the CFL
    limit above.  Returns (x, v, dts) with dts the float32 substeps."""
    x, v = _f64(x, 3), _f64(v, 3)
    t_rem = np.float32(dt_frame)
    dts = []
    while True:
        dt, more = cfl_substep(t_rem, cfl_rate(v, prm["r"]), dt_max, cfl, max_sub - len(dts))
        step = dict(prm, dt=float(dt))
        x, v, _, _ = pbd_step(x, v, inv_m, sdf, step, mode=mode)
        dts.append(dt)
        if not more:
            return x, v, np.array(dts, np.float32)
        t_rem = np.float32(t_rem - dt)


def rollout(lr_x, lr_v, inv_m, hr_x, hr_v, sdf, pb, up, frames, n_sub=1, tapes=None):
    """`frames` frames of the two-level method: per frame n_sub LR steps of
    Algorithm 1 (parameters pb, pb["dt"] each), then one HR frame of Sec. 4
    (parameters up) driven by the new LR state.  Decisions are recorded
    (tapes None) or replayed from the tapes of an earlier call.  Returns a
    dict with the final state, the per-operation inputs (for rollout_vjp)
    and the tapes."""
    X, V, x, v = _f64(lr_x, 3), _f64(lr_v, 3), _f64(hr_x, 3), _f64(hr_v, 3)
    ops, out_tapes = [], []
    k = 0
    for _ in range(frames):
        for _ in range(n_sub):
            ops.append(("lr", X, V))
            X, V, t = pbd_step_tape(X, V, inv_m, sdf, pb, None if tapes is None else tapes[k])
            out_tapes.append(t)
            k += 1
        ops.append(("hr", X, V, x, v))
        x, v, t = upsample_tape(X, V, x, v, sdf, up, None if tapes is None else tapes[k])
        out_tapes.append(t)
        k += 1
    return dict(lr_x=X, lr_v=V, hr_x=x, hr_v=v, ops=ops, tapes=out_tapes)


def rollout_vjp(ro, inv_m, sdf, pb, up, g_hr_x, g_hr_v, g_lr_x=None, g_lr_v=None, replay=False):
    """Reverse mode of ``rollout`` by the chain rule over its operations, last
    first (``pbd_step_vjp`` and ``upsample_vjp`` at the recorded inputs).
    With replay, every operation's reverse mode takes its decisions from the
    rollout's tapes (ro["tapes"], one per operation in order): the
    derivative of the replayed rollout.  Returns (dL/dlr_x, dL/dlr_v,
    dL/dhr_x, dL/dhr_v) at the initial state."""
    a, b = _f64(g_hr_x, 3).copy(), _f64(g_hr_v, 3).copy()
    GX = np.zeros_like(ro["lr_x"]) if g_lr_x is None else _f64(g_lr_x, 3).copy()
    GV = np.zeros_like(ro["lr_v"]) if g_lr_v is None else _f64(g_lr_v, 3).copy()
    tapes = ro["tapes"] if replay else [None] * len(ro["ops"])
    for op, tape in zip(reversed(ro["ops"]), reversed(tapes)):
        if op[0] == "hr":
            _, X, V, x, v = op
            gX, gV, a, b = upsample_vjp(X, V, x, v, sdf, up, a, b, tape=tape)
            GX += gX
            GV += gV
        else:
            _, X, V = op
            GX, GV = pbd_step_vjp(X, V, inv_m, sdf, pb, GX, GV, tape=tape)
    return GX, GV, a, b


def pairs_within(a, b, R, use_grid=False):
    """All (i, j) with |a_i - b_j| < R, sorted by (i, j)."""
    a, b = _f64(a, 3), _f64(b, 3)
    fn = _L().or_pairs_within_grid if use_grid else _L().or_pairs_within
    n = fn(_ptr(a), len(a), _ptr(b), len(b), float(R), None, None, 0)
    if n < 0:
        raise RuntimeError("pair search failed")
    oi = np.zeros(max(n, 1), np.int64)
    oj = np.zeros(max(n, 1), np.int64)
    fn(_ptr(a), len(a), _ptr(b), len(b), float(R), _ptr(oi), _ptr(oj), n)
    return oi[:n], oj[:n]


# ------------------------------------------------- initial sampling (Sec. 4) ---
def _mesh(V, T):
    V = _f64(V, 3)
    T = np.ascontiguousarray(np.asarray(T, dtype=np.int32).reshape(-1, 3))
    if len(T) and (T.min() < 0 or T.max() >= len(V)):
        raise ValueError("triangle index outside the vertex array")
    return V, T


def winding_number(V, T, points):
    """Generalized winding number of the triangle mesh (V, T) at each point
    (1 inside a closed counter-clockwise mesh, 0 outside)."""
    V, T = _mesh(V, T)
    pts = _f64(points, 3)
    return np.array([_L().or_winding_number(_ptr(V), _ptr(T), len(T), _ptr(pts[i])) for i in range(len(pts))])


def sample_grid(V, r):
    """(lo, h, dims) of the sampling grid: cells of side 2 r / sqrt(3) over
    the bounding box of the vertices."""
    V = _f64(V, 3)
    lo = np.zeros(3)
    h = np.zeros(1)
    dims = np.zeros(3, np.int64)
    _L().or_sample_grid(_ptr(V), len(V), float(r), _ptr(lo), _ptr(h), _ptr(dims))
    return lo, float(h[0]), dims


def sample_volume(V, T, candidates, r):
    """The volume sampler of Sec. 4 (see or_sample_volume): indices of the
    chosen candidates in ascending cell order, and every candidate's inside
    flag."""
    V, T = _mesh(V, T)
    cand = _f64(candidates, 3)
    sel = np.zeros(max(1, len(cand)), np.int64)
    inside = np.zeros(max(1, len(cand)), np.uint8)
    n = _L().or_sample_volume(_ptr(V), len(V), _ptr(T), len(T), _ptr(cand), len(cand), float(r), _ptr(sel), len(sel),
                              _ptr(inside))
    if n < 0:
        raise RuntimeError(f"or_sample_volume failed ({n})")
    return sel[:n].copy(), inside[:len(cand)].astype(bool)


def sample_surface(V, candidates, r):
    """The surface sampler (see or_sample_surface): indices of the chosen
    candidates in ascending cell order."""
    V = _f64(V, 3)
    cand = _f64(candidates, 3)
    sel = np.zeros(max(1, len(cand)), np.int64)
    n = _L().or_sample_surface(_ptr(V), len(V), _ptr(cand), len(cand), float(r), _ptr(sel), len(sel))
    if n < 0:
        raise RuntimeError(f"or_sample_surface failed ({n})")
    return sel[:n].copy()
