"""Shared helpers of the parity tests: oracle parameter sets built from a
scene, and the comparison rule for float32 results against the FP64 oracle.

Tolerance (per particle, Euclidean norm), after one step from the same state:
  position  |x_gpu - x_ref| <= 1e-5 |x_ref| + 1e-6 L
  velocity  |v_gpu - v_ref| <= 1e-5 |v_ref| + 1e-6 L / dt
with L the largest edge of the scene box.  A particle whose result hangs on
a decision taken within the oracle's margin of its threshold is accepted on
either branch (flag 1) or only checked for finiteness (flag 2)."""
import numpy as np

C1 = 512.0 / 729.0
C2 = 0.6
RTOL = 1e-5
ATOL_L = 1e-6


def box_size(sc):
    return float(np.max(np.asarray(sc["box_hi"]) - np.asarray(sc["box_lo"])))


def f32(a):
    """The float32 value the C ABI receives for a scalar argument."""
    return float(np.float32(a))


def up_prm(sc, dt, eps_w=1e-4, eps_x=None):
    g = sc.get("gravity", (0.0, 0.0, -9.81))
    L = box_size(sc)
    return dict(r_low=f32(sc["r_low"]), r_high=f32(sc["r_high"]), dt=f32(dt), gx=f32(g[0]), gy=f32(g[1]),
                gz=f32(g[2]), c1=C1, c2=C2, eps_w=eps_w, eps_x=2e-6 * L if eps_x is None else eps_x)


def within(a, ref, rtol, atol):
    d = np.linalg.norm(np.asarray(a, float) - ref, axis=1)
    return d <= rtol * np.linalg.norm(ref, axis=1) + atol


def check_hr(sc, dt, gx, gv, ref, max_multi_frac=1e-3):
    """Compare GPU HR positions/velocities (n,3) with an oracle result."""
    L = box_size(sc)
    # float32 rounding of the advected position, amplified where the SDF
    # rule is ill-conditioned (near boundary edges): 2 ulp of |x|
    dpos = 2.0 * np.finfo(np.float32).eps * np.linalg.norm(ref["x"], axis=1)
    ax = ATOL_L * L + ref["diag"][:, 4] * dpos
    av = ATOL_L * L / dt + ref["diag"][:, 5] * dpos
    gx = np.asarray(gx, float)[:, :3]
    gv = np.asarray(gv, float)[:, :3]
    assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gv))
    prim = within(gx, ref["x"], RTOL, ax) & within(gv, ref["v"], RTOL, av)
    alt = within(gx, ref["alt_x"], RTOL, ax) & within(gv, ref["alt_v"], RTOL, av)
    fl = ref["flag"]
    ok = np.where(fl == 0, prim, np.where(fl == 1, prim | alt, True))
    bad = np.nonzero(~ok)[0]
    if len(bad):
        i = bad[0]
        raise AssertionError(
            f"{len(bad)} of {len(ok)} HR particles outside tolerance; first {i}: gpu x {gx[i]} v {gv[i]} "
            f"ref x {ref['x'][i]} v {ref['v'][i]} flag {fl[i]} diag {ref['diag'][i]}")
    assert (fl == 2).mean() <= max_multi_frac
    return dict(n=len(ok), flag1=int((fl == 1).sum()), flag2=int((fl == 2).sum()),
                max_dx=float(np.linalg.norm(gx - ref["x"], axis=1)[fl == 0].max(initial=0.0)),
                max_dv=float(np.linalg.norm(gv - ref["v"], axis=1)[fl == 0].max(initial=0.0)))


def pb_prm(sc, dt, n_stab, iters, eps_x=1e-7, eps_impact=1e-9, mass_k=1.0, friction_mode=0):
    """Oracle LR-step parameters matching a context built from the scene with
    default gs_params (height-scaled mass k = 1/m, ground at the box floor,
    neighbour radius 3 r_LR)."""
    g = sc.get("gravity", (0.0, 0.0, -9.81))
    r = f32(sc["r_low"])
    return dict(r=r, dt=f32(dt), gx=f32(g[0]), gy=f32(g[1]), gz=f32(g[2]), mu_s=f32(sc["mu_s"]),
                mu_k=f32(sc["mu_k"]), n_stab=n_stab, iters=iters, mass_k=mass_k, ground_z=f32(sc["box_lo"][2]),
                rc=f32(np.float32(3.0) * np.float32(r)), friction_mode=friction_mode, eps_x=eps_x,
                eps_impact=eps_impact)


def diff_prms(sc):
    """(LR-step, HR-frame) oracle parameters of a differentiable-rollout
    scene: one LR step and one HR frame of the same dt per step."""
    return (pb_prm(sc, sc["dt"], sc["n_stab"], sc["iters"], eps_impact=0.0),
            up_prm(sc, sc["dt"], eps_x=1e-6))
