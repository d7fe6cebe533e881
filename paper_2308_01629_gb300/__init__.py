"""Python binding of libgs (include/gs.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and does
nothing but convert arguments; all of the method runs in the CUDA kernels of
``libgs.so``.  The library must have been built (``build.build()`` or
``__graft_entry__.build()``); if it is missing this module raises instead of
falling back to anything else.

``Context`` is a small convenience owner of one ``gs_ctx`` that builds the C
scene structure from the dictionaries of the ``scenes`` package and moves
numpy arrays or torch tensors through ``gs_write`` / ``gs_read``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GS_OK, GS_ERR_ARG, GS_ERR_OOM, GS_ERR_CUDA = 0, -1, -2, -3
GS_ERR_DOMAIN, GS_ERR_TIMEOUT, GS_ERR_STATE, GS_ERR_CAPACITY = -4, -5, -6, -7
STATUS_NAMES = {0: "GS_OK", -1: "GS_ERR_ARG", -2: "GS_ERR_OOM", -3: "GS_ERR_CUDA", -4: "GS_ERR_DOMAIN",
                -5: "GS_ERR_TIMEOUT", -6: "GS_ERR_STATE", -7: "GS_ERR_CAPACITY"}
GS_SDF_BOX_INTERIOR, GS_SDF_CONE_SHELL, GS_SDF_SOLID_BOX = 1, 2, 3
GS_MAX_SDF = 16
(GS_FIELD_LR_POS, GS_FIELD_LR_VEL, GS_FIELD_HR_POS, GS_FIELD_HR_VEL, GS_FIELD_HR_POS_INTERNAL,
 GS_FIELD_HR_VEL_INTERNAL, GS_FIELD_LR_CELL_START, GS_FIELD_LR_SORTED_INDEX, GS_FIELD_HR_SORTED_KEY,
 GS_FIELD_LR_MATERIAL) = range(10)
GS_MAX_MATERIALS = 16
GS_FIELD_LR_BODY = 10
GS_MAX_BODIES = 256
GS_MAX_SUBSTEPS = 256
GS_TIMER_BIN_LOW, GS_TIMER_RESORT, GS_TIMER_GATHER, GS_TIMER_STEP_LOW, GS_TIMER_COUNT = range(5)


class gs_sdf(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("p", ctypes.c_float * 12), ("vel", ctypes.c_float * 3),
                ("mu_s", ctypes.c_float), ("mu_k", ctypes.c_float)]


class gs_params(ctypes.Structure):
    _fields_ = [("gravity", ctypes.c_float * 3), ("mu_s", ctypes.c_float), ("mu_k", ctypes.c_float),
                ("c1", ctypes.c_float), ("c2", ctypes.c_float), ("n_stab", ctypes.c_int32),
                ("mass_scale_k", ctypes.c_float), ("ground_z", ctypes.c_float),
                ("neighbor_radius", ctypes.c_float), ("friction_mode", ctypes.c_int32),
                ("resort_every", ctypes.c_int32), ("max_neighbors", ctypes.c_int32)]


class gs_scene(ctypes.Structure):
    _fields_ = [("box_lo", ctypes.c_float * 3), ("box_hi", ctypes.c_float * 3), ("n_low", ctypes.c_int32),
                ("n_sdf", ctypes.c_int32), ("sdf", ctypes.POINTER(gs_sdf)), ("params", gs_params),
                ("n_high", ctypes.c_int64)]


class gs_grid_info(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("h", ctypes.c_float), ("inv_h", ctypes.c_float),
                ("dims", ctypes.c_int32 * 3), ("n_cell", ctypes.c_int64)]


class gs_scene_layout(ctypes.Structure):
    _fields_ = [("lr_offset", ctypes.c_int64), ("n_low", ctypes.c_int64), ("hr_offset", ctypes.c_int64),
                ("n_high", ctypes.c_int64), ("hr_slot_offset", ctypes.c_int64), ("hr_slot_end", ctypes.c_int64),
                ("cell_offset", ctypes.c_int64), ("grid", gs_grid_info), ("r_low", ctypes.c_float),
                ("r_high", ctypes.c_float)]


_P = ctypes.c_void_p
_SIGS = {
    "gs_default_params": (None, [ctypes.POINTER(gs_params)]),
    "gs_create": (ctypes.c_int, [ctypes.POINTER(gs_scene), ctypes.c_float, ctypes.c_float, ctypes.c_int, _P,
                                 ctypes.POINTER(_P)]),
    "gs_destroy": (None, [_P]),
    "gs_last_error": (ctypes.c_char_p, [_P]),
    "gs_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(gs_grid_info)]),
    "gs_write": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t, ctypes.c_int]),
    "gs_read": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t, ctypes.c_int]),
    "gs_set_sdf": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(gs_sdf)]),
    "gs_bin_low": (ctypes.c_int, [_P]),
    "gs_resort_high": (ctypes.c_int, [_P]),
    "gs_step_low": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_int]),
    "gs_upsample": (ctypes.c_int, [_P, ctypes.c_float]),
    "gs_sync": (ctypes.c_int, [_P]),
    "gs_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "gs_timing_read": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64)]),
    "gs_launch_count": (ctypes.c_int64, [_P]),
    "gs_bin_points_static": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(gs_grid_info), _P, _P, _P]),
    "gs_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(gs_scene), ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int), _P,
                                       ctypes.POINTER(_P)]),
    "gs_scene_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(gs_scene_layout)]),
    "gs_frame": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_int, ctypes.c_int]),
    "gs_set_graphs": (ctypes.c_int, [_P, ctypes.c_int]),
    "gs_set_materials": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
    "gs_frame_adaptive": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int,
                                         ctypes.c_int]),
    "gs_substeps": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gs_set_lr_solver": (ctypes.c_int, [_P, ctypes.c_int]),
    "gs_write_async": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t, ctypes.c_int]),
    "gs_read_async": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t, ctypes.c_int]),
    "gs_set_pipeline": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "gs_set_tuning": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "gs_autotune": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "gs_upsample_forward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_float]),
    "gs_upsample_backward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_float]),
    "gs_step_low_forward": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_int]),
    "gs_step_low_backward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_int]),
    "gs_step_low_trace": (ctypes.c_int, [_P, _P, _P, ctypes.c_float, ctypes.c_int, _P, _P, ctypes.c_int]),
    "gs_set_decision_record": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int]),
    "gs_set_alloc_failure": (None, [ctypes.c_longlong]),
    "gs_hr_slab_range": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "gs_set_hr_slab": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "gs_set_step_tapes": (ctypes.c_int, [_P, ctypes.c_int]),
    "gs_set_gather_timer": (ctypes.c_int, [_P, ctypes.c_int]),
    "gs_set_deterministic_backward": (ctypes.c_int, [_P, ctypes.c_int]),
    "gs_gather_timer_ms": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "gs_step_low_forward_taped": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_int, ctypes.c_int64]),
    "gs_step_low_backward_taped": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P]),
    "gs_rollout_forward": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "gs_rollout_backward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gs_sample_surface": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_double, _P,
                                         ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "gs_sample_volume": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_double,
                                        _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _P]),
    "gs_hr_slab_assemble": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t, ctypes.c_int]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libgs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libgs.so is not built ({path}); run __graft_entry__.build() first")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class GsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


# --------------------------------------------------- thin C entry points ---
def gs_default_params():
    p = gs_params()
    lib().gs_default_params(ctypes.byref(p))
    return p


def gs_create(scene, r_low, r_high, ratio, stream=None):
    ctx = _P()
    rc = lib().gs_create(ctypes.byref(scene), r_low, r_high, ratio, stream, ctypes.byref(ctx))
    if rc != GS_OK:
        raise GsError(rc, "gs_create failed")
    return ctx


def gs_batch_create(scenes, r_low, r_high, ratio, stream=None):
    n = len(scenes)
    arr = (gs_scene * n)(*scenes)
    rl = (ctypes.c_float * n)(*[float(a) for a in r_low])
    rh = (ctypes.c_float * n)(*[float(a) for a in r_high])
    ra = (ctypes.c_int * n)(*[int(a) for a in ratio])
    ctx = _P()
    rc = lib().gs_batch_create(n, arr, rl, rh, ra, stream, ctypes.byref(ctx))
    if rc != GS_OK:
        raise GsError(rc, "gs_batch_create failed")
    return ctx


def gs_destroy(ctx):
    lib().gs_destroy(ctx)


def gs_scene_info(ctx, scene):
    out = gs_scene_layout()
    rc = lib().gs_scene_info(ctx, int(scene), ctypes.byref(out))
    if rc != GS_OK:
        raise GsError(rc, "gs_scene_info failed")
    return out


def gs_frame(ctx, dt, n_sub, iters):
    return lib().gs_frame(ctx, dt, n_sub, iters)


def gs_set_graphs(ctx, enable):
    return lib().gs_set_graphs(ctx, int(enable))


def gs_set_lr_solver(ctx, persistent):
    return lib().gs_set_lr_solver(ctx, int(persistent))


def gs_set_pipeline(ctx, enable, warps_per_block=8, blocks_per_sm=1):
    return lib().gs_set_pipeline(ctx, int(enable), int(warps_per_block), int(blocks_per_sm))


def gs_frame_adaptive(ctx, dt, dt_max, cfl, max_sub, iters):
    return lib().gs_frame_adaptive(ctx, float(dt), float(dt_max), float(cfl), int(max_sub), int(iters))


def gs_substeps(ctx):
    """(status, dts): the LR step lengths of the latest adaptive frame."""
    out = np.zeros(GS_MAX_SUBSTEPS, np.float32)
    n = ctypes.c_int()
    rc = lib().gs_substeps(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(out), ctypes.byref(n))
    return rc, out[:max(n.value, 0)].copy()


def gs_set_materials(ctx, mu):
    """mu: (n, 2) array of (mu_s, mu_k) per material; empty turns materials off."""
    mu = np.ascontiguousarray(np.asarray(mu, np.float32).reshape(-1, 2))
    return lib().gs_set_materials(ctx, len(mu), mu.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))


def gs_set_tuning(ctx, warps_per_block, blocks_per_sm):
    return lib().gs_set_tuning(ctx, int(warps_per_block), int(blocks_per_sm))


def gs_autotune(ctx, dt, reps=5):
    w, b, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(ctx, lib().gs_autotune(ctx, dt, int(reps), ctypes.byref(w), ctypes.byref(b), ctypes.byref(us)),
           "gs_autotune")
    return w.value, b.value, us.value


def gs_last_error(ctx):
    return lib().gs_last_error(ctx).decode()


def _check(ctx, rc, what):
    if rc != GS_OK:
        raise GsError(rc, f"{what}: {gs_last_error(ctx)}")
    return rc


def gs_info(ctx):
    nl, nh, g = ctypes.c_int64(), ctypes.c_int64(), gs_grid_info()
    _check(ctx, lib().gs_info(ctx, ctypes.byref(nl), ctypes.byref(nh), ctypes.byref(g)), "gs_info")
    return nl.value, nh.value, g


def gs_write(ctx, field, ptr, nbytes, src_is_device):
    return lib().gs_write(ctx, field, ptr, nbytes, int(src_is_device))


def gs_write_async(ctx, field, ptr, nbytes, src_is_device):
    return lib().gs_write_async(ctx, field, ptr, nbytes, int(src_is_device))


def gs_read_async(ctx, field, ptr, nbytes, dst_is_device):
    return lib().gs_read_async(ctx, field, ptr, nbytes, int(dst_is_device))


def gs_read(ctx, field, ptr, nbytes, dst_is_device):
    return lib().gs_read(ctx, field, ptr, nbytes, int(dst_is_device))


def gs_set_sdf(ctx, index, sdf):
    return lib().gs_set_sdf(ctx, index, ctypes.byref(sdf))


def gs_bin_low(ctx):
    return lib().gs_bin_low(ctx)


def gs_resort_high(ctx):
    return lib().gs_resort_high(ctx)


def gs_step_low(ctx, dt, iters):
    return lib().gs_step_low(ctx, dt, iters)


def gs_upsample(ctx, dt):
    return lib().gs_upsample(ctx, dt)


def gs_sync(ctx):
    return lib().gs_sync(ctx)


def gs_set_timing(ctx, enable):
    return lib().gs_set_timing(ctx, int(enable))


def gs_timing_read(ctx, timer):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(ctx, lib().gs_timing_read(ctx, timer, ctypes.byref(ms), ctypes.byref(n)), "gs_timing_read")
    return ms.value, n.value


def gs_launch_count(ctx):
    return lib().gs_launch_count(ctx)


GS_STATIC_BIN_MAX_POINTS = 262144


def gs_bin_points_static(pos4_ptr, n, grid, sorted_index_ptr, cell_start_ptr, stream=None):
    """Binning with the library's static scratch (no allocation); device pointers."""
    return lib().gs_bin_points_static(pos4_ptr, n, ctypes.byref(grid), sorted_index_ptr, cell_start_ptr, stream)


def gs_upsample_forward(ctx, lr_pos, lr_vel, hr_pos_in, hr_vel_in, hr_pos_out, hr_vel_out, dt):
    return lib().gs_upsample_forward(ctx, lr_pos, lr_vel, hr_pos_in, hr_vel_in, hr_pos_out, hr_vel_out, dt)


def gs_upsample_backward(ctx, lr_pos, lr_vel, hr_pos_in, hr_vel_in, g_hr_pos_out, g_hr_vel_out, g_lr_pos, g_lr_vel,
                         g_hr_pos_in, g_hr_vel_in, dt):
    return lib().gs_upsample_backward(ctx, lr_pos, lr_vel, hr_pos_in, hr_vel_in, g_hr_pos_out, g_hr_vel_out,
                                      g_lr_pos, g_lr_vel, g_hr_pos_in, g_hr_vel_in, dt)


def gs_step_low_forward(ctx, x_in, v_in, x_out, v_out, dt, iters):
    return lib().gs_step_low_forward(ctx, x_in, v_in, x_out, v_out, dt, iters)


def gs_step_low_backward(ctx, x_in, v_in, g_x_out, g_v_out, g_x_in, g_v_in, dt, iters):
    return lib().gs_step_low_backward(ctx, x_in, v_in, g_x_out, g_v_out, g_x_in, g_v_in, dt, iters)


def gs_set_alloc_failure(after):
    lib().gs_set_alloc_failure(int(after))


def gs_hr_slab_range(n_slots, part, n_parts):
    """(status, begin, end): slab `part` of `n_parts` of n_slots HR slots."""
    b, e = ctypes.c_int64(), ctypes.c_int64()
    rc = lib().gs_hr_slab_range(int(n_slots), int(part), int(n_parts), ctypes.byref(b), ctypes.byref(e))
    return rc, b.value, e.value


def gs_set_deterministic_backward(ctx, enable):
    return lib().gs_set_deterministic_backward(ctx, int(enable))


def gs_set_gather_timer(ctx, enable):
    return lib().gs_set_gather_timer(ctx, int(enable))


def gs_gather_timer_ms(ctx):
    """(status, ms of the latest frame's gather)."""
    ms = ctypes.c_float()
    rc = lib().gs_gather_timer_ms(ctx, ctypes.byref(ms))
    return rc, ms.value


def gs_set_step_tapes(ctx, n_slots):
    return lib().gs_set_step_tapes(ctx, int(n_slots))


def gs_step_low_forward_taped(ctx, x_in, v_in, x_out, v_out, dt, iters, tag):
    return lib().gs_step_low_forward_taped(ctx, x_in, v_in, x_out, v_out, float(dt), int(iters), int(tag))


def gs_step_low_backward_taped(ctx, tag, g_x_out, g_v_out, g_x_in, g_v_in):
    return lib().gs_step_low_backward_taped(ctx, int(tag), g_x_out, g_v_out, g_x_in, g_v_in)


def gs_rollout_forward(ctx, lr_x0, lr_v0, hr_x0, hr_v0, dt, frames, n_sub, iters, checkpoint_every, lr_x, lr_v,
                       hr_x, hr_v):
    return lib().gs_rollout_forward(ctx, lr_x0, lr_v0, hr_x0, hr_v0, float(dt), int(frames), int(n_sub), int(iters),
                                    int(checkpoint_every), lr_x, lr_v, hr_x, hr_v)


def gs_rollout_backward(ctx, g_lr_x, g_lr_v, g_hr_x, g_hr_v, g_lr_x0, g_lr_v0, g_hr_x0, g_hr_v0):
    return lib().gs_rollout_backward(ctx, g_lr_x, g_lr_v, g_hr_x, g_hr_v, g_lr_x0, g_lr_v0, g_hr_x0, g_hr_v0)


def gs_sample_volume(vertices, triangles, candidates, r, capacity=None):
    """(status, selected, inside): the volume sampler of Sec. 4 on a closed
    triangle mesh (see include/gs.h).  Arrays are marshalled as float64 /
    int32; selected holds candidate indices in ascending cell order."""
    V = np.ascontiguousarray(np.asarray(vertices, np.float64).reshape(-1, 3))
    T = np.ascontiguousarray(np.asarray(triangles, np.int32).reshape(-1, 3))
    C = np.ascontiguousarray(np.asarray(candidates, np.float64).reshape(-1, 3))
    cap = len(C) if capacity is None else int(capacity)
    sel = np.zeros(max(cap, 1), np.int64)
    inside = np.zeros(max(len(C), 1), np.uint8)
    n = ctypes.c_int64()
    rc = lib().gs_sample_volume(V.ctypes.data, len(V), T.ctypes.data, len(T), C.ctypes.data, len(C), float(r),
                                sel.ctypes.data, cap, ctypes.byref(n), inside.ctypes.data)
    return rc, sel[:min(n.value, cap)].copy(), inside[:len(C)].astype(bool)


def gs_sample_surface(vertices, candidates, r, capacity=None):
    """(status, selected): the surface sampler (see include/gs.h)."""
    V = np.ascontiguousarray(np.asarray(vertices, np.float64).reshape(-1, 3))
    C = np.ascontiguousarray(np.asarray(candidates, np.float64).reshape(-1, 3))
    cap = len(C) if capacity is None else int(capacity)
    sel = np.zeros(max(cap, 1), np.int64)
    n = ctypes.c_int64()
    rc = lib().gs_sample_surface(V.ctypes.data, len(V), C.ctypes.data, len(C), float(r), sel.ctypes.data, cap,
                                 ctypes.byref(n))
    return rc, sel[:min(n.value, cap)].copy()


def sample_surface(vertices, candidates, r):
    """Indices of the chosen surface candidates; raises on error."""
    rc, sel = gs_sample_surface(vertices, candidates, r)
    if rc != GS_OK:
        raise GsError(rc, "gs_sample_surface failed")
    return sel


def sample_volume(vertices, triangles, candidates, r):
    """Indices of the chosen candidates (ascending cell order); raises on
    error."""
    rc, sel, _ = gs_sample_volume(vertices, triangles, candidates, r)
    if rc != GS_OK:
        raise GsError(rc, "gs_sample_volume failed")
    return sel


def gs_set_hr_slab(ctx, part, n_parts):
    return lib().gs_set_hr_slab(ctx, int(part), int(n_parts))


def gs_hr_slab_assemble(ctx, pos, vel, nbytes, src_is_device):
    return lib().gs_hr_slab_assemble(ctx, pos, vel, nbytes, int(src_is_device))


def gs_set_decision_record(ctx, hr_record, lr_candidates, lr_pair_bits, lr_sdf_bits, max_passes):
    return lib().gs_set_decision_record(ctx, hr_record, lr_candidates, lr_pair_bits, lr_sdf_bits, max_passes)


def gs_step_low_trace(ctx, x_in, v_in, dt, iters, x_trace, xt_trace, n_records):
    return lib().gs_step_low_trace(ctx, x_in, v_in, dt, iters, x_trace, xt_trace, n_records)


# ------------------------------------------------------------ marshalling ---
def make_sdf(rec) -> gs_sdf:
    s = gs_sdf()
    s.kind = int(rec["kind"])
    for k, v in enumerate(rec["p"][:12]):
        s.p[k] = float(v)
    for k, v in enumerate(rec["vel"][:3]):
        s.vel[k] = float(v)
    s.mu_s = float(rec["mu_s"])
    s.mu_k = float(rec["mu_k"])
    return s


def make_scene(sc, **overrides):
    """C scene from a ``scenes`` dictionary; keyword overrides set gs_params
    fields (e.g. n_stab=1, resort_every=0)."""
    prm = gs_default_params()
    g = sc.get("gravity", (0.0, 0.0, -9.81))
    for k in range(3):
        prm.gravity[k] = float(g[k])
    prm.mu_s = float(sc.get("mu_s", prm.mu_s))
    prm.mu_k = float(sc.get("mu_k", prm.mu_k))
    for k, v in overrides.items():
        if k == "gravity":
            for a in range(3):
                prm.gravity[a] = float(v[a])
        else:
            setattr(prm, k, v)
    arr = (gs_sdf * max(1, len(sc["sdfs"])))(*[make_sdf(r) for r in sc["sdfs"]])
    scene = gs_scene()
    for k in range(3):
        scene.box_lo[k] = float(sc["box_lo"][k])
        scene.box_hi[k] = float(sc["box_hi"][k])
    scene.n_low = int(len(sc["lr_pos"]))
    scene.n_high = int(len(sc["hr_pos"])) if "hr_pos" in sc else 0
    scene.n_sdf = len(sc["sdfs"])
    scene.sdf = ctypes.cast(arr, ctypes.POINTER(gs_sdf))
    scene.params = prm
    scene._keep = arr
    return scene


def _ptr_of(a):
    """(pointer, nbytes, is_device) of a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data, a.nbytes, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a.numel() * a.element_size(), int(a.is_cuda)
    raise TypeError(f"unsupported buffer type {type(a)}")


class Context:
    """Owner of one gs_ctx built from a ``scenes`` dictionary, or from a list
    of them (one batched context; arrays are concatenated in scene order)."""

    def __init__(self, sc, stream=None, load_state=True, **overrides):
        if isinstance(stream, str) and stream == "torch":
            # torch's current stream; its legacy default stream has handle 0,
            # which the C side would take as "create a stream", so pass the
            # legacy-stream handle (1) instead
            import torch
            h = torch.cuda.current_stream().cuda_stream
            stream = h if h else 1
        batch = isinstance(sc, (list, tuple))
        self.scene_list = list(sc) if batch else [sc]
        self._c_scenes = [make_scene(s, **overrides) for s in self.scene_list]
        if batch:
            self.ctx = gs_batch_create(self._c_scenes, [s["r_low"] for s in self.scene_list],
                                       [s["r_high"] for s in self.scene_list], [s["ratio"] for s in self.scene_list],
                                       stream)
        else:
            s0 = self.scene_list[0]
            self.ctx = gs_create(self._c_scenes[0], float(s0["r_low"]), float(s0["r_high"]), int(s0["ratio"]),
                                 stream)
        self.n_low, self.n_high, self.grid = gs_info(self.ctx)
        self.layouts = [gs_scene_info(self.ctx, k) for k in range(len(self.scene_list))]
        last = self.layouts[-1]
        self.hr_slots = int(last.hr_slot_end)
        self.n_cell_total = int(last.cell_offset + last.grid.n_cell + 1)
        self.sdf_offsets = np.cumsum([0] + [len(s["sdfs"]) for s in self.scene_list])
        if load_state:
            for f, k in ((GS_FIELD_LR_POS, "lr_pos"), (GS_FIELD_LR_VEL, "lr_vel"), (GS_FIELD_HR_POS, "hr_pos"),
                         (GS_FIELD_HR_VEL, "hr_vel")):
                self.write(f, np.ascontiguousarray(np.concatenate([s[k] for s in self.scene_list])))
            if any("lr_body" in s for s in self.scene_list):
                # rigid bodies (after the positions: the rest shapes come from
                # them); every scene's ids follow the previous scenes'
                ids, base = [], 0
                for s in self.scene_list:
                    b = np.asarray(s.get("lr_body", np.zeros(len(s["lr_pos"]))), np.uint32)
                    ids.append(np.where(b > 0, b + base, 0).astype(np.uint32))
                    base += int(b.max(initial=0))
                self.write(GS_FIELD_LR_BODY, np.ascontiguousarray(np.concatenate(ids)))

    def close(self):
        if self.ctx:
            gs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def write(self, field, buf):
        p, n, dev = _ptr_of(buf)
        return _check(self.ctx, gs_write(self.ctx, field, p, n, dev), "gs_write")

    def read(self, field, out=None):
        if out is None:
            counts = {GS_FIELD_LR_POS: (self.n_low, 4), GS_FIELD_LR_VEL: (self.n_low, 4),
                      GS_FIELD_HR_POS: (self.n_high, 4), GS_FIELD_HR_VEL: (self.n_high, 4),
                      GS_FIELD_HR_POS_INTERNAL: (self.hr_slots, 4), GS_FIELD_HR_VEL_INTERNAL: (self.hr_slots, 4),
                      GS_FIELD_LR_CELL_START: (self.n_cell_total + 1,),
                      GS_FIELD_LR_SORTED_INDEX: (self.n_low,), GS_FIELD_HR_SORTED_KEY: (self.hr_slots,),
                      GS_FIELD_LR_MATERIAL: (self.n_low,), GS_FIELD_LR_BODY: (self.n_low,)}
            shape = counts[field]
            out = np.zeros(shape, np.float32 if len(shape) == 2 else np.uint32)
        p, n, dev = _ptr_of(out)
        _check(self.ctx, gs_read(self.ctx, field, p, n, dev), "gs_read")
        return out

    def write_async(self, field, buf):
        """Stage a field for the next state-reading call; buf must stay valid
        and unchanged until sync()."""
        p, n, dev = _ptr_of(buf)
        return _check(self.ctx, gs_write_async(self.ctx, field, p, n, dev), "gs_write_async")

    def read_async(self, field, out):
        """Copy the field's current value into out (filled after sync())."""
        p, n, dev = _ptr_of(out)
        _check(self.ctx, gs_read_async(self.ctx, field, p, n, dev), "gs_read_async")
        return out

    def scene_slice(self, scene, field):
        """Index range of one scene inside a concatenated LR or HR field."""
        L = self.layouts[scene]
        if field in (GS_FIELD_LR_POS, GS_FIELD_LR_VEL):
            return slice(L.lr_offset, L.lr_offset + L.n_low)
        return slice(L.hr_offset, L.hr_offset + L.n_high)

    def set_sdf(self, index, rec, scene=0):
        k = int(self.sdf_offsets[scene]) + int(index)
        return _check(self.ctx, gs_set_sdf(self.ctx, k, make_sdf(rec)), "gs_set_sdf")

    def bin_low(self):
        return _check(self.ctx, gs_bin_low(self.ctx), "gs_bin_low")

    def resort_high(self):
        return _check(self.ctx, gs_resort_high(self.ctx), "gs_resort_high")

    def step_low(self, dt, iters):
        return _check(self.ctx, gs_step_low(self.ctx, float(dt), int(iters)), "gs_step_low")

    def upsample(self, dt):
        return _check(self.ctx, gs_upsample(self.ctx, float(dt)), "gs_upsample")

    def frame(self, dt, n_sub, iters):
        return _check(self.ctx, gs_frame(self.ctx, float(dt), int(n_sub), int(iters)), "gs_frame")

    def set_graphs(self, on=True):
        return _check(self.ctx, gs_set_graphs(self.ctx, on), "gs_set_graphs")

    def frame_adaptive(self, dt, iters, dt_max=0.005, cfl=0.4, max_sub=64):
        """One frame of dt with CFL-limited LR substeps (at most dt_max each,
        a grain moves at most cfl diameters per step) and one HR frame."""
        return _check(self.ctx, gs_frame_adaptive(self.ctx, dt, dt_max, cfl, max_sub, iters), "gs_frame_adaptive")

    def substeps(self):
        """The LR step lengths of the latest adaptive frame (float32 array)."""
        rc, dts = gs_substeps(self.ctx)
        _check(self.ctx, rc, "gs_substeps")
        return dts

    def set_materials(self, mu, ids=None):
        """Grain materials (Sec. 3): mu is an (n, 2) table of (mu_s, mu_k);
        ids (uint32 per LR particle, optional) assigns them.  An empty table
        returns to the scenes' coefficients."""
        _check(self.ctx, gs_set_materials(self.ctx, mu), "gs_set_materials")
        if ids is not None:
            self.write(GS_FIELD_LR_MATERIAL, np.ascontiguousarray(np.asarray(ids, np.uint32)))

    def set_lr_solver(self, persistent=True):
        return _check(self.ctx, gs_set_lr_solver(self.ctx, persistent), "gs_set_lr_solver")

    def set_pipeline(self, enable=True, warps_per_block=8, blocks_per_sm=1):
        return _check(self.ctx, gs_set_pipeline(self.ctx, enable, warps_per_block, blocks_per_sm), "gs_set_pipeline")

    def set_deterministic_backward(self, enable=True):
        """LR gradients of the HR frame's reverse mode gathered in a fixed
        order (bitwise reproducible) or added by float atomics (the
        default)."""
        return _check(self.ctx, gs_set_deterministic_backward(self.ctx, enable), "gs_set_deterministic_backward")

    def set_gather_timer(self, enable=True):
        """Events around the gather of every HR frame (graph replays too)."""
        return _check(self.ctx, gs_set_gather_timer(self.ctx, enable), "gs_set_gather_timer")

    def gather_timer_ms(self):
        """The latest frame's gather time (waits for that frame)."""
        rc, ms = gs_gather_timer_ms(self.ctx)
        _check(self.ctx, rc, "gs_gather_timer_ms")
        return ms

    def set_step_tapes(self, n_slots):
        """Keep the recorded passes of the latest n_slots taped LR steps for
        their backward (0: none)."""
        _check(self.ctx, gs_set_step_tapes(self.ctx, n_slots), "gs_set_step_tapes")
        self.step_tapes = int(n_slots)

    def set_hr_slab(self, part, n_parts):
        """Restrict this context's HR frames to slab `part` of `n_parts` of
        its cell-ordered HR slots (n_parts = 1: the whole set)."""
        return _check(self.ctx, gs_set_hr_slab(self.ctx, part, n_parts), "gs_set_hr_slab")

    def hr_slab_range(self, part, n_parts):
        """[begin, end) of slab `part` of `n_parts` of this context's HR slots."""
        rc, b, e = gs_hr_slab_range(self.hr_slots, part, n_parts)
        _check(self.ctx, rc, "gs_hr_slab_range")
        return b, e

    def hr_slab_assemble(self, pos, vel):
        """Write the whole HR state in internal slot order (float32 [slots, 4]
        each, host arrays or device tensors) and end the partial state."""
        pp, n, dev = _ptr_of(pos)
        pv, nv, devv = _ptr_of(vel)
        if nv != n or devv != dev:
            raise ValueError("pos and vel must have the same size and live on the same side")
        return _check(self.ctx, gs_hr_slab_assemble(self.ctx, pp, pv, n, dev), "gs_hr_slab_assemble")

    def set_tuning(self, warps_per_block, blocks_per_sm):
        return _check(self.ctx, gs_set_tuning(self.ctx, warps_per_block, blocks_per_sm), "gs_set_tuning")

    def autotune(self, dt, reps=5):
        return gs_autotune(self.ctx, float(dt), reps)

    def sync(self):
        return _check(self.ctx, gs_sync(self.ctx), "gs_sync")

    def set_timing(self, on=True):
        return _check(self.ctx, gs_set_timing(self.ctx, on), "gs_set_timing")

    def timing_read(self, timer):
        return gs_timing_read(self.ctx, timer)

    def launches(self):
        return gs_launch_count(self.ctx)
