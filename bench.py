"""Benchmark of one simulation frame of the two-level granular method.

A step is one frame of the whole hot path on the digging workload (50,527 LR
/ 2,021,080 HR particles, r_LR = 0.0089 m, ratio 40): the kinematic bucket's
pose update, four LR steps of Algorithm 1 (dt = 1/240 s each, 2
stabilization + 8 solver passes, with binning and candidate search), and one HR
upsampling frame of Sec. 4 (LR re-binning, the HR reorder every 8 frames,
the fused gather / blend / advection / SDF kernel).

  value  HR particles per second of whole frames, device-timed with CUDA
         events on the library's stream, inputs resident, L2 flushed between
         timed steps (a 512 MiB write, then a 512 MiB read, so no dirty line
         is written back inside the frame); summed over ranks.  The same
         frames after the write alone are reported beside it.
  e2e    the same frames through the C ABI with the full state (LR and HR
         position and velocity) copied from pinned host memory before and
         the HR result copied back after every step.
  roofline  the upsampling kernel: algorithmic bytes (64 B per HR particle
         read + written, 32 B per LR particle, 4 B per cell start) over its
         average CUDA-event duration, against the measured HBM copy peak.
  cpu_baseline  the FP64 oracle's plain definitions on this machine's host
         cores on a bounded sample (the frame's LR steps of the whole LR set
         + the HR frame of 200,000 random HR particles, scaled to the frame;
         the LR steps also on one thread).

--impl reference runs that oracle alone as the reference arm.
Under torchrun every rank steps its own replica of the scene (weak scaling,
no collective on the data path); rank 0 prints one JSON line.  With
--partition slab the ranks split one scene's HR set instead (strong scaling,
an all-gather of the HR slabs before each HR reorder).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "high-res particles/sec (gs_upsample) and HBM GB/s vs peak at 2M; batched vs plain"
UNIT = "HR particles/s"
DT = 1.0 / 60.0
N_SUB = 4            # LR substeps per frame: dt_LR = 1/240 s, about the paper's 0.005 s
DT_LR_MAX, CFL = 0.005, 0.4   # adaptive frames: the paper's default LR step and the CFL number
FLUSH_BYTES = 512 << 20
# DRAM bytes of one upsampling launch on this workload, and its DRAM, SM and
# issue utilisation, from an ncu capture of the kernel source with this hash
# (profiles/); reported only while the source is unchanged.
TRAFFIC_CAPTURE = {"source_sha1": "6be7d4f2f05b84c922ae0661ecf4df758ad19515", "bytes": 82662400,
                   "dram_throughput_pct": 6.8, "sm_throughput_pct": 59.1, "issue_active_pct": 62.2}


class L2Flush:
    """Evicts L2 (129 MB) between timed steps: a 512 MiB write, then, when
    clean, a 512 MiB read of a second buffer, which writes the first one's
    dirty lines back before the timed work instead of inside it.  Runs on
    torch's current stream (the library's)."""

    def __init__(self, torch, dev):
        self.w = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.r = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.sink = None

    def __call__(self, k, clean=True):
        self.w.fill_(float(k))
        if clean:
            self.sink = self.r.sum()


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gs", "reference"], default="gs")
    ap.add_argument("--workload", choices=["digging", "funnel", "cube"], default="digging")
    ap.add_argument("--bed-size", type=float, default=1.0,
                    help="digging bed edge in metres (same particle density; 2.0 gives 4x the particles)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU baseline sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-diff", action="store_true")
    ap.add_argument("--no-materials", action="store_true", help="skip the grain-material frame timing")
    ap.add_argument("--no-adaptive", action="store_true", help="skip the CFL-limited substep frame timing")
    ap.add_argument("--no-solid", action="store_true", help="skip the particle-sampled bucket frame timing")
    ap.add_argument("--no-castle", action="store_true",
                    help="skip the mesh-sampled sand-castle scene (volume sampler and frame timing)")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="do not try pipelined frames (HR frame overlapping the next frame's LR steps)")
    ap.add_argument("--partition", choices=["replicas", "slab"], default="replicas",
                    help="under torchrun: every rank steps its own replica of the scene (weak scaling), or the "
                         "ranks split one scene's HR slots into slabs, each computing the LR state itself, with "
                         "one all-gather of the slabs before each HR reorder (strong scaling)")
    ap.add_argument("--diff-only", action="store_true",
                    help="time the differentiable rollout alone (--warmup and --steps count rollouts); for profilers")
    ap.add_argument("--batch-scenes", type=int, default=256)
    ap.add_argument("--gather-shape", default=None, metavar="WxB",
                    help="fix the gather's launch shape (warps per block x blocks per SM, 0: one item per warp) "
                         "instead of autotuning it; profiler runs use it, since a profiler skews the tuner's timing")
    return ap.parse_args(argv)


def make_scene(name, bed_size=1.0):
    if name == "digging":
        return scenes.digging(size=bed_size)
    return {"funnel": scenes.funnel, "cube": scenes.cube}[name]()


def workload_config(sc):
    return {"workload": f"{sc['name']} scene, {len(sc['lr_pos'])} LR / {len(sc['hr_pos'])} HR particles, "
                        f"r_LR {sc['r_low']} m, ratio {sc['ratio']}",
            "n_low": len(sc["lr_pos"]), "n_high": len(sc["hr_pos"]), "r_low": sc["r_low"],
            "ratio": sc["ratio"], "dt": DT, "lr_solver_iters": sc["iters"], "n_stab": 2,
            "hr_reorder_every": 8, "lr_steps_per_frame": N_SUB, "dt_low": DT / N_SUB,
            "l2": "flushed between timed steps (512 MiB write, then a 512 MiB read that leaves no dirty line)"}


def bucket_at(sc, frame):
    if "bucket_index" not in sc:
        return None
    return sc["bucket_index"], scenes.bucket_sdf(frame * DT)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ------------------------------------------------------------- clocks ---
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [a.strip() for a in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------- CPU baseline ---
CPU_SAMPLE_HR = 200_000   # HR particles per sample, the same in both arms


def oracle_frame_rate(sc, budget_s, sample_hr=CPU_SAMPLE_HR):
    """HR particles/s of the FP64 oracle's plain definitions on the host
    cores: the frame's LR steps of the whole LR set plus the HR frame of a
    random HR subset, scaled to the full frame, repeated until the time
    budget is used.  The LR steps are timed on one thread and on every core
    (the value uses every core); the HR sample on every core."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    r = sc["r_low"]
    g = sc["gravity"]
    pp = dict(r=r, dt=DT / N_SUB, gx=g[0], gy=g[1], gz=g[2], mu_s=sc["mu_s"], mu_k=sc["mu_k"], n_stab=2,
              iters=sc["iters"], mass_k=1.0, ground_z=sc["box_lo"][2], rc=3 * r, friction_mode=0, eps_x=1e-7,
              eps_impact=1e-9)
    up = dict(r_low=r, r_high=sc["r_high"], dt=DT, gx=g[0], gy=g[1], gz=g[2], c1=512 / 729, c2=0.6, eps_w=1e-4,
              eps_x=2e-6)
    M = len(sc["hr_pos"])
    ns = min(sample_hr, M)
    rng = np.random.default_rng(0)
    sdf = scenes.sdf_table(sc["sdfs"])
    lr_x, lr_v, im = sc["lr_pos"][:, :3], sc["lr_vel"][:, :3], sc["lr_pos"][:, 3]
    hr_x, hr_v = sc["hr_pos"][:, :3], sc["hr_vel"][:, :3]

    def lr_steps(threads):
        oracle.set_threads(threads)
        t0 = time.perf_counter()
        x1, v1 = lr_x, lr_v
        for _ in range(N_SUB):
            x1, v1 = oracle.pbd_step_plain(x1, v1, im, sdf, pp)
        return x1, v1, time.perf_counter() - t0

    _, _, t_lr1 = lr_steps(1)                     # once on one thread
    t_lr = t_up = 0.0
    reps = 0
    t_start = time.perf_counter()
    while reps == 0 or time.perf_counter() - t_start < budget_s:
        sub = np.sort(rng.choice(M, size=ns, replace=False))
        x1, v1, t = lr_steps(cores)
        t0 = time.perf_counter()
        oracle.upsample_plain(x1, v1, hr_x[sub], hr_v[sub], sdf, up)
        t_up += time.perf_counter() - t0
        t_lr += t
        reps += 1
    oracle.set_threads(1)
    frame_s = (t_lr + t_up * M / ns) / reps
    return {"value": M / frame_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "lr_steps_ms_1_thread": 1e3 * t_lr1, f"lr_steps_ms_{cores}_threads": 1e3 * t_lr / reps,
            "hr_us_per_particle": 1e6 * t_up / reps / ns,
            "sample": f"{reps} x ({N_SUB} FP64 LR steps of all {len(lr_x)} LR particles + the HR frame of {ns} "
                      f"random HR particles, on {cores} threads; the oracle's plain definitions), scaled to the "
                      f"{M}-particle frame; the LR steps also timed once on 1 thread"}


# ----------------------------------------------------------- batched ---
def run_batched(args, dev, stream, gs, torch):
    """Many independent scenes in one context (one graph-replayed frame for
    all of them) against the same scenes in separate contexts."""
    sl = scenes.batch(n_scenes=args.batch_scenes)
    iters = 8
    M = sum(len(s["hr_pos"]) for s in sl)
    batch = gs.Context(sl, stream=stream.cuda_stream)
    for _ in range(2):
        batch.frame(DT, N_SUB, iters)
    tw, tb, tus = batch.autotune(DT, reps=3)
    batch.set_graphs(True)
    tried = {}
    for shape in (None, (8, 2), (16, 2), (8, 4)):
        if shape is None:
            batch.set_pipeline(False, 8, 1)
        else:
            batch.set_pipeline(True, *shape)
        tried["sequential" if shape is None else f"pipelined {shape[0]}x{shape[1]}"] = \
            frame_ms(lambda: batch.frame(DT, N_SUB, iters), stream, dev, torch)
    pick = min(tried, key=tried.get)
    if pick == "sequential":
        batch.set_pipeline(False, 8, 1)
    else:
        w, b = (int(t) for t in pick.split()[1].split("x"))
        batch.set_pipeline(True, w, b)
    for _ in range(3):
        batch.frame(DT, N_SUB, iters)
    torch.cuda.synchronize(dev)
    k = max(5, args.steps // 5)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    flush = L2Flush(torch, dev)
    l0 = batch.launches()
    for i in range(k):
        flush(i)
        ev[i][0].record(stream)
        batch.frame(DT, N_SUB, iters)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    batch.sync()
    nl = (batch.launches() - l0) / k
    ms = sum(a.elapsed_time(b2) for a, b2 in ev) / k
    batch.close()
    # the same scenes, one context each, launched one after the other
    ctxs = [gs.Context(s, stream=stream.cuda_stream) for s in sl]
    for c in ctxs:
        c.frame(DT, N_SUB, iters)
    torch.cuda.synchronize(dev)
    k2 = 3
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k2)]
    for i in range(k2):
        flush(i)
        ev2[i][0].record(stream)
        for c in ctxs:
            c.frame(DT, N_SUB, iters)
        ev2[i][1].record(stream)
    torch.cuda.synchronize(dev)
    ms2 = sum(a.elapsed_time(b2) for a, b2 in ev2) / k2
    for c in ctxs:
        c.sync()
        c.close()
    return {"scenes": len(sl), "n_low": int(sum(len(s["lr_pos"]) for s in sl)), "n_high": int(M),
            "frame": f"{N_SUB} LR steps of {DT / N_SUB:.5f} s ({iters} solver passes) + 1 upsampling frame",
            "batched_ms_per_frame": ms, "batched_hr_per_s": M / (ms / 1e3), "batched_kernels_per_frame": nl,
            "separate_ms_per_frame": ms2, "separate_hr_per_s": M / (ms2 / 1e3),
            "speedup_vs_separate": ms2 / ms, "frame_ms_tried": tried, "frame_mode": pick,
            "upsample_tuning": {"warps_per_block": tw, "blocks_per_sm": tb,
                                                                   "upsample_us": tus}}


def run_diff(args, dev, stream, gs, torch, reps=None, warm=2, with_plain=True):
    """The differentiable form on the falling-column workload (4k LR / 64k
    HR, 30 steps of one LR step and one HR frame, recomputation checkpoints
    every 5 steps): forward + loss + backward to the initial LR velocities,
    against the plain in-place forward of the same rollout.  reps timed
    rollouts of each (default max(3, steps / 10)) after warm untimed ones."""
    from paper_2308_01629_gb300.diff import rollout
    sc = scenes.diff_column()
    dt, F, iters, every = sc["dt"], sc["steps"], sc["iters"], sc["checkpoint_every"]
    M = len(sc["hr_pos"])
    k = max(3, args.steps // 10) if reps is None else reps
    with torch.cuda.stream(stream):
        plain = gs.Context(sc, stream=stream.cuda_stream)
        ctx = gs.Context(sc, stream=stream.cuda_stream)
        plain.set_graphs(True)   # frames, and the functional LR steps, replayed as graphs
        ctx.set_graphs(True)
        state = [torch.from_numpy(np.ascontiguousarray(sc[n])).to(dev) for n in ("lr_pos", "lr_vel", "hr_pos",
                                                                                  "hr_vel")]
        target = torch.from_numpy(sc["target"]).to(dev)

        def plain_rollout():
            for _ in range(F):
                plain.frame(dt, 1, iters)

        def diff_rollout(native=True):
            X, V, x, v = state
            V = V.clone().requires_grad_(True)
            out = rollout(ctx, X, V, x, v, dt, frames=F, n_sub=1, iters=iters, checkpoint_every=every, native=native)
            loss = ((out[2][:, :3] - target) ** 2).sum()
            loss.backward()
            return V.grad

        def timed(fn):
            for _ in range(warm):
                fn()
            torch.cuda.synchronize(dev)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
            for a, b in ev:
                a.record(stream)
                fn()
                b.record(stream)
            torch.cuda.synchronize(dev)
            return sum(a.elapsed_time(b) for a, b in ev) / k

        ms_plain = timed(plain_rollout) if with_plain else None
        l0 = ctx.launches()
        ms_diff = timed(diff_rollout)
        nl = (ctx.launches() - l0) / (k + warm)
        ms_torch = timed(lambda: diff_rollout(native=False)) if with_plain else None
        ctx.set_deterministic_backward(True)
        ms_det = timed(diff_rollout) if with_plain else None
        ctx.set_deterministic_backward(False)
        plain.close()
        ctx.close()
    return {"workload": f"falling column {len(sc['lr_pos'])} LR / {M} HR, {F} steps of {dt:.6f} s, "
                        f"checkpoint every {every}", "loss": "sum |x_HR - target|^2 after the rollout",
            "plain_forward_ms_per_rollout": ms_plain, "forward_backward_ms_per_rollout": ms_diff,
            "forward_backward_hr_steps_per_s": M * F / (ms_diff / 1e3),
            "backward_overhead_vs_plain_forward": ms_diff / ms_plain if ms_plain else None,
            "library_kernels_per_rollout": nl,
            "rollout": "run by the library (gs_rollout_forward / _backward, one CUDA graph each)",
            "torch_driven_forward_backward_ms_per_rollout": ms_torch,
            "deterministic_backward_ms_per_rollout": ms_det}


def run_diff_only(args):
    """--diff-only: the differentiable rollout alone (--warmup untimed and
    --steps timed rollouts, no plain forward), for profiler runs."""
    import torch

    import paper_2308_01629_gb300 as gs
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    return {"differentiable": run_diff(args, dev, stream, gs, torch, reps=max(1, args.steps), warm=args.warmup,
                                       with_plain=False)}


def frame_ms(fn, stream, dev, torch, warm=2, reps=3):
    """Mean time of fn() on the stream over reps calls after warm calls."""
    for _ in range(warm):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / reps


def max_over_ranks(x, world, dev):
    """The largest value of x over all ranks (one all_reduce, outside the
    timed work); x itself on a single rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units processed by all ranks per second of the slowest rank (weak
    scaling: every rank processes the same number of units)."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------- GPU arm ---
def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2308_01629_gb300 as gs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # a dedicated stream: the library enqueues on it, the events and the L2
    # flush are recorded on it (the legacy default stream has handle 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    sc = make_scene(args.workload, args.bed_size)
    N, M = len(sc["lr_pos"]), len(sc["hr_pos"])
    ctx = gs.Context(sc, stream=stream.cuda_stream)
    flush = L2Flush(torch, dev)
    frame = [0]

    def step(c, adaptive=False):
        # one frame: the bucket pose, N_SUB LR steps (or CFL-limited steps of
        # at most DT_LR_MAX) and the HR frame; with graphs on and timers off
        # it is one graph launch
        b = bucket_at(sc, frame[0])
        if b is not None:
            c.set_sdf(*b)
        if adaptive:
            c.frame_adaptive(DT, sc["iters"], dt_max=DT_LR_MAX, cfl=CFL)
        else:
            c.frame(DT, N_SUB, sc["iters"])
        frame[0] += 1

    def barrier():
        if world > 1:
            dist.barrier()

    # clocks are sampled from before the warm-up to the end of the timed
    # steps (the timed region alone can be shorter than one sample period)
    # the library's launch-shape autotuner on the first frames' state
    step(ctx)
    if args.gather_shape:
        tune_w, tune_b = (int(t) for t in args.gather_shape.split("x"))
        ctx.set_tuning(tune_w, tune_b)
        tune_us = None
    else:
        tune_w, tune_b, tune_us = ctx.autotune(DT, reps=3)
    ctx.set_graphs(True)
    pipe = {"enabled": False}
    if not args.no_pipeline:
        # sequential frames against pipelined ones (the HR frame of frame f
        # overlapping the LR steps of frame f + 1, for a few gather shapes):
        # whichever whole frame is faster is timed below
        tried = {}
        for shape in (None, (8, 1), (8, 3), (4, 2), (4, 0)):
            if shape is None:
                ctx.set_pipeline(False, 8, 1)
            else:
                ctx.set_pipeline(True, *shape)
            tried["sequential" if shape is None else f"pipelined {shape[0]}x{shape[1]}"] = \
                frame_ms(lambda: step(ctx), stream, dev, torch)
        name = min(tried, key=tried.get)
        if name == "sequential":
            ctx.set_pipeline(False, 8, 1)
        else:
            w, b = (int(t) for t in name.split()[1].split("x"))
            ctx.set_pipeline(True, w, b)
            pipe = {"enabled": True, "gather_warps_per_block": w, "gather_blocks_per_sm": b,
                    "note": "each timed frame runs its LR steps on the main stream while the HR frame of the "
                            "previous frame runs on a second stream; K timed frames hold K frames of each"}
        pipe["frame_ms_tried"] = tried
    # the gather's own time inside the timed frames: events of the library
    # around its launches, recorded by every replay of the frame graph (not
    # with pipelined frames, whose gather runs on the library's second stream)
    gather_live = not pipe["enabled"]
    if gather_live:
        ctx.set_gather_timer(True)
    clk = Clocks(local)
    time.sleep(0.3)
    for _ in range(args.warmup):
        step(ctx)
    torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    gather_ms_live = []
    launches0 = ctx.launches()
    barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush(k)
        starts[k].record(stream)
        step(ctx)
        ends[k].record(stream)
        if gather_live:   # waits for this frame; the next frame's flush and events follow
            gather_ms_live.append(ctx.gather_timer_ms())
    torch.cuda.synchronize(dev)
    barrier()
    wall = time.perf_counter() - wall0
    launches = ctx.launches() - launches0
    ctx.sync()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(step_ms))
    # the same frames after a write-only flush: its dirty lines are written
    # back while the frame runs (reported beside the clean-flush number)
    for k in range(args.steps):
        flush(k, clean=False)
        starts[k].record(stream)
        step(ctx)
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    dirty_ms = float(sum(s.elapsed_time(e) for s, e in zip(starts, ends)))
    time.sleep(0.15)
    clocks = clk.stop()
    if clocks:
        clocks["window"] = "warm-up and both timed loops"

    # The same frames with the library's event timers around each phase
    # (timers bypass the graphs): the breakdown and the gather kernel's
    # launch duration for the roofline.
    ctx.set_timing(True)
    for t in range(gs.GS_TIMER_COUNT):
        ctx.timing_read(t)
    n_brk = max(4, args.steps // 2)
    for k in range(n_brk):
        flush(k)
        step(ctx)
    torch.cuda.synchronize(dev)
    ctx.sync()
    gather_ms, gather_n = ctx.timing_read(gs.GS_TIMER_GATHER)
    lr_ms, lr_n = ctx.timing_read(gs.GS_TIMER_STEP_LOW)
    bin_ms, bin_n = ctx.timing_read(gs.GS_TIMER_BIN_LOW)
    rs_ms, rs_n = ctx.timing_read(gs.GS_TIMER_RESORT)
    ctx.set_timing(False)
    total_ms = max_over_ranks(total_ms, world, dev)
    dirty_ms = max_over_ranks(dirty_ms, world, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(M * args.steps, world, total_ms / 1e3)

    # grain materials (per-particle friction, Sec. 3 cross coefficients):
    # the same frames with the bed above its median height a second
    # material, against frames without a table, timed alike (graph replay,
    # no L2 flush, alternating so both see the same stretch of the run)
    materials = None
    if not args.no_materials:
        table, ids = scenes.materials(sc, seed=0, layout="layers")
        tried = {"scene_coefficients": [], "two_materials": []}
        for _ in range(3):
            ctx.set_materials([])
            tried["scene_coefficients"].append(frame_ms(lambda: step(ctx), stream, dev, torch, warm=3, reps=8))
            ctx.set_materials(table, ids)
            tried["two_materials"].append(frame_ms(lambda: step(ctx), stream, dev, torch, warm=3, reps=8))
        ctx.set_materials([])
        base_ms, mat_ms = (float(np.median(tried[k])) for k in ("scene_coefficients", "two_materials"))
        materials = {"layout": "LR above the median height: material 1, below: material 0",
                     "table_mu_s_mu_k": table[:2].tolist(), "frame_ms_scene_coefficients": base_ms,
                     "frame_ms_two_materials": mat_ms, "overhead": mat_ms / base_ms - 1.0,
                     "timing": "median of 3 alternating runs of 8 graph-replayed frames, L2 not flushed"}

    # CFL-limited substeps (Sec. 5.2): the same frames with the LR steps
    # decided on the device each frame (default 0.005 s, shortened by the
    # CFL condition), against the fixed four steps, timed alike
    adaptive = None
    if not args.no_adaptive:
        tried = {"fixed_4_steps": [], "adaptive": []}
        steps = []
        for _ in range(3):
            tried["fixed_4_steps"].append(frame_ms(lambda: step(ctx), stream, dev, torch, warm=3, reps=8))
            tried["adaptive"].append(frame_ms(lambda: step(ctx, adaptive=True), stream, dev, torch, warm=3,
                                              reps=8))
            steps.append(len(ctx.substeps()))
        fixed_ms, adapt_ms = (float(np.median(tried[k])) for k in ("fixed_4_steps", "adaptive"))
        adaptive = {"dt_lr_max": DT_LR_MAX, "cfl": CFL, "frame_ms_fixed_4_steps": fixed_ms,
                    "frame_ms_adaptive": adapt_ms, "lr_steps_per_frame": steps,
                    "timing": "median of 3 alternating runs of 8 graph-replayed frames, L2 not flushed; the "
                              "adaptive frame's LR steps run in a device-side loop (conditional graph node)"}

    # particle-sampled rigid body (Sec. 3 / Sec. 4): the same bed with the
    # bucket sampled as LR particles of inverse mass 0 (moving with the
    # bucket's velocity) instead of the bucket SDF, in a second context,
    # timed alike against the SDF bucket's frames
    # and a rigid body by shape matching (Sec. 3): a boulder of 389 LR
    # particles (5000 kg/m^3) hurled into the same bed at 2 m/s
    solid = None
    if not args.no_solid and args.workload == "digging":
        ps = scenes.digging_particle_bucket(size=args.bed_size)
        pb = scenes.digging_with_boulder(size=args.bed_size)
        extra = {}
        for name, s in (("particle_bucket", ps), ("boulder", pb)):
            x = gs.Context(s, stream=stream.cuda_stream)
            x.set_tuning(tune_w, tune_b)
            x.set_graphs(True)
            extra[name] = (x, s)
        tried = {"sdf_bucket": [], "particle_bucket": [], "boulder": []}
        for _ in range(3):
            tried["sdf_bucket"].append(frame_ms(lambda: step(ctx), stream, dev, torch, warm=3, reps=8))
            for name, (x, s) in extra.items():
                tried[name].append(frame_ms(lambda: x.frame(DT, N_SUB, s["iters"]), stream, dev, torch, warm=3,
                                            reps=8))
        for x, _ in extra.values():
            x.sync()
            x.close()
        solid = {"bucket_particles": int(ps["n_solid"]), "n_low": len(ps["lr_pos"]),
                 "frame_ms_sdf_bucket": float(np.median(tried["sdf_bucket"])),
                 "frame_ms_particle_bucket": float(np.median(tried["particle_bucket"])),
                 "boulder_particles": int(pb["n_body"]),
                 "frame_ms_boulder_shape_matched": float(np.median(tried["boulder"])),
                 "timing": "median of 3 alternating runs of 8 graph-replayed frames, L2 not flushed"}

    # the sand-castle scene of Sec. 5 seeded by the library's volume sampler
    # (castle grains and HR particles, an icosphere boulder as one rigid body
    # flying at it): the sampler's time and the scene's frame time
    castle = None
    if not args.no_castle:
        t_sample = {}

        def timed_sample(V, T, C, r):
            t0 = time.perf_counter()
            sel = gs.sample_volume(V, T, C, r)
            t_sample.setdefault(f"r={r}", []).append((len(C), len(sel), 1e3 * (time.perf_counter() - t0)))
            return sel
        cs = scenes.castle_scene(timed_sample)
        x = gs.Context(cs, stream=stream.cuda_stream)
        x.set_graphs(True)
        frames_ms = [frame_ms(lambda: x.frame(DT, N_SUB, cs["iters"]), stream, dev, torch, warm=3, reps=8)
                     for _ in range(3)]
        x.sync()
        x.close()
        castle = {"n_low_grains": int(len(cs["lr_pos"]) - cs["n_body"]), "boulder_particles": int(cs["n_body"]),
                  "n_high": len(cs["hr_pos"]), "r_low": cs["r_low"], "r_high": cs["r_high"],
                  "frame_ms": float(np.median(frames_ms)),
                  "hr_per_s": len(cs["hr_pos"]) / (float(np.median(frames_ms)) / 1e3),
                  "sampling": [{"mesh_and_radius": k, "candidates": v[0][0], "samples": v[0][1],
                                "ms_including_transfers": round(v[0][2], 2)} for k, v in t_sample.items()],
                  "timing": "median of 3 runs of 8 graph-replayed frames, L2 not flushed; the sampler by host "
                            "wall clock around gs_sample_volume (host arrays in and out)"}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pin = {}
        for k in ("lr_pos", "lr_vel", "hr_pos", "hr_vel"):
            t = torch.empty(sc[k].shape, dtype=torch.float32, pin_memory=True)
            t.numpy()[:] = sc[k]
            pin[k] = t
        out_x = torch.empty((M, 4), dtype=torch.float32, pin_memory=True)
        out_v = torch.empty((M, 4), dtype=torch.float32, pin_memory=True)
        fields = ((gs.GS_FIELD_LR_POS, "lr_pos"), (gs.GS_FIELD_LR_VEL, "lr_vel"),
                  (gs.GS_FIELD_HR_POS, "hr_pos"), (gs.GS_FIELD_HR_VEL, "hr_vel"))

        def e2e_step():
            # synchronous calls: each write returns once its data is on the
            # device and checked, each read once the values are on the host
            for f, k in fields:
                ctx.write(f, pin[k])
            step(ctx)
            ctx.read(gs.GS_FIELD_HR_POS, out_x)
            ctx.read(gs.GS_FIELD_HR_VEL, out_v)

        def e2e_step_async():
            # the same transfers through the asynchronous calls: this frame's
            # inputs go up while the previous frame computes, its results come
            # down while the next one does
            for f, k in fields:
                ctx.write_async(f, pin[k])
            step(ctx)
            ctx.read_async(gs.GS_FIELD_HR_POS, out_x)
            ctx.read_async(gs.GS_FIELD_HR_VEL, out_v)

        def timed_e2e(fn):
            for _ in range(2):
                fn()
            ctx.sync()
            torch.cuda.synchronize(dev)
            barrier()
            t0 = time.perf_counter()
            for _ in range(ne):
                fn()
            ctx.sync()   # every transfer of every timed frame is complete
            torch.cuda.synchronize(dev)
            barrier()
            return max_over_ranks(time.perf_counter() - t0, world, dev)

        ne = max(3, args.steps // 2)
        te_sync = timed_e2e(e2e_step)
        te = timed_e2e(e2e_step_async)
        e2e = {"value": whole_job_rate(M * ne, world, te), "unit": UNIT, "h2d_bytes_per_step": int((2 * N + 2 * M) * 16),
               "d2h_bytes_per_step": int(2 * M * 16), "ms_per_step": 1e3 * te / ne,
               "api": "gs_write_async x4, gs_frame, gs_read_async x2 per frame; gs_sync at the end of the timed region",
               "synchronous_api_ms_per_step": 1e3 * te_sync / ne}

    ctx.close()
    batched = None if args.no_batched else run_batched(args, dev, stream, gs, torch)
    differentiable = None if args.no_diff else run_diff(args, dev, stream, gs, torch)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None

    pk = peaks()
    ncell = int(ctx.grid.n_cell) if hasattr(ctx, "grid") else 0
    alg_bytes = 64 * M + 32 * N + 4 * (ncell + 1)
    gather_avg_s = gather_ms / max(gather_n, 1) / 1e3   # breakdown frames, no graphs
    live_s = float(np.mean(gather_ms_live)) / 1e3 if gather_ms_live else None
    roof_s = live_s if live_s else gather_avg_s
    achieved = alg_bytes / roof_s / 1e9
    peak = pk["hbm_gbs"] if pk else 6800.0
    src = b"".join(open(os.path.join(ROOT, "paper_2308_01629_gb300", "csrc", f), "rb").read()
                   for f in ("upsample.cu", "sdf.cuh"))   # the kernel's sources
    sha = hashlib.sha1(src).hexdigest()
    captured = TRAFFIC_CAPTURE["source_sha1"] == sha
    traffic = TRAFFIC_CAPTURE["bytes"] if captured else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded scene generators)",
        "config": workload_config(sc),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_upsample (fused gather + blend + advection + SDF)",
                     "peak_source": "measured" if pk else "fallback",
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_us": roof_s * 1e6,
                     "duration_source": ("CUDA events of the library around the gather's launches inside each "
                                         "timed frame (graph event nodes)") if live_s else
                                        "library event timers in frames after the timed region (no graphs)",
                     "avg_launch_us_breakdown_frames": gather_avg_s * 1e6,
                     # from the same capture as traffic: the gather is bound by instruction
                     # issue on the CUDA cores, not by DRAM
                     "ncu": ({k: TRAFFIC_CAPTURE[k] for k in ("dram_throughput_pct", "sm_throughput_pct",
                                                             "issue_active_pct")} if captured else None)},
        "breakdown_ms_per_step": {"lr_steps": lr_ms / n_brk, "lr_binning_for_upsample": bin_ms / max(bin_n, 1),
                                  "hr_reorder_amortized": rs_ms / n_brk,
                                  "upsample_kernel": gather_ms / max(gather_n, 1),
                                  "source": f"{n_brk} frames after the timed region, library event timers "
                                            "around each phase (no graphs)"},
        "timed_region": "one CUDA-graph launch per frame (bucket pose copied before it)",
        "upsample_tuning": {"warps_per_block": tune_w, "blocks_per_sm": tune_b, "autotune_us": tune_us},
        "pipeline": pipe,
        "upsample_kernel_hr_per_s": M / roof_s,
        "wall_s_timed_region": wall,
        "l2_write_only_flush": {"ms_per_step": dirty_ms / args.steps,
                                "value": whole_job_rate(M * args.steps, world, dirty_ms / 1e3),
                                "note": "the same frames after a 512 MiB write alone, whose dirty lines are "
                                        "written back while the frame runs"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "e2e": e2e,
        "batched": batched,
        "differentiable": differentiable,
        "materials": materials,
        "adaptive_substeps": adaptive,
        "solid_particles": solid,
        "castle": castle,
    }
    if not args.no_cpu:
        line["cpu_baseline"] = oracle_frame_rate(sc, args.cpu_seconds)
    if world > 1:
        dist.destroy_process_group()
    return line


def run_slab(args):
    """One scene's HR set split across the ranks by slabs of its cell-ordered
    slots, the LR steps run by every rank; before each HR reorder the ranks
    all-gather their slabs (inside the timed frames).  value = the scene's
    HR particles per second of the slowest rank (strong scaling)."""
    import torch
    import torch.distributed as dist

    import paper_2308_01629_gb300 as gs
    from paper_2308_01629_gb300 import slabs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sc = make_scene(args.workload, args.bed_size)
    M = len(sc["hr_pos"])
    ctx = gs.Context(sc, stream=stream.cuda_stream)
    flush = L2Flush(torch, dev)
    if args.gather_shape:
        ctx.set_tuning(*(int(t) for t in args.gather_shape.split("x")))
    ctx.set_hr_slab(rank, world)
    ctx.set_graphs(True)
    frame = [0]
    exchanges = [0]

    def step():
        if world > 1 and frame[0] > 0 and frame[0] % 8 == 0:   # the reorder of this frame needs every slab
            slabs.assemble(ctx, rank, world)
            exchanges[0] += 1
        b = bucket_at(sc, frame[0])
        if b is not None:
            ctx.set_sdf(*b)
        ctx.frame(DT, N_SUB, sc["iters"])
        frame[0] += 1

    clk = Clocks(local)
    time.sleep(0.3)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = ctx.launches()
    ex0 = exchanges[0]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms = 0.0
    for k in range(args.steps):
        flush(k)
        start.record(stream)
        step()
        end.record(stream)
        end.synchronize()   # the exchange synchronizes on the host; time each frame on its own
        total_ms += start.elapsed_time(end)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    time.sleep(0.15)
    clocks = clk.stop()
    launches = ctx.launches() - launches0
    ctx.sync()
    b, e = ctx.hr_slab_range(rank, world)
    total_ms = max_over_ranks(total_ms, world, dev)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return None
    return {"metric": METRIC, "value": M * args.steps / (total_ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scene generators)",
            "config": dict(workload_config(sc), partition=f"HR slabs of one scene over {world} rank(s)",
                           slab_slots_rank0=[b, e], exchanges_timed=exchanges[0] - ex0),
            "timed_region": "per frame: the slab all-gather when a reorder is due, then one CUDA-graph launch",
            "gpu_launches": int(launches), "clocks": clocks,
            "e2e": None, "note": "auxiliary mode: no e2e, roofline or CPU baseline legs"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    sc = make_scene(args.workload, args.bed_size)
    per = min(8.0, max(1.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_frame_rate(sc, 0.0, sample_hr=20_000)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_frame_rate(sc, per))
    wall = time.perf_counter() - t0
    v = float(np.mean([a["value"] for a in vals]))
    M = len(sc["hr_pos"])
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * M / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded scene generators)",
            "config": workload_config(sc), "wall_s": wall,
            "cpu_baseline": dict({k: a for k, a in vals[0].items() if k not in ("value", "sample")},
                                 value=v, sample=f"{len(vals)} step(s), each: " + vals[0]["sample"]),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.impl == "reference":
        line = run_reference(args)
    elif args.diff_only:
        line = run_diff_only(args)
    elif args.partition == "slab":
        line = run_slab(args)
    else:
        line = run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
