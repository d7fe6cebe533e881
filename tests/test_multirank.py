"""Host logic of the multi-rank paths on CPU with two gloo ranks: the
benchmark's replicas (weak scaling, no collective on the data path; the
timing reduction takes the slowest rank, the whole-job rate counts the units
of all ranks; the reference arm runs on rank 0 only), and the exchange of one
scene's HR slabs (every rank updates its slab, one all-gather puts the whole
state back on every rank)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank                  # rank 1 is the slow one
        total_ms = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
        rate = bench.whole_job_rate(1000 * 4, world, total_ms / 1e3)
        ref = bench.run_reference(bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])) \
            if rank == 1 else "rank0-skipped"
        out.put((rank, total_ms, rate, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_and_count_all_units():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total_ms, rate, ref in res:
        assert total_ms == 15.0                       # the maximum over both ranks
        assert rate == pytest.approx(2 * 4000 / 0.015)  # both ranks' units over the slowest time
    assert res[1][3] is None                          # the reference arm does no work off rank 0


def _slab_rank_main(rank, world, port, out):
    """One scene's HR slots split by slabs: each rank's own slab holds the
    true values, the rest stale values of its own; the gather-back leaves
    the true values everywhere on every rank."""
    import torch.distributed as dist

    from paper_2308_01629_gb300 import slabs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 32 * 37                                    # an odd number of items: unequal slabs
        true_pos = torch.arange(4 * n, dtype=torch.float32).reshape(n, 4)
        true_vel = -0.5 * true_pos
        pos = torch.full((n, 4), 1000.0 + rank)
        vel = torch.full((n, 4), -1000.0 - rank)
        b, e = slabs.slab_ranges(n, world)[rank]
        pos[b:e] = true_pos[b:e]
        vel[b:e] = true_vel[b:e]
        slabs.all_gather_slabs(pos, vel, rank, world)
        out.put((rank, (b, e), bool(torch.equal(pos, true_pos)), bool(torch.equal(vel, true_vel))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_back_their_hr_slabs():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == (0, 32 * 18) and res[1][1] == (32 * 18, 32 * 37)
    assert all(r[2] and r[3] for r in res)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.whole_job_rate(100, 1, 0.5) == 200


def test_reference_arm_line_follows_the_contract(monkeypatch):
    """The reference arm (the FP64 oracle on the host cores, rank 0) prints
    one JSON line with the contract's keys, the workload's config, a
    cpu_baseline describing the run and an e2e with no device transfers."""
    import json

    import bench
    monkeypatch.delenv("RANK", raising=False)
    line = bench.run_reference(bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"]))
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    assert line["ms_per_step"] == pytest.approx(1e3 * line["config"]["n_high"] / line["value"])
    assert line["config"]["workload"].startswith("digging") and line["config"]["n_high"] == 2021080
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    json.loads(json.dumps(line))


def test_profile_commands_use_existing_bench_flags():
    """Every bench.py flag named in the commands recorded under profiles/
    exists, so each recorded command still runs."""
    import pathlib
    import re

    import bench
    root = pathlib.Path(bench.__file__).resolve().parent
    parser_flags = set()
    src = (root / "bench.py").read_text()
    parser_flags.update(re.findall(r'add_argument\("(--[a-z0-9-]+)"', src))
    assert "--gather-shape" in parser_flags and "--no-e2e" in parser_flags
    files = sorted((root / "profiles").glob("*.md"))
    assert files
    for f in files:
        text = f.read_text()
        cmd = text[text.index("python bench.py"):]
        cmd = cmd[:cmd.index("\n\n")]
        for flag in re.findall(r"(--[a-z0-9-]+)", cmd):
            assert flag in parser_flags, f"{f.name}: {flag}"
