"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2): the timed region is
the slowest rank's, and the aggregate rate counts every rank's replica."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [100.0, 250.0][rank]
    res = bench.aggregate_ranks(ms_local, steps=50, sites_per_rank=1000, world_size=world, device="cpu")
    # each rank's own estimate of the timed region differs; every rank must run the same count
    reps = bench.repeats_for([10.0, 2.0][rank], 1.0, world, device="cpu")
    q.put((rank, (res, reps)))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        (ms_total, ms_step, mlups), reps = out[rank]
        assert reps == 500                            # the larger of 100 and 500 repeats
        assert ms_total == 250.0                      # max over ranks
        assert ms_step == 5.0
        assert mlups == pytest.approx(2 * 1000 / 5e-3 / 1e6)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.aggregate_ranks(80.0, 40, 2000, 1) == (80.0, 2.0, 2000 / 2e-3 / 1e6)


def test_timed_region_repeats_cover_the_clock_window():
    """A short timed region (20 steps of ~0.28 ms) is repeated to cover the clock window; a
    long one still runs at least three times, and the count is capped."""
    import bench
    assert bench.repeats_for(5.6, 1.5, 1) == 268
    assert bench.repeats_for(560.0, 1.5, 1) == 3
    assert bench.repeats_for(1e-4, 1.5, 1) == 2000


def _reference_line(monkeypatch, capsys, steps, warmup, rank="0"):
    import argparse
    import json
    import bench
    monkeypatch.setenv("RANK", rank)
    monkeypatch.setattr(bench, "REF_BUDGET_S", 2.0)
    bench.run_reference(argparse.Namespace(steps=steps, warmup=warmup, gpus=1))
    out = capsys.readouterr().out.strip()
    return json.loads(out) if out else None


def test_reference_arm_line(monkeypatch, capsys):
    """The oracle arm prints one line with the contract's keys; its window shrinks to keep a
    long run within the oracle-time budget."""
    line = _reference_line(monkeypatch, capsys, steps=3, warmup=1)
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["steps"] == 3 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    long_run = _reference_line(monkeypatch, capsys, steps=100, warmup=3)
    assert long_run["config"]["sample"].startswith("16x2048")


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    assert _reference_line(monkeypatch, capsys, steps=3, warmup=1, rank="1") is None


def test_traffic_records_follow_code_not_comments():
    """A traffic record stays valid through comment and layout edits of a kernel's sources and
    lapses when its code changes (bench.py then reports no traffic figure)."""
    import bench
    a = "int f(int x) {  // doubles x\n    return 2 * x; /* fast\n path */\n}\n"
    b = "// f\nint f(int x) {\n  return 2 * x;\n}"
    c = "int f(int x) { return 3 * x; }"
    assert bench.code_of(a) == bench.code_of(b) != bench.code_of(c)


def test_fp64_roof():
    """The second roof: FP64 instructions per site x sites per second against the probe's rate;
    no figure for a kernel without a stated count or without a measured rate."""
    import bench
    r = bench.fp64_roof("k_step_ff", 2_000_000, 0.5, 4e11)
    assert r["instr_per_site"] == 42 and r["bound"] == "fp64_pipe"
    assert r["achieved"] == pytest.approx(42 * 2e6 / 0.5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 400.0)
    assert bench.fp64_roof("k_adjoint_ff", 1, 1.0, 1e9)["instr_per_site"] == 78
    assert bench.fp64_roof("k_step_f32", 1, 1.0, 1e9) is None
    assert bench.fp64_roof("k_step_ff", 1, 1.0, None) is None
