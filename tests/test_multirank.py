"""The multi-process path of bench.py on CPU: two `gloo` ranks.

The path shards instances across ranks with no data-path exchange; the only
collectives are the timing barrier and the max over ranks.  These tests check
that the ranks' batches are disjoint and cover the job, that every rank sees
the slowest rank's time, and the whole-job rate."""
import json
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, local, ws = bench.dist_env()
        assert (r, local, ws) == (rank, rank, world)
        specs = bench.workload_specs("toeplitz10", r)
        seeds = [sp[1] for sp in specs]
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        # a rank's slow step: rank r took (r + 1) * 10 ms
        t = bench.max_over_ranks(dist, torch, float(10 * (rank + 1)), "cpu")
        dist.barrier()
        if rank == 0:
            out.put((gathered, t))
        else:
            out.put((None, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_instances_and_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gathered = next(g for g, _ in results if g is not None)
    times = [t for _, t in results]
    assert times == [20.0, 20.0]  # every rank sees the slowest rank
    flat = [s for shard in gathered for s in shard]
    assert len(flat) == len(set(flat)) == world * bench.BATCH  # disjoint, complete
    assert sorted(flat) == list(range(world * bench.BATCH))
    # whole-job rate: both ranks' instances over the slowest rank's time
    assert bench.job_rate(world, bench.BATCH, 5, 20.0) == pytest.approx(2 * 32 * 5 / 0.02)


def test_uneven_batches_differ_per_rank():
    a = bench.workload_specs("uneven", 0)
    b = bench.workload_specs("uneven", 1)
    assert len(a) == len(b) == 64
    assert [s[1] for s in a] != [s[1] for s in b]


def test_reference_arm_nonzero_rank_does_no_work(monkeypatch):
    """Under torchrun only rank 0 runs the oracle; the others return at once."""
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "cpu_oracle_rate", lambda *a, **k: called.append(1))

    class Args:
        gpus, steps, warmup = 2, 3, 3

    assert bench.run_reference(Args()) is None
    assert not called


def test_reference_arm_line_on_rank0(monkeypatch, capsys):
    """Rank 0 prints one JSON line in the bench contract, its value from the
    CPU oracle (here stubbed to a fixed rate), e2e without copies."""
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    calls = []

    def fake_rate(budget_s, max_shifts):
        calls.append(budget_s)
        return 0.25, 16, "stub sample"

    monkeypatch.setattr(bench, "cpu_oracle_rate", fake_rate)

    class Args:
        gpus, steps, warmup = 1, 3, 2

    bench.run_reference(Args())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert len(calls) == 5 and all(0.2 <= b <= 2.0 for b in calls)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] == pytest.approx(0.25) and line["ms_per_step"] == pytest.approx(4000.0)
    assert line["steps"] == 3 and line["warmup"] == 2 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 16
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_bench_work_accounting():
    """The headline's algorithmic and executed work per step (8N FLOP per paper
    term; per 16 amplitudes of a 64-term tile one FP16 MMA of 128 x 80 x 16 on
    the tensor cores, and of a pair of tiles one 128 x 128 x 16)."""
    shapes = [(10, 4, 64)] * 32
    terms, alg, exe = bench.work_of(shapes, tensor=True)
    assert terms == 32 * 101 * (64 * 64 + 64) == 13_445_120
    assert alg == terms * 8 * 1024  # 110.1 GFLOP
    assert exe == 32 * 101 * 2 * 128 * 80 * 16 * (1024 // 16) == 67_779_952_640
    # L = 256: four diagonal tiles and six pairs of tiles per shift
    _, _, exe_hs = bench.work_of([(10, 6, 256)], tensor=True)
    assert exe_hs == 141 * (4 * 2 * 128 * 80 * 16 * 64 + 6 * 2 * 128 * 128 * 16 * 64)
    # a state smaller than a stage still runs the stage's MMAs (zero rows)
    _, _, exe_small = bench.work_of([(4, 2, 16)], tensor=True)
    assert exe_small == 25 * 8 * 2 * 128 * 80 * 16
    _, _, exe_cc = bench.work_of(shapes, tensor=False)
    assert bench.executed_gram_entries(64) == 136 * 16
    assert bench.executed_gram_entries(128) == 2 * 136 * 16 + 2 * 128 * 16
    assert exe_cc == 32 * 101 * (136 * 16 * 2 * 1024 + 64 * 4 * 1024)


def test_bench_peaks_measured_or_fallback(monkeypatch):
    peaks, src = bench.measured_peaks()
    if src == "of measured":
        assert peaks["hbm_gbs"] > 1000 and peaks["bf16_tflops"] > 100
    monkeypatch.setattr(bench.os.path, "exists", lambda p: False)
    peaks, src = bench.measured_peaks()
    assert src == "of fallback" and peaks == {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
