"""The multi-rank leg of bench.py on CPU: two gloo ranks (replicas, no data
path collective) agree on the job time (max over ranks) and the whole-job
rate; the reference arm does its work on rank 0 only."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [80.0, 95.5][rank]
    job_ms = bench.max_over_ranks(ms, torch, "cpu", world)
    q.put((rank, job_ms, bench.job_rate(world, 1.0e10, job_ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_job_time_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [95.5, 95.5]
    assert all(abs(g[2] - 2 * 1.0e10 / 0.0955) < 1e-3 for g in got)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, torch, "cpu", 1) == 12.5
    assert bench.job_rate(1, 100.0, 1000.0) == 100.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        ref_sample, warmup, steps, gpus, separate = 48, 1, 1, 2, False
    assert bench.run_reference(A(), None) == 0
    assert capsys.readouterr().out == ""


def test_bench_json_parts_serialise_for_real_and_complex_k():
    """The bench line's host-side parts: the workload description for a real
    and a complex wavenumber (the profiling override), and the counted-flop
    roofline with the FP64 pipe figures, all JSON-serialisable; the counted
    rate is pairs x flops per pair / time over the stated peak."""
    import json
    import workloads as W

    class A:
        separate = False
        gpus = 1

    for k in (20.0, complex("20+1j")):
        wl = W.cfg2()
        wl.k = k
        cfg = bench.config_dict(wl, A())
        json.dumps(cfg)
        assert cfg["terms_per_step"] == 3 * wl.n_ctr * wl.n_src * (2 * wl.p + 1)
        assert ("20+1j" in cfg["workload"]) == isinstance(k, complex)
    hw = bench.hw_roofline(500.0, 10**8, 0.05, (0.9, 0.85))
    json.dumps(hw)
    assert abs(hw["achieved"] - 500.0 * 1e8 / 0.05 / 1e9) < 1e-9
    assert abs(hw["frac"] - hw["achieved"] / bench.FP64_PEAK_GFLOPS) < 1e-12
    assert hw["fp64_pipe_busy"]["of_elapsed_cycles"] == 0.85
    assert bench.hw_roofline(None, 1, 1.0) is None


def test_bench_spread_of_alternating_arms():
    """The batched comparison's statistics: median (mean of the middle two for
    an even count), min, max and sample count."""
    assert bench.spread([3.0, 1.0, 2.0]) == {"median": 2.0, "min": 1.0, "max": 3.0, "samples": 3}
    assert bench.spread([4.0, 1.0, 3.0, 2.0])["median"] == 2.5
