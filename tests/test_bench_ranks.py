"""The benchmark's multi-rank path on CPU (gloo, world size 2).

The CG does not shard across GPUs here (replicas only): each rank solves its
own system, and the process group only provides the barrier, the sum of the
work and the max of the time. These tests run that host logic with two gloo
ranks; nothing touches a GPU.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench

    ranks = bench.Ranks()
    try:
        assert ranks.backend == "gloo"
        ranks.barrier()
        # rank r did (r + 1) GFLOP in (r + 1) * 0.5 s
        rate, tmax = bench.whole_job_rate((rank + 1) * 1e9, (rank + 1) * 0.5, ranks)
        q.put((rank, rate, tmax))
        # the reference arm runs on rank 0 only; other ranks return without work
        if rank != 0:
            class A:
                steps, warmup, gpus = 1, 0, world

            bench.run_reference(A(), ranks)
            q.put((rank, "ref-skipped", None))
    finally:
        ranks.close()


def test_whole_job_rate_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    out = [q.get(timeout=5) for _ in range(3)]
    rates = [o for o in out if o[1] != "ref-skipped"]
    assert len(rates) == 2
    for _, rate, tmax in rates:
        assert tmax == pytest.approx(1.0)          # max over ranks
        assert rate == pytest.approx(3.0)          # (1 + 2) GFLOP / 1.0 s
    assert any(o[1] == "ref-skipped" and o[0] == 1 for o in out)


def test_single_rank_needs_no_process_group(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    import bench

    ranks = bench.Ranks()
    assert ranks.dist is None
    rate, tmax = bench.whole_job_rate(2e9, 0.5, ranks)
    assert rate == pytest.approx(4.0) and tmax == 0.5


def test_clock_sampler_keeps_only_the_timed_regions():
    """Samples are filtered by timestamp to the tagged timed regions (one record per tag prefix, or over all
    regions); samples of other GPUs are dropped; throttle reasons are read per field."""
    import datetime

    import bench

    rows = [
        "2026/01/01 10:00:00.000, GPU-abc, 1200, 2070, 300, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/01/01 10:00:01.000, GPU-abc, 2070, 2070, 900, 0x4, Not Active, Not Active, Not Active, Active",
        "2026/01/01 10:00:01.050, GPU-abc, 2055, 2070, 910, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/01/01 10:00:01.100, GPU-zzz, 900, 2070, 100, 0x0, Active, Not Active, Not Active, Not Active",
        "2026/01/01 10:00:05.000, GPU-abc, 800, 2070, 200, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/01/01 10:00:07.000, GPU-abc, 1980, 2070, 950, 0x0, Not Active, Active, Not Active, Not Active",
    ]

    class FakeProc:
        def terminate(self):
            pass

        def communicate(self, timeout=None):
            return "\n".join(rows) + "\n", ""

    c = bench.ClockSampler("GPU-abc")
    c.proc = FakeProc()
    T = lambda s_, us=0: datetime.datetime(2026, 1, 1, 10, 0, s_, us)  # noqa: E731
    c.windows = [("main", T(0, 500000), T(2)), ("forms.batched", T(6), T(8))]
    c.stop()
    out = c.summary("main")
    assert out["samples"] == 2
    assert out["sm_mhz"] == (2070 + 2055) / 2
    assert out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]
    f = c.summary("forms")
    assert f["samples"] == 1 and f["sm_mhz"] == 1980 and f["reasons"] == ["hw_thermal_slowdown"]
    assert c.summary("")["samples"] == 3
    assert c.summary("nothing") is None


def test_reference_arm_prints_its_contract_line():
    """`bench.py --impl reference` runs the oracle on the host and prints one JSON line with the keys the
    reference arm must carry (it needs no GPU)."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=900, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["value"] == d["value"]
