"""The multi-rank bits of bench.py on CPU (gloo, 2 ranks): the job time is the slowest
rank's, the job value aggregates the replicas, and only rank 0 runs the reference arm."""
import io
import contextlib
import multiprocessing as mp
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.max_over_ranks(1.5 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, v))


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 3.0, 1: 3.0}


def test_single_process_and_job_value():
    assert bench.max_over_ranks(2.5, "cpu") == 2.5
    assert bench.job_value(1000, 4, 500.0) == pytest.approx(8000.0)


def test_reference_arm_only_on_rank0(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(type("A", (), dict(steps=1, warmup=0))())
    assert buf.getvalue() == ""


def test_clock_summary_keeps_the_timed_region():
    """Only samples stamped inside the timed region count; a throttle reason outside it is not
    reported; a region between two samples takes the nearest one and says so."""
    import datetime

    base = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def line(dt_s, sm, reason=""):
        ts = (base + datetime.timedelta(seconds=dt_s)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        flags = ["Active" if reason == nm else "Not Active"
                 for nm in ("hw", "hw_thermal", "sw_thermal", "sw_power_cap")]
        return f"{ts}, 0, {sm} MHz, 2070 MHz, 900.00 W, 0x0, " + ", ".join(flags)

    lines = [line(0.0, 1200, "hw"), line(0.05, 2070), line(0.10, 2070, "sw_power_cap"), line(0.15, 2055),
             line(0.20, 1500, "hw_thermal"), "garbage"]
    t = lambda s: (base + datetime.timedelta(seconds=s)).timestamp()  # noqa: E731
    c = bench.summarise_clocks(lines, t(0.04), t(0.16))
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    c = bench.summarise_clocks(lines, t(0.16), t(0.17))
    assert c["samples"] == 0 and c["sm_mhz"] == 2055.0 and "note" in c
    assert bench.summarise_clocks([], t(0), t(1))["reasons"] == ["no samples"]
