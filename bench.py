#!/usr/bin/env python
"""Benchmark of the SE(2)-grid traversability hot path on the full local map:
400 x 400 cells at 0.05 m, 72 yaw bins, 0.9 x 0.6 m footprint, fractal terrain with steps and
5 % unknown cells.  One step = a full rebuild of the map (11.52 M SE(2) cells) followed by 50
rolling shifts of 10 cells in random directions, each recomputing only the affected bands (the
50 moves go through one seb_map_shift_batch call; their time as 50 separate seb_map_shift calls
is reported beside it).

Prints one JSON line.  value = SE(2) cells assessed per second over the timed steps (cells
actually recomputed: the rebuild plus every shift band), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (a bounded random sample of the
same workload's cells per step); under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 400
K = 72
RES = 0.05
LENGTH, WIDTH = 0.9, 0.6
# local-mapping cycle: the paper's densest configuration (18 x 18 m at 0.1 m, 30 yaw bins)
CYCLE_SIDE, CYCLE_RES, CYCLE_YAWS = 180, 0.1, 30
N_SHIFTS = 50
WORLD = 1200
WORKLOAD = "se2_map_400x400x72_rebuild_plus_50_shifts"
METRIC = "SE(2) cells/s (400x400x72 map: full rebuild + 50 rolling shifts per step)"

# ncu DRAM traffic of one full-map rebuild launch (dram__bytes_read.sum + dram__bytes_write.sum),
# valid only for the kernel source it was captured on (hash of the assess kernel's sources).
NCU_TRAFFIC = {"sources_sha": "a5cced13a7129ce9", "bytes": 768000 + 187603968}


def algorithmic_flop_per_cell(table):
    """Algorithmic FP32 FLOP of one cell and one yaw pair, by the direct count of Algorithm 1's
    arithmetic (an FMA counts 2): every footprint point is centred (1) and enters the four
    moment sums z', di z', dj z', z'^2 (8), and ~200 go to the covariance, eigen-solve, frame
    and risk of the pair: 9 N + 200 with N points."""
    return 9 * len(np.asarray(table)) + 200


def sliding_flop_per_cell(table):
    """Algorithmic FP32 FLOP of one cell and one yaw pair in the sliding-row-sum formulation
    (an FMA counts 2).  Per row run of length n the first column of a 4-column block sums n
    points (z - ref, A, B, C: 6 FLOP each); the other 3 columns slide the run by one cell
    (two new z' and 12 FLOP for A, B, C and the column's B: 14 each); each column then adds
    its run sums to S0..S3 (5).  Per cell: 1.5 N + 15.5 R, with N points and R runs, plus ~200
    for the eigen-solve, frame and risk of the pair."""
    t = np.asarray(table)
    runs = 0
    for dj in np.unique(t[:, 1]):
        di = np.sort(t[t[:, 1] == dj, 0])
        runs += 1 + int(np.count_nonzero(np.diff(di) > 1))
    return 1.5 * len(t) + 15.5 * runs + 200


def kernel_sources_sha():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2503_02412_gb300", "csrc")
    for f in ("seb_assess.cu", "seb_device.cuh", "seb_internal.h"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the per-row measurements")
    ap.add_argument("--sur-patches", type=int, default=200_000, help="surrogate training patches")
    ap.add_argument("--profile-cycle", action="store_true",
                    help="run only the local-mapping cycle row (the program profiled for its launch list)")
    ap.add_argument("--profile-query", action="store_true",
                    help="run three forward and three backward pose queries of 1,048,576 poses only")
    ap.add_argument("--profile-surrogate", action="store_true",
                    help="run five surrogate inferences (with the exact fallback) of the 400x400x72 map only")
    ap.add_argument("--profile-sdf", action="store_true",
                    help="three SDFs of the 400x400x72 risk grid and nothing else (for ncu)")
    ap.add_argument("--profile-rebuild", action="store_true",
                    help="only run three full rebuilds of the map (a short program for ncu)")
    ap.add_argument("--profile-shift", action="store_true",
                    help="only run a rebuild and three 10-cell moves as separate calls (for ncu)")
    ap.add_argument("--profile-train", action="store_true",
                    help="only run three surrogate training steps of 256 patches (for ncu)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def workload(seed=1):
    """World, window origins and shift sequence (identical on every rank: replicas)."""
    from synthetic import fractal_world, shift_sequence

    world = fractal_world(seed, WORLD, RES)
    o = [(WORLD - NX) // 2, (WORLD - NY) // 2]
    origins = [tuple(o)]
    for dx, dy in shift_sequence(seed + 1, N_SHIFTS, 10):
        o = [min(max(o[0] + dx, 0), WORLD - NX), min(max(o[1] + dy, 0), WORLD - NY)]
        origins.append(tuple(o))
    return world, origins


def oracle_params(**kw):
    """Oracle parameters (a plain record of the assessment parameters) of the 400x400x72 map, or
    of the given geometry.  The oracle's arithmetic runs only in the CPU-baseline leg."""
    import oracle

    return oracle.OracleParams(**(kw or dict(nx=NX, ny=NY, n_yaw=K, res=RES, length=LENGTH, width=WIDTH)))


def cpu_baseline(world, origins, budget_s, rng_seed=0, accuracy_jobs=None):
    """Times the FP64 oracle on a bounded random sample of the rebuild's cells: fresh random
    draws, each sized by a short calibration to about a second, until budget_s has passed.
    With accuracy_jobs, the same leg then runs the oracle on those fixed samples and reports the
    GPU's error against it (accuracy_vs_oracle)."""
    import oracle

    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    o = origins[0]
    e = world[o[1]:o[1] + NY, o[0]:o[0] + NX].astype(np.float64)
    rng = np.random.default_rng(rng_seed)
    p = oracle_params()

    def draw(n):
        return np.stack([rng.integers(0, NX, n), rng.integers(0, NY, n), rng.integers(0, K, n)], 1).astype(np.int32)

    n = 20000
    while True:  # calibrate: grow the draw until one takes about a second
        cells = draw(n)
        t0 = time.perf_counter()
        oracle.assess_cells(p, e, cells, o, n_threads=cores)
        dt = time.perf_counter() - t0
        if dt > min(1.0, budget_s / 4) or n >= 20_000_000:
            break
        n = int(n * min(8.0, max(2.0, min(1.0, budget_s / 4) / max(dt, 1e-3))))
    total_n, total_t, draws = 0, 0.0, 0
    while total_t < budget_s:
        cells = draw(n)
        t0 = time.perf_counter()
        oracle.assess_cells(p, e, cells, o, n_threads=cores)
        total_t += time.perf_counter() - t0
        total_n += n
        draws += 1
    res = {"value": total_n / total_t, "unit": "SE(2) cells/s", "cores": cores, "kind": "oracle",
           "sample": f"{total_n} random (c, r, k) cells of the 400x400x72 rebuild ({draws} draws of {n}), "
                     f"FP64 brute force, {total_t:.2f} s"}
    if accuracy_jobs:
        res["accuracy"] = accuracy_vs_oracle(accuracy_jobs, cores)
    return res


def accuracy_vs_oracle(jobs, cores):
    """Part of the CPU-baseline leg: runs the FP64 oracle on fixed samples of cells and reports
    the error of the GPU outputs on them, per output channel (max and p99 |delta| over the
    cells both sides assess; z in m, angles in rad), with the count of cells whose FP32
    conditioning bound C_GAP u / (g n_z) exceeds 1e-4 (g the oracle's relative eigen-gap).
    jobs: {label: (geometry dict, elevation [ny][nx] float64, cells [n][3] (c, r, k), origin,
    gpu outputs [n][5], gpu flags [n])}."""
    import oracle

    u32, c_gap = 2.0 ** -24, 16.0
    out = {}
    for label, (geom, elev, cells, origin, g, gf) in jobs.items():
        r, rf, gap = oracle.assess_cells(oracle_params(**geom), elev, cells, origin, n_threads=cores)
        ok = ((rf & 5) == 0) & ((gf & 5) == 0)
        d = np.abs(g[ok].astype(np.float64) - r[ok])
        with np.errstate(invalid="ignore", divide="ignore"):
            sp, sr = np.sin(r[ok, 1]), np.sin(r[ok, 2])
            nz = np.sqrt(np.clip(1 - sp * sp - sr * sr, 1e-12, 1))
            ill = int((c_gap * u32 / (gap[ok] * nz) > 1e-4).sum())
        row = {"cells": int(len(cells)), "assessed_both": int(ok.sum()), "ill_conditioned": ill,
               "unknown_bits_equal": bool(np.array_equal(rf & 1, gf & 1))}
        for ch, name in enumerate(("z", "pitch", "roll", "rough", "risk")):
            row[name] = {"max": float(d[:, ch].max()) if d.size else None,
                         "p99": float(np.percentile(d[:, ch], 99)) if d.size else None}
        out[label] = row
    return out


class Clocks:
    """nvidia-smi sampling of the SM clock and the throttle reasons.  Sampling is live before
    start() returns, and only the samples stamped between start() and stop() count."""

    INTERVAL_MS = 50

    def __init__(self, index):
        d = os.environ.get("SEB_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(d, f"seb_clocks_rank{index}.csv")
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.t0 = self.t1 = None
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader",
                                       "-lms", str(self.INTERVAL_MS)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
            return
        deadline = time.time() + 10.0  # the first sample: nvidia-smi has started
        while time.time() < deadline and self.p.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(2 * self.INTERVAL_MS / 1e3)  # the sample in flight lands
        self.p.terminate()
        self.p.wait()
        self.f.close()
        return summarise_clocks(open(self.path).read().splitlines(), self.t0, self.t1)


def summarise_clocks(lines, t0, t1):
    """Median SM clock, maximum clock and the throttle reasons seen in the samples stamped
    within [t0, t1] (host epoch seconds).  A region shorter than the sampling interval holds
    no sample; it then takes the one nearest its middle and says so."""
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            sm, smax = float(parts[2].split()[0]), float(parts[3].split()[0])
        except ValueError:
            continue
        rows.append((ts, sm, smax, [nm for nm, v in zip(names, parts[6:10]) if v.lower().startswith("active")]))
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    inside = [r for r in rows if t0 is not None and t0 <= r[0] <= t1]
    note = None
    if not inside:
        mid = 0.5 * (t0 + t1) if t0 is not None else rows[-1][0]
        inside = [min(rows, key=lambda r: abs(r[0] - mid))]
        note = "timed region shorter than the sampling interval: the sample nearest its middle"
    out = {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": float(max(r[2] for r in inside)),
           "reasons": sorted({nm for r in inside for nm in r[3]}), "samples": len(inside) if note is None else 0,
           "interval_ms": Clocks.INTERVAL_MS}
    if note:
        out["note"] = note
    return out


def max_over_ranks(x, device):
    """Maximum of a float over the ranks of the job (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells_per_rank, world_size, job_ms):
    """Whole-job throughput: every rank (a replica) assesses its own map."""
    return cells_per_rank * world_size / (job_ms / 1e3)


def flush_l2(buf):
    buf.add_(1)  # writes 256 MB (> 129 MB L2)


def run_reference(args):
    rank, _, world_size = dist_env()
    if rank != 0:
        return
    world, origins = workload()
    per_step = max(1.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    cb = cpu_baseline(world, origins, min(5.0, per_step * 4))  # sizes the steps only
    import oracle

    p = oracle_params()
    o = origins[0]
    e = world[o[1]:o[1] + NY, o[0]:o[0] + NX].astype(np.float64)
    rng = np.random.default_rng(1)
    n = int(cb["value"] * per_step)
    cells = np.stack([rng.integers(0, NX, n), rng.integers(0, NY, n), rng.integers(0, K, n)], 1).astype(np.int32)
    for _ in range(args.warmup):
        oracle.assess_cells(p, e, cells[: max(1, n // 10)], o, n_threads=cb["cores"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.assess_cells(p, e, cells, o, n_threads=cb["cores"])
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "SE(2) cells/s", "n_gpus": world_size, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_cells_per_step": n, "l2": "n/a (host)"},
            "cpu_baseline": dict(cb, value=value,
                                 sample=f"{n} random (c, r, k) cells per step of the 400x400x72 map, FP64 oracle"),
            "e2e": {"value": value, "unit": "SE(2) cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def profile_query():
    """Three forward and three backward continuous-pose queries of 1,048,576 poses on the
    100x100 map at 0.1 m (0.6x0.4 m footprint, 36 yaw bins)."""
    import torch

    import paper_2503_02412_gb300 as seb
    from paper_2503_02412_gb300 import abi
    from synthetic import bumpy_plane, random_poses

    dev = torch.device("cuda")
    st = torch.cuda.current_stream(dev)
    c = seb.SebParams(nx=100, ny=100, n_yaw=36, res=0.1, length=0.6, width=0.4).c()
    e = torch.from_numpy(bumpy_plane(0)).to(dev)
    n = 1 << 20
    poses = torch.from_numpy(random_poses(4, n, 100, 100, 0.1, 5)).to(dev)
    out = torch.empty(n, 5, device=dev)
    fl = torch.empty(n, dtype=torch.uint8, device=dev)
    sv = torch.empty(n, abi.SEB_QUERY_SAVED, device=dev)
    g = torch.randn(n, 5, device=dev)
    gp = torch.empty(n, 3, device=dev)
    for _ in range(3):
        abi.seb_query_poses(c, e.data_ptr(), 0, 0, poses.data_ptr(), n, out.data_ptr(), fl.data_ptr(), sv.data_ptr(),
                            st.cuda_stream)
    for _ in range(3):
        abi.seb_query_poses_backward(c, e.data_ptr(), 0, 0, poses.data_ptr(), sv.data_ptr(), g.data_ptr(), gp.data_ptr(),
                                     n, st.cuda_stream)
    torch.cuda.synchronize()


def profile_surrogate():
    """Five surrogate inferences of the 400x400x72 fractal map with the exact fallback (weights
    from the seeded initialisation: the timing does not depend on them)."""
    import torch

    import paper_2503_02412_gb300 as seb
    from paper_2503_02412_gb300 import surrogate
    from synthetic import fractal_steps_nan

    s = surrogate.Surrogate(seb.SebParams(nx=NX, ny=NY, n_yaw=K, res=RES, length=LENGTH, width=WIDTH), max_batch=256)
    s.init(11)
    e = torch.from_numpy(fractal_steps_nan(13)).cuda()
    out, fl, mask = s.infer(e)
    for _ in range(4):
        s.infer_into(e, out, fl, mask)
    torch.cuda.synchronize()


def profile_rebuild():
    """Three rebuilds of the 400x400x72 map and nothing else: the program ncu captures."""
    import torch

    import paper_2503_02412_gb300 as seb
    from synthetic import fractal_steps_nan

    e = torch.from_numpy(fractal_steps_nan(0)).cuda()
    m = seb.SebMap(seb.SebParams(nx=NX, ny=NY, n_yaw=K, res=RES, length=LENGTH, width=WIDTH))
    for _ in range(3):
        m.update(e)
    m.check()
    torch.cuda.synchronize()


def profile_shift():
    """A rebuild of the 400x400x72 map and the first three 10-cell moves of the bench workload as
    separate seb_map_shift calls, nothing else: the program ncu captures (launch 2 is a move)."""
    import torch

    import paper_2503_02412_gb300 as seb

    world_np, origins = workload()
    world = torch.from_numpy(world_np).cuda()
    wins = [world[o[1]:o[1] + NY, o[0]:o[0] + NX].contiguous() for o in origins[:4]]
    m = seb.SebMap(seb.SebParams(nx=NX, ny=NY, n_yaw=K, res=RES, length=LENGTH, width=WIDTH))
    m.update(wins[0], origins[0])
    for w, o in zip(wins[1:], origins[1:4]):
        m.shift(w, o)
    m.check()
    torch.cuda.synchronize()


def profile_train():
    """Three surrogate training steps of 256 patches (one labelled batch, tcgen05 engine) after
    the batch is made: the program ncu captures for the backward kernels."""
    import torch

    import paper_2503_02412_gb300 as seb
    from paper_2503_02412_gb300 import abi, surrogate

    s = surrogate.Surrogate(seb.SebParams(nx=NX, ny=NY, n_yaw=K, res=RES, length=LENGTH, width=WIDTH), max_batch=256)
    s.init(11)
    s.make_batch(np.random.default_rng(0), 256)
    for i in range(3):
        abi.seb_sur_train_step(s.handle, 256, 1e-3, i + 1, 0)
    torch.cuda.synchronize()


def profile_sdf():
    """Three signed distance fields of the 400x400x72 fractal map's risk channel (obstacles
    risk >= 1, clamp 2 m) after one rebuild: the program ncu captures."""
    import torch

    import paper_2503_02412_gb300 as seb
    from paper_2503_02412_gb300 import abi
    from synthetic import fractal_steps_nan

    m = seb.SebMap(seb.SebParams(nx=NX, ny=NY, n_yaw=K, res=RES, length=LENGTH, width=WIDTH))
    m.update(torch.from_numpy(fractal_steps_nan(0)).cuda())
    risk = seb.SE2Grid.from_map(m, 4)
    out = torch.empty((K, NY, NX), device="cuda")
    work = torch.empty(abi.seb_sdf_workspace_bytes(NX, NY, K), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        seb.risk_sdf(risk, 1.0, 2.0, out=out, work=work)
    m.check()
    torch.cuda.synchronize()


def main():
    args = parse()
    if args.profile_rebuild:
        return profile_rebuild()
    if args.profile_sdf:
        return profile_sdf()
    if args.profile_shift:
        return profile_shift()
    if args.profile_train:
        return profile_train()
    if args.profile_surrogate:
        return profile_surrogate()
    if args.profile_query:
        return profile_query()
    if args.profile_cycle:
        import torch

        import paper_2503_02412_gb300 as seb

        dev = torch.device("cuda", 0)
        print(json.dumps(local_mapping_cycle(seb, dev, torch.cuda.current_stream(dev))))
        return None
    if args.impl == "reference":
        return run_reference(args)
    rank, local_rank, world_size = dist_env()
    import torch

    if world_size > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    import paper_2503_02412_gb300 as seb
    from paper_2503_02412_gb300 import abi

    abi.load()  # fails loudly if the CUDA library is missing: no fallback
    world_np, origins = workload()
    world = torch.from_numpy(world_np).to(dev)
    wins = [world[o[1]:o[1] + NY, o[0]:o[0] + NX].contiguous() for o in origins]
    params = seb.SebParams(nx=NX, ny=NY, n_yaw=K, res=RES, length=LENGTH, width=WIDTH)
    m = seb.SebMap(params, dev)
    stream = torch.cuda.current_stream(dev)
    l2buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step(ev_rebuild=None):
        if ev_rebuild is not None:
            ev_rebuild[0].record(stream)
        m.update(wins[0], origins[0])
        if ev_rebuild is not None:
            ev_rebuild[1].record(stream)
        cells = m.view().last_cells
        m.shift_batch(wins[1:], origins[1:])
        cells += m.view().last_cells
        return cells

    for _ in range(args.warmup):
        step()
    m.check()
    torch.cuda.synchronize(dev)
    if world_size > 1:
        torch.distributed.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    total_ms = 0.0
    rebuild_ms = []
    cells_total = 0
    launches = 0
    for _ in range(args.steps):
        flush_l2(l2buf)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        cells_total += step((ev[2], ev[3]))
        ev[1].record(stream)
        ev[1].synchronize()
        total_ms += ev[0].elapsed_time(ev[1])
        rebuild_ms.append(ev[2].elapsed_time(ev[3]))
        launches += 1 + sum(1 for i in range(1, len(origins)) if origins[i] != origins[i - 1])
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    n64, ndeg = m.check()
    total_ms = max_over_ranks(total_ms, dev)
    if world_size > 1:
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = job_value(cells_total, world_size, total_ms)
    # the same 50 moves as separate seb_map_shift calls (each waits for the previous kernel)
    m.update(wins[0], origins[0])
    es = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    es[0].record(stream)
    for w, o in zip(wins[1:], origins[1:]):
        m.shift(w, o)
    es[1].record(stream)
    es[1].synchronize()
    shift_single_us = es[0].elapsed_time(es[1]) / N_SHIFTS * 1e3

    # roofline of the dominant kernel (the full-map rebuild launch)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    tables = [abi.seb_footprint_table(params.c(), k) for k in range(K // 2)]
    flop = NX * NY * sum(algorithmic_flop_per_cell(t) for t in tables)
    flop_exec = NX * NY * sum(sliding_flop_per_cell(t) for t in tables)
    rb = float(np.mean(rebuild_ms))
    achieved = flop / (rb * 1e-3) / 1e12
    achieved_exec = flop_exec / (rb * 1e-3) / 1e12
    peak = sms * 128 * 2 * 2070e6 / 1e12  # FP32 lanes x FMA x max SM clock
    traffic = NCU_TRAFFIC["bytes"] if NCU_TRAFFIC["sources_sha"] == kernel_sources_sha() else None

    # the whole step against the same peak: the rebuild's FLOP plus those of every cell the 50
    # moves recompute (each recomputed (x, y) cell takes all K yaws, i.e. sum over the pairs)
    flop_xy = sum(algorithmic_flop_per_cell(t) for t in tables)  # one (x, y) cell, all yaw pairs
    cells_per_step = cells_total // args.steps
    step_flop = cells_per_step / K * flop_xy
    shift_flop = (cells_per_step - NX * NY * K) / K * flop_xy / N_SHIFTS
    shift_us = (ms_per_step - rb) / N_SHIFTS * 1e3

    # the rolled map after the 50 separate shifts above, sampled for the oracle comparison of the
    # CPU-baseline leg (rolling is bit-identical to a rebuild, so this is also the rebuild's error)
    acc_jobs = {}
    if rank == 0 and world_size == 1 and not args.no_cpu_baseline:
        out_l, fl_l = m.outputs()
        rng = np.random.default_rng(11)
        ns = 1_000_000
        cs = np.stack([rng.integers(0, NX, ns), rng.integers(0, NY, ns), rng.integers(0, K, ns)], 1).astype(np.int32)
        cti = torch.from_numpy(cs.astype(np.int64)).to(dev)
        g = out_l[:, cti[:, 2], cti[:, 1], cti[:, 0]].T.contiguous().cpu().numpy()
        gf = fl_l[cti[:, 2], cti[:, 1], cti[:, 0]].cpu().numpy()
        of = origins[-1]
        acc_jobs["400x400x72_after_50_shifts"] = (
            dict(nx=NX, ny=NY, n_yaw=K, res=RES, length=LENGTH, width=WIDTH),
            world_np[of[1]:of[1] + NY, of[0]:of[0] + NX].astype(np.float64), cs, tuple(of), g, gf)
        del out_l, fl_l

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(seb, m, world_np, origins, args, dev)
    rows = None if args.no_rows or world_size > 1 else measure_rows(seb, args, dev, acc_jobs)
    line = {
        "metric": METRIC,
        "value": value, "unit": "SE(2) cells/s", "n_gpus": world_size, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "n_yaw": K, "res_m": RES,
                   "footprint_m": [LENGTH, WIDTH], "shifts_per_step": N_SHIFTS,
                   "cells_per_step": cells_total // args.steps, "parallelism": f"replicas x{world_size}",
                   "l2": "flushed before every timed step (256 MB write)"},
        "rebuild_ms": rb, "rebuild_cells_per_s": NX * NY * K / (rb * 1e-3),
        "shift_us_mean": (ms_per_step - rb) / N_SHIFTS * 1e3,
        "shift_us_mean_single_calls": shift_single_us,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "assess_kernel_sl<float> (rebuild)",
                     "flop_per_launch": flop,
                     "flop_basis": "algorithmic: 9 N + 200 per cell and yaw pair (N footprint points)",
                     "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x 2070 MHz",
                     "executed": {"flop_per_launch": flop_exec, "achieved": achieved_exec, "frac": achieved_exec / peak,
                                  "flop_basis": "sliding row sums as run: 1.5 N + 15.5 R + 200 per cell and yaw pair"},
                     "step": {"flop": step_flop, "achieved": step_flop / (ms_per_step * 1e-3) / 1e12,
                              "frac": step_flop / (ms_per_step * 1e-3) / 1e12 / peak,
                              "basis": "rebuild + 50 shifts in one batch: recomputed cells x the same per-cell FLOP"},
                     "shift": {"flop_mean": shift_flop, "us_mean": shift_us,
                               "achieved": shift_flop / (shift_us * 1e-6) / 1e12,
                               "frac": shift_flop / (shift_us * 1e-6) / 1e12 / peak,
                               "basis": "one 10-cell move of the batch: band cells x the same per-cell FLOP"}},
        "gpu_launches": launches, "fp64_solves": n64, "degenerate": ndeg, "clocks": clk,
    }
    if e2e is not None:
        line["e2e"] = e2e
    if rows is not None:
        line["rows"] = rows
    if rank == 0 and world_size == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(world_np, origins, args.cpu_seconds, accuracy_jobs=acc_jobs)
        line["accuracy"] = line["cpu_baseline"].pop("accuracy", None)
    if rank == 0:
        print(json.dumps(line))
    if world_size > 1:
        torch.distributed.destroy_process_group()


def _time(fn, reps, stream):
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_rows(seb, args, dev, acc_jobs=None):
    """The other rows of the hot path, each on its own configuration, outside the timed step:
    continuous-pose query forward / backward (1,048,576 poses on the 100x100 map), the
    reduced-precision rebuild (1024x1024x72, FP32 / BF16 / FP16 elevation) and the learned
    surrogate against the exact kernel on the 400x400x72 map."""
    import torch

    from paper_2503_02412_gb300 import abi
    from paper_2503_02412_gb300.surrogate import Surrogate
    from synthetic import bumpy_plane, fractal_steps_nan, random_poses

    st = torch.cuda.current_stream(dev)
    rows = {}
    # S9 / S10
    pq = seb.SebParams(nx=100, ny=100, n_yaw=36, res=0.1, length=0.6, width=0.4)
    e = torch.from_numpy(bumpy_plane(0)).to(dev)
    n = 1 << 20
    poses = torch.from_numpy(random_poses(4, n, 100, 100, 0.1, 5)).to(dev)
    out = torch.empty(n, 5, device=dev)
    fl = torch.empty(n, dtype=torch.uint8, device=dev)
    sv = torch.empty(n, abi.SEB_QUERY_SAVED, device=dev)
    g = torch.randn(n, 5, device=dev)
    gp = torch.empty(n, 3, device=dev)
    c = pq.c()
    fwd = lambda: abi.seb_query_poses(c, e.data_ptr(), 0, 0, poses.data_ptr(), n, out.data_ptr(), fl.data_ptr(),  # noqa: E731
                                      sv.data_ptr(), st.cuda_stream)
    bwd = lambda: abi.seb_query_poses_backward(c, e.data_ptr(), 0, 0, poses.data_ptr(), sv.data_ptr(),  # noqa: E731
                                               g.data_ptr(), gp.data_ptr(), n, st.cuda_stream)
    tf, tb = _time(fwd, 10, st), _time(bwd, 10, st)
    # the query gathers 4 bilinear corners per lattice point; the 40 KB map is copied into every
    # CTA's shared memory, so its roofline is the shared-memory bandwidth (152 SMs x 128 bytes per
    # clock at 2070 MHz, from the unit counts: no measured figure); the L2 read bandwidth, measured
    # by summing an L2-resident buffer, is reported beside it
    l2 = l2_read_gbs(dev, st)
    n_lat = len(abi.seb_footprint_table(c, 0))
    gather = n * n_lat * 4 * 4  # bytes of corner heights read per forward
    smem_gbs = torch.cuda.get_device_properties(dev).multi_processor_count * 128 * 2070e6 / 1e9
    ach = gather / (tf * 1e-3) / 1e9
    rows["query_1M_poses"] = {"fwd_ms": tf, "bwd_ms": tb, "fwd_poses_per_s": n / tf * 1e3,
                              "bwd_poses_per_s": n / tb * 1e3, "config": "100x100 map at 0.1 m, 0.6x0.4 m",
                              "roofline": {"bound": "smem", "gather_bytes_fwd": gather, "achieved_gbs_fwd": ach,
                                           "peak_gbs": smem_gbs, "frac_fwd": ach / smem_gbs,
                                           "peak_basis": "SMs x 128 bytes per clock x 2070 MHz (unit counts)",
                                           "l2_peak_gbs": l2, "frac_fwd_of_l2": ach / l2,
                                           "l2_basis": "measured: L2-resident 16 MB copy, read + write bytes"}}
    # trilinear SE(2) lookup of the grid at the same poses, against the exact query
    abi.seb_query_poses(c, e.data_ptr(), 0, 0, poses.data_ptr(), n, out.data_ptr(), fl.data_ptr(), 0, st.cuda_stream)
    mq = seb.SebMap(pq, dev)
    mq.update(e)
    val = torch.empty(n, device=dev)
    grad = torch.empty(n, 3, device=dev)
    lfl = torch.empty(n, dtype=torch.uint8, device=dev)
    gv = torch.randn(n, device=dev)
    grids = [abi.seb_map_grid(mq.handle, ch) for ch in range(5)]
    lk = lambda: abi.seb_se2_lookup(grids[4], poses.data_ptr(), n, 1.0, val.data_ptr(), grad.data_ptr(),  # noqa: E731
                                    lfl.data_ptr(), st.cuda_stream)
    lkv = lambda: abi.seb_se2_lookup_vjp(grids[4], poses.data_ptr(), n, gv.data_ptr(), gp.data_ptr(),  # noqa: E731
                                         st.cuda_stream)
    tl, tv = _time(lk, 20, st), _time(lkv, 20, st)
    err = {}
    known = fl == 0
    for ch, name in ((0, "z"), (1, "pitch"), (2, "roll"), (4, "risk")):
        abi.seb_se2_lookup(grids[ch], poses.data_ptr(), n, float("nan"), val.data_ptr(), None, None, st.cuda_stream)
        d = (val - out[:, ch]).abs()[known & torch.isfinite(val)]
        err[f"{name}_p50"] = float(d.quantile(0.5)) if d.numel() else None
        err[f"{name}_p99"] = float(d.quantile(0.99)) if d.numel() else None
    rows["lookup_1M_poses"] = {"value_grad_ms": tl, "vjp_ms": tv, "poses_per_s": n / tl * 1e3,
                               "vs_exact_query_fwd": tf / tl, "error_vs_exact_query": err,
                               "config": "risk channel of the 100x100x36 map at the query's poses"}
    del poses, out, fl, sv, g, gp, val, grad, lfl, gv, mq
    # signed distance field of the obstacle set of the 400x400x72 map, read back by the lookup
    mc2 = seb.SebMap(seb.SebParams(nx=NX, ny=NY, n_yaw=K, res=RES, length=LENGTH, width=WIDTH), dev)
    mc2.update(torch.from_numpy(fractal_steps_nan(0)).to(dev))
    risk = seb.SE2Grid.from_map(mc2, 4)
    sdf_t = torch.empty((K, NY, NX), device=dev)
    work = torch.empty(abi.seb_sdf_workspace_bytes(NX, NY, K), dtype=torch.uint8, device=dev)
    sdf_grid = seb.risk_sdf(risk, 1.0, 2.0, out=sdf_t, work=work)
    ts = _time(lambda: seb.risk_sdf(risk, 1.0, 2.0, out=sdf_t, work=work), 20, st)
    n2 = 1 << 20
    p2 = torch.from_numpy(random_poses(5, n2, NX, NY, RES, 12)).to(dev)
    v2 = torch.empty(n2, device=dev)
    g2 = torch.empty(n2, 3, device=dev)
    tl2 = _time(lambda: abi.seb_se2_lookup(sdf_grid.g, p2.data_ptr(), n2, 2.0, v2.data_ptr(), g2.data_ptr(), None,
                                           st.cuda_stream), 20, st)
    obst = float((sdf_t < 0).float().mean())
    rows["sdf_400x400x72"] = {"sdf_ms": ts, "cells_per_s": NX * NY * K / ts * 1e3, "obstacle_frac": obst,
                              "lookup_1M_value_grad_ms": tl2,
                              "hbm_gbs": 16 * NX * NY * K / ts / 1e6,  # risk in, work out + in, sdf out
                              "config": "risk channel of the 400x400x72 fractal map, obstacles risk >= 1, clamp 2 m"}
    # nearest-neighbour inpainting of the same map before its assessment
    e2 = torch.from_numpy(fractal_steps_nan(0)).to(dev)
    filled = torch.empty_like(e2)
    iw = torch.empty(abi.seb_inpaint_workspace_bytes(NX, NY), dtype=torch.uint8, device=dev)
    seb.inpaint_nearest(e2, 0, out=filled, work=iw)
    # the C ABI call itself (the Python wrapper's host overhead exceeds these ~10 us kernels)
    ti = _time(lambda: abi.seb_inpaint_nearest(e2.data_ptr(), NX, NY, 0, iw.data_ptr(), iw.numel(), filled.data_ptr(),
                                               None, st.cuda_stream), 50, st)
    tu = _time(lambda: mc2.update(filled), 10, st)
    n_unknown_raw = float(torch.isnan(e2).float().mean())
    rows["inpaint_400x400"] = {"inpaint_ms": ti, "rebuild_after_inpaint_ms": tu, "unknown_frac_before": n_unknown_raw,
                               "config": "fractal map with 5 % NaN discs, unbounded nearest-neighbour filling"}
    del mc2, sdf_t, work, p2, v2, g2, sdf_grid, risk, e2, filled, iw
    rows["local_mapping_cycle_180x180x30"] = local_mapping_cycle(seb, dev, st)
    # S8: every storage / summation form on the 1024 x 1024 x 72 map, timed, and its outputs on a
    # fixed sample of 20,000 cells kept for the oracle comparison of the CPU-baseline leg (against
    # the unquantised FP64 terrain: the whole error of the form; and against the heights the form
    # stores: the arithmetic's share)
    e3_64 = bumpy_plane(21, 1024, 1024, 0.05, dtype=np.float64)
    e3 = torch.from_numpy(e3_64.astype(np.float32)).to(dev)
    rng = np.random.default_rng(4)
    cells3 = np.stack([rng.integers(0, 1024, 20000), rng.integers(0, 1024, 20000), rng.integers(0, 72, 20000)],
                      1).astype(np.int32)
    ci = torch.from_numpy(cells3.astype(np.int64)).to(dev)
    prec = {}
    C3 = dict(nx=1024, ny=1024, n_yaw=72, res=0.05, length=0.9, width=0.6)
    forms = (("f32", dict(elev_dtype=torch.float32), e3),
             ("bf16", dict(elev_dtype=torch.bfloat16), e3.to(torch.bfloat16)),
             ("f16", dict(elev_dtype=torch.float16), e3.to(torch.float16)),
             ("bf16_tiled", dict(elev_dtype="bf16_tiled"), seb.encode_bf16_tiled(e3)),
             ("f32_compensated", dict(precision="compensated"), e3))
    for name, kw, ed in forms:
        m = seb.SebMap(seb.SebParams(**C3, **kw), dev)
        t = _time(lambda: m.update(ed), 5, st)
        prec[name] = {"rebuild_ms": t, "cells_per_s": 1024 * 1024 * 72 / t * 1e3}
        g = m.out_phys[:, ci[:, 2], ci[:, 1], ci[:, 0]].T.contiguous().cpu().numpy()
        gf = m.flags_phys[ci[:, 2], ci[:, 1], ci[:, 0]].cpu().numpy()
        if acc_jobs is not None:
            op = dict(C3)  # the oracle's parameters are built in the CPU-baseline leg
            acc_jobs[f"1024x1024x72_{name}_vs_fp64_terrain"] = (op, e3_64, cells3, (0, 0), g, gf)
            if name in ("bf16", "f16"):
                stored = ed.float().cpu().numpy().astype(np.float64)
                acc_jobs[f"1024x1024x72_{name}_vs_stored_heights"] = (op, stored, cells3, (0, 0), g, gf)
            elif name == "bf16_tiled":
                d, b = seb.tiled_parts(ed, 1024, 1024)
                idx = np.arange(1024) // 16
                stored = (b.cpu().numpy()[idx][:, idx] + d.float().cpu().numpy()).astype(np.float32)
                acc_jobs[f"1024x1024x72_{name}_vs_stored_heights"] = (op, stored.astype(np.float64), cells3, (0, 0), g,
                                                                      gf)
        del m
        torch.cuda.empty_cache()
    rows["precision_1024x1024x72"] = prec
    # S11 / S12
    C2 = dict(nx=NX, ny=NY, n_yaw=K, res=RES, length=LENGTH, width=WIDTH)
    sur = Surrogate(seb.SebParams(**C2), max_batch=256, device=dev)
    sur.init(11)
    t0 = time.perf_counter()
    losses = sur.train(args.sur_patches, batch=256, lr=3e-3, seed=4000, log_every=50)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    em = torch.from_numpy(fractal_steps_nan(13)).to(dev)
    m = seb.SebMap(seb.SebParams(**C2), dev)
    m.update(em)
    ex, exf = m.outputs()
    o, f, mk = sur.infer(em)
    surc = ((f & abi.SEB_FLAG_SURROGATE) != 0) & ((exf & 5) == 0)
    err = {}
    for ch, nm in ((0, "z"), (1, "pitch"), (2, "roll"), (4, "risk")):
        d = (o[ch] - ex[ch]).abs()[surc]
        err[nm + "_p50"] = float(d.median())
        err[nm + "_p99"] = float(torch.quantile(d[: 1 << 20].float(), 0.99))
    t_exact = _time(lambda: m.update(em), 10, st)
    t_sur = _time(lambda: sur.infer_into(em, o, f, mk, exact_fallback=False), 10, st)
    t_all = _time(lambda: sur.infer_into(em, o, f, mk), 10, st)
    # tensor-pipe share of the batch path: the three 32 -> 32 layers run as tcgen05 implicit GEMMs
    # (forward; backward dgrad and wgrad with the gradient split into two BF16 operands)
    bt = 256
    t_fwd = _time(lambda: abi.seb_sur_forward(sur.handle, bt), 10, st)
    t_step = _time(lambda: abi.seb_sur_train_step(sur.handle, bt, 1e-6, 10_000, 0), 10, st)
    sides = (46, 44, 40, 32, 16)
    mm = 2 * 288 * 32  # FLOP per pixel of one 32 -> 32 layer (and of its dgrad / wgrad)
    f_fwd = bt * mm * sum(sides[l + 1] ** 2 for l in (1, 2, 3))
    f_bwd = bt * mm * sum(sides[l] ** 2 + sides[l + 1] ** 2 for l in (1, 2, 3))  # dgrad + wgrad, algorithmic
    peak_bf16 = measured_peak("bf16_tflops_sustained", 1708.0)
    rows["surrogate_400x400x72"] = {
        "train_patches": args.sur_patches, "train_s": train_s, "loss_first": losses[0][1], "loss_last": losses[-1][1],
        "engine": "tcgen05", "fallback_frac": float(mk.float().mean()), "error_vs_exact_on_surrogate_cells": err,
        "exact_rebuild_ms": t_exact, "surrogate_only_ms": t_sur, "surrogate_with_fallback_ms": t_all,
        "gain_vs_exact": t_exact / t_all,
        "tensor_pipe": {
            "batch": bt, "forward_ms": t_fwd, "train_step_ms": t_step,
            "tcgen05_flop_forward": f_fwd, "tcgen05_flop_train_step": f_fwd + f_bwd,
            "achieved_tflops_forward": f_fwd / (t_fwd * 1e-3) / 1e12,
            "achieved_tflops_train_step": (f_fwd + f_bwd) / (t_step * 1e-3) / 1e12,
            "peak_tflops": peak_bf16, "peak_basis": "measured BF16 dense, sustained",
            "frac_forward": f_fwd / (t_fwd * 1e-3) / 1e12 / peak_bf16,
            "frac_train_step": (f_fwd + f_bwd) / (t_step * 1e-3) / 1e12 / peak_bf16,
            "basis": "algorithmic FLOP of the tcgen05 layers over the whole forward / train-step time (the first "
                     "layer, the head, the loss and Adam run on CUDA cores inside the same time)"}}
    return rows


def l2_read_gbs(dev, st, mb=16, reps=100):
    """Throughput of the L2 cache: a 16 MB float buffer copied into another (both L2-resident
    after the first pass) reps times, bytes read plus written over CUDA-event time."""
    import torch

    a = torch.ones(mb * 1024 * 1024 // 4, device=dev)
    b = torch.empty_like(a)
    for _ in range(3):
        b.copy_(a)
    t = _time(lambda: b.copy_(a), reps, st)
    return 2 * a.numel() * 4 / (t * 1e-3) / 1e9


def measured_peak(key, fallback):
    """A peak from MEASURED_PEAKS.json at the repository root, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except (OSError, KeyError, ValueError):
        return fallback


def local_mapping_cycle(seb, dev, st, n_scans=6, reps=5):
    """The whole GPU local-mapping cycle of Sec. V on the paper's densest configuration (18 x 18 m
    at 0.1 m, 30 yaw bins: 972,000 SE(2) cells): one synthetic LiDAR scan (32 x 1024 rays) ->
    elevation update (window move, ray casting, filtering, variances, Kalman fusion) -> window
    copy -> nearest-neighbour inpainting -> full traversability rebuild -> signed distance field
    of the obstacles.  Scans are generated on the host beforehand along a path and are resident
    on the device; the cycle is timed with CUDA events."""
    import torch

    from synthetic import fractal_world, lidar_scan

    n, K, res = CYCLE_SIDE, CYCLE_YAWS, CYCLE_RES
    world = fractal_world(7, 700, res=res)
    S_S = np.diag([0.02, 0.02, 0.02]) ** 2
    S_R = np.diag([0.004, 0.004, 0.002]) ** 2
    S_B = np.diag([0.01, 0.01, 0.01]) ** 2
    scans = []
    for k in range(n_scans):
        x, y, yaw = 30.0 + 0.15 * k, 30.0 + 0.05 * k, 0.1 * k
        R_B, p_B, R_BS, p_BS, pts = lidar_scan(100 + k, world, res, x, y, yaw, n_rings=32, n_az=1024, max_range=9.0)
        scans.append((seb.scan_pose(R_B, p_B, R_BS, p_BS, S_S, S_R, S_B), torch.from_numpy(pts).to(dev)))
    em = seb.ElevationMap(n, n, res, max(len(p) for _, p in scans), z_min=-1.0, z_max=1.0)
    params = seb.SebParams(nx=n, ny=n, n_yaw=K, res=res, length=0.6, width=0.4)
    m = seb.SebMap(params, dev)
    h = torch.empty((n, n), device=dev)
    v = torch.empty((n, n), device=dev)
    filled = torch.empty((n, n), device=dev)
    iw = torch.empty(abi_inpaint_bytes(seb, n), dtype=torch.uint8, device=dev)
    sdf = torch.empty((K, n, n), device=dev)
    sw = torch.empty(seb.abi.seb_sdf_workspace_bytes(n, n, K), dtype=torch.uint8, device=dev)

    def cycle(pose, pts):
        em.integrate(pose, pts)
        em.outputs(h, v)
        seb.inpaint_nearest(h, 0, out=filled, work=iw)
        vw = em.view()
        m.update(filled, (vw.origin_i, vw.origin_j))
        seb.risk_sdf(seb.SE2Grid.from_map(m, 4), 1.0, 2.0, out=sdf, work=sw)

    for pose, pts in scans:  # warm-up: the map fills as the robot moves
        cycle(pose, pts)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        for pose, pts in scans:
            cycle(pose, pts)
    b.record(st)
    b.synchronize()
    ms = a.elapsed_time(b) / (reps * n_scans)
    cells = n * n * K
    return {"ms_per_cycle": ms, "se2_cells_per_s": cells / ms * 1e3, "se2_cells": cells,
            "points_per_scan": int(np.mean([len(p) for _, p in scans])),
            "paper_budget_ms": 50.0, "known_frac_after_update": float(torch.isfinite(h).float().mean()),
            "steps": "elevation update + copy + inpaint + traversability rebuild + SDF",
            "config": "180x180 at 0.1 m, 30 yaws, 0.6x0.4 m footprint, 32x1024-ray synthetic scans"}


def abi_inpaint_bytes(seb, n):
    return seb.abi.seb_inpaint_workspace_bytes(n, n)


def run_e2e(seb, m, world_np, origins, args, dev):
    """Same step through the public API with host buffers, pipelined as an application would run
    it: the step's windows (one pinned host array) are copied host -> device on an upload stream
    into one of two device window sets while the previous step computes; the compute stream
    waits for its set, then runs the rebuild and the shift batch; at the end of the step the
    outputs (5 channels + flags, in window order) are snapshotted with copy_out and read back to
    pinned host memory on a download stream while the next step computes.  The timed region
    covers all steps and ends when the last read-back has landed in host memory."""
    import torch

    n = len(origins)
    host_set = torch.from_numpy(np.stack([world_np[o[1]:o[1] + NY, o[0]:o[0] + NX] for o in origins])).pin_memory()
    dsets = [torch.empty((n, NY, NX), dtype=torch.float32, device=dev) for _ in range(2)]
    stage = torch.empty((5, K, NY, NX), dtype=torch.float32, device=dev)
    stage_fl = torch.empty((K, NY, NX), dtype=torch.uint8, device=dev)
    hout = torch.empty(stage.numel(), dtype=torch.float32).pin_memory()
    hfl = torch.empty(stage_fl.numel(), dtype=torch.uint8).pin_memory()
    comp = torch.cuda.current_stream(dev)
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    set_ready = [torch.cuda.Event() for _ in range(2)]
    set_free = [torch.cuda.Event() for _ in range(2)]
    stage_ready, stage_free = torch.cuda.Event(), torch.cuda.Event()
    h2d = host_set.numel() * 4
    d2h = hout.numel() * 4 + hfl.numel()
    state = {"k": 0}

    def step():
        k = state["k"]
        state["k"] ^= 1
        ws = dsets[k]
        with torch.cuda.stream(up):
            up.wait_event(set_free[k])  # the batch that last read this set is done
            ws.copy_(host_set, non_blocking=True)
            set_ready[k].record(up)
        comp.wait_event(set_ready[k])
        m.update(ws[0], origins[0])
        cells = m.view().last_cells
        m.shift_batch([ws[i] for i in range(1, n)], origins[1:])
        cells += m.view().last_cells
        set_free[k].record(comp)
        comp.wait_event(stage_free)  # the previous read-back has left the staging buffers
        m.outputs(stage, stage_fl)
        stage_ready.record(comp)
        with torch.cuda.stream(down):
            down.wait_event(stage_ready)
            hout.copy_(stage.reshape(-1), non_blocking=True)
            hfl.copy_(stage_fl.reshape(-1), non_blocking=True)
            stage_free.record(down)
        return cells

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    cells = 0
    for _ in range(args.steps):
        cells += step()
    comp.wait_event(stage_free)  # the last read-back is in host memory
    e1.record(comp)
    e1.synchronize()
    total = e0.elapsed_time(e1)
    ws_n = int(os.environ.get("WORLD_SIZE", 1))
    return {"value": cells * ws_n / (total / 1e3), "unit": "SE(2) cells/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": total / args.steps,
            "pipeline": "window uploads and output read-backs on their own streams, overlapped with the updates"}


if __name__ == "__main__":
    main()
