"""Benchmark: the DSMC collision phase (HCAO LB relaxation + QK chemistry).

Headline workload: the CH4 + H -> CH3 + H2 exchange mixture, 16384 cells x
1200 particles (19.7M), 50/50 CH4/H at 4000 K, one stretch coupled to the
reaction coordinate, FP32 velocities with fixed-point energy bookkeeping.
One step = one collision phase over all cells.  `--workload heat_bath` times
the 4096-cell x 500-particle CH4-like heat bath at 15000 K instead.

Prints one JSON line.  `value` = particle-steps/s over the timed steps, device
time from CUDA events on the library's stream around every step.  The
exchange mixture's particle state (630 MB of records) is 5x the L2, so its
steps run back to back without a flush; a state below twice the L2 (the heat
bath, the triatomic) is flushed (a 256 MiB write) before every timed step.
For the headline the same steps with a flush before each are reported
beside it (`l2_flushed`).
`e2e` = the same metric through the C ABI with host buffers: every step loads
the state from pinned host memory, steps, and reads the moments back.
--impl reference times the oracle (CPU) instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_31548_b300 import workloads as W  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
WORKLOADS = {
    "exchange": "ch4_h_exchange_16384x1200_4000K",
    "heat_bath": "ch4_heat_bath_4096x500_15000K_dissociation",
}
KERNEL_SRC = os.path.join(ROOT, "paper_2606_31548_b300", "csrc", "hcao_kernels.cuh")
FUSED_SRC = os.path.join(ROOT, "paper_2606_31548_b300", "csrc", "hcao_fused.cuh")
# DRAM bytes per step of the collide phase (ncu), keyed by (workload, path)
TRAFFIC_FILES = {
    ("exchange", "queue"): os.path.join(ROOT, "profiles", "collide_ch4_h_exchange_traffic.json"),
}

# Algorithmic lane-operations of the relaxation kernel per unit of K5 work (the
# least integer/FP32 lane operations each unit needs):
#   level evaluation (the acceptance weight at the budget): 2 loads, subtract,
#     bucket index (bit cast, shift, subtract, 2 clamps), table offset, compare = 12
#   mode draw: one quarter of a Philox4x32-10 block (10 rounds x 8 ops / 4)
#     + alias slot (multiply, shift, 2 loads, compare, 3 selects) + acceptance
#     on the word's low 8 bits (2 conversions, 2 multiplies, 2 compares) = 34
#   molecule sample: vibrational energy of up to 9 modes twice + setup = 60
#   pair: members, two record loads, relative energy, isotropic direction,
#     scattering, two record stores, event word = 160
OPS_PER_UNIT = (12, 34, 60, 160)
SMS, LANES_PER_SM = 148, 128


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2032.0)), "measured"
    except Exception:
        return 6400.0, 2032.0, "fallback"


def _kernel_hash():
    """First 16 hex digits of the sha256 of the collision kernels' source
    (hcao_kernels.cuh, then hcao_fused.cuh)."""
    import hashlib
    h = hashlib.sha256()
    for p in (KERNEL_SRC, FUSED_SRC):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_per_step(workload: str, path: str):
    """DRAM bytes per step of the collide phase from the committed ncu
    summary, or None if there is none for this workload and path or the
    kernel source changed since it was taken."""
    try:
        with open(TRAFFIC_FILES[(workload, path)]) as f:
            t = json.load(f)
        if t.get("kernel_src_sha256_16") != _kernel_hash():
            return None
        return t
    except Exception:
        return None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def _max_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return x


def _sum_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())
    return x


CELLS_PER_RANK = {"exchange": 16384, "heat_bath": 4096}


def headline_workload(kind: str, rank: int = 0, world: int = 1, **kw):
    """The cells rank `rank` steps: the contiguous range [rank C, (rank + 1) C)
    of one workload of world x C cells (C = 16384 for the exchange mixture,
    4096 for the heat bath), drawn cell by cell so that the split does not
    change the particles, and keyed by the global cell index: each rank steps
    its range exactly as the whole workload would (no data-path collective)."""
    C = kw.pop("cells_per_rank", CELLS_PER_RANK[kind])
    return W.cell_range(kind, rank * C, (rank + 1) * C, world * C, **kw)


def aggregate(units: float, seconds: float):
    """Whole-job figures: units summed over ranks, time the slowest rank's."""
    return _sum_over_ranks(units), _max_over_ranks(seconds)


class Clocks:
    """nvidia-smi sampling (every 50 ms) around the timed region; only samples
    whose timestamps fall inside it are kept."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.dev = device
        self.p = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"hcao_bench_clocks_{os.getpid()}_{device}.csv")
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            deadline = time.time() + 15
            while time.time() < deadline:  # wait for the first sample
                time.sleep(0.05)
                if os.path.getsize(self.path) > 0:
                    break
        except Exception:
            self.p = None
        return self

    def start(self):
        import datetime
        self.t0 = datetime.datetime.now()

    def stop(self):
        import datetime
        self.t1 = datetime.datetime.now()
        time.sleep(0.12)

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        import datetime
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons, n_all = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            n_all += 1
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                mhz, mxx = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            if self.t0 and self.t1 and not (self.t0 <= ts <= self.t1):
                continue
            sm.append(mhz)
            mx = mxx
            for n, v in zip(names, parts[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples_in_timed_region": len(sm), "samples_total": n_all}


def cpu_baseline(kind: str = "exchange", budget_s: float = 12.0, cells: int = 48):
    """The oracle, as it stands, on a bounded sample of the same workload:
    `cells` evenly spaced cells of the headline workload, stepped until
    ~budget_s (cells are independent and keyed by their index, so a sample of
    cells steps exactly as those cells do in the whole workload)."""
    import oracle
    w = headline_workload(kind)
    pick = np.arange(cells) * (w.n_cells // cells)
    sel = np.isin(w.cell, pick)
    o = oracle.Oracle()
    for s in w.species:
        o.add_species(s)
    for r in w.reactions:
        o.add_reaction(r)
    o.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
    o.load(0, w.v[sel], w.qn0()[sel], w.species_idx[sel], w.cell[sel])
    o.init_vibration(0, w.T_vib0)
    psteps = 0
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s and steps < 2000:
        n = o.count(0)
        o.step(1)
        psteps += n
        steps += 1
    dt = time.perf_counter() - t0
    acc = int(o.read_counters(0)[1])
    per_cell = int(np.bincount(w.cell, minlength=w.n_cells).max())
    return {"value": psteps / dt, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "host_cores": os.cpu_count(),
            "collisions_per_s": acc / dt,
            "sample": f"{cells} of the {w.n_cells} cells ({int(sel.sum())} particles, "
                      f"{per_cell} per cell), {steps} steps, single-threaded FP64 C oracle, "
                      f"{dt:.1f} s, on a host with {os.cpu_count()} cores"}


L2_BYTES = 126 * 1024 * 1024


def needs_flush(w, prec) -> bool:
    """Timing rule: between timed steps either L2 is flushed or the state is
    larger than L2.  A state below twice L2 (after the growth of a
    dissociating workload) is flushed before every timed step."""
    rec = 32 if prec == 1 else 64  # FP32 / FP64 record bytes
    return w.n * rec < 2 * L2_BYTES


def l2_note(w, prec) -> str:
    rec = 32 if prec == 1 else 64
    if needs_flush(w, prec):
        return "flushed (256 MiB write) before every timed step"
    return (f"not flushed: the particle state ({w.n * rec / 2**20:.0f} MiB of records) is "
            f"{w.n * rec / L2_BYTES:.1f}x the 126 MB L2; steps run back to back as in a long run")


def run_config(hcao, torch, stream, w, prec, steps: int, warmup: int, flush) -> dict:
    """Device throughput of one more configuration: `warmup` untimed steps,
    then `steps` steps timed one by one with CUDA events (L2 flushed before
    each unless the state is well above L2); particle-steps counted from the
    particles entering each step."""
    do_flush = needs_flush(w, prec)
    ctx = hcao.from_workload(w, precision=prec, stream=stream.cuda_stream)
    for _ in range(warmup):
        ctx.step(1)
    ctx.sync()
    c0 = ctx.read_counters(0)
    comp0 = composition(ctx, w)
    ms, ps = 0.0, 0
    for _ in range(steps):
        ps += ctx.count(0)
        if do_flush:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.step(1)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    c1 = ctx.read_counters(0)
    comp1 = composition(ctx, w)
    ctx.close()
    t = ms / 1e3
    return {"workload": w.name, "particles": int(w.n), "cells": int(w.n_cells), "T0_K": w.T_tr0,
            "reactions": [r.type for r in w.reactions],
            "composition": {"timed_start": comp0, "timed_end": comp1},
            "precision": "fp64" if prec == hcao.FP64 else "fp32", "steps": steps, "warmup": warmup,
            "l2": l2_note(w, prec), "particle_steps_per_s": ps / t, "collisions_per_s": float(c1[1] - c0[1]) / t,
            "reactions_per_s": float(sum(c1[8:]) - sum(c0[8:])) / t, "ms_per_step": 1e3 * t / steps}


def run_batched(hcao, torch, prec, stream, n_res: int, steps: int):
    """Many independent single-cell reservoirs (particle counts log-uniform
    10k-2M, T uniform 5000-30000 K, triatomic or CH4-like): all in one context
    and one CUDA-graph launch per step (launch shapes autotuned during the
    first steps), against the plain per-job loop (one reservoir at a time in
    the same context, one CUDA-graph launch per step).  A job = load + init +
    `steps` collision phases + moments read back; results are identical either
    way (tests/test_gpu_batched.py)."""
    bw = W.batched_reservoirs(n_res=n_res, steps=steps)
    n_total = bw.n
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = hcao.from_batched(bw, precision=prec, stream=stream.cuda_stream)
    g.sync()
    t_load = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    chosen = None
    left = steps
    if steps >= 10:
        chosen = g.autotune(1)  # 7 or 9 live steps (the work-class placement is timed too)
        left = steps - int(g.read_counters(0)[7])
    g.step(left)
    e1.record(stream)
    g.sync()
    for i in range(n_res):
        g.read_moments(i)
    t_b = time.perf_counter() - t0
    dev_b = e0.elapsed_time(e1) / 1e3
    g.close()
    # plain per-job loop
    p = hcao.Context(precision=prec, stream=stream.cuda_stream)
    p.set_species(bw.species)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dev_p = 0.0
    for w in bw.reservoirs:
        rid = p.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
        p.load_particles(rid, w.v, w.qn0(), w.species_idx, w.cell)
        p.init_vibration(rid, w.T_vib0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        p.step(steps)  # one CUDA-graph launch per step
        b.record(stream)
        p.sync()
        dev_p += a.elapsed_time(b) / 1e3
        p.read_moments(rid)
        p.remove_reservoir(rid)
    t_p = time.perf_counter() - t0
    p.close()
    return {"workload": f"{n_res} single-cell reservoirs, {n_total} particles, {steps} steps",
            "batched_jobs_per_s": n_res / t_b, "plain_jobs_per_s": n_res / t_p,
            "jobs_speedup": t_p / t_b,
            "batched_particle_steps_per_s_device": n_total * steps / dev_b,
            "plain_particle_steps_per_s_device": n_total * steps / dev_p,
            "batched_load_s": t_load,
            "autotuned": None if chosen is None else {"select_grid": chosen[0], "relax_grid": chosen[1],
                                                     "queue_by_work_class": bool(chosen[2])},
            "note": "jobs/s include load, init, stepping and the moments read back; the "
                    "device rates time the stepping only"}


def run_served(hcao, prec, stream, n_jobs: int, rate: float, recombination: bool):
    """Serving: Poisson-arriving reservoir jobs (rate 1/s, sizes log-uniform
    10k-4M particles, 200-2000 steps, relaxation / heat-bath / CH4-CH3-H
    equilibrium kinds) submitted to the library's continuous-batching engine
    at their arrival times, against the plain loop: one job at a time, first
    come first served (load, init, step(n) as one CUDA-graph launch per step,
    moments read back).  Latency = completion - arrival."""
    sw = W.served_jobs(n_jobs=n_jobs, rate=rate, recombination=recombination)
    jobs = sw.jobs

    def stats(lat):
        lat = np.sort(np.asarray(lat))
        return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "max_s": float(lat.max())}

    # recombination rounds hold N/3 pairs (a third body per pair): twice the
    # default rounds for the hottest relaxation jobs' (sigma g)_max
    ctx = hcao.Context(precision=prec, stream=stream.cuda_stream, max_rounds=4)
    ctx.set_species(sw.species)
    ctx.set_reactions(sw.reactions)
    ctx.serve_start()
    t0 = time.monotonic()
    ids = []
    for j in jobs:
        d = t0 + j.arrival - time.monotonic()
        if d > 0:
            time.sleep(d)
        ids.append(ctx.serve_submit(j.workload, j.steps))
    res = {}
    while len(res) < len(ids):
        for jid in ids:
            if jid not in res:
                r = ctx.serve_poll(jid)
                if r is not None:
                    res[jid] = r
        time.sleep(0.001)
    _, _, _, iters = ctx.serve_stats()
    timing = ctx.serve_timing()
    ctx.serve_stop()
    ctx.close()
    lat_s = [res[jid].t_done - (t0 + j.arrival) for jid, j in zip(ids, jobs)]
    span_s = max(res[jid].t_done for jid in ids) - t0
    queue_s = [res[jid].t_admit - res[jid].t_submit for jid in ids]

    p = hcao.Context(precision=prec, stream=stream.cuda_stream, max_rounds=4)
    p.set_species(sw.species)
    p.set_reactions(sw.reactions)
    t0 = time.monotonic()
    lat_p = []
    for j in jobs:
        d = t0 + j.arrival - time.monotonic()
        if d > 0:
            time.sleep(d)
        w = j.workload
        rid = p.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
        p.load_particles(rid, w.v, w.qn0(), w.species_idx, w.cell)
        p.init_vibration(rid, w.T_vib0)
        p.step(j.steps)
        p.read_moments(rid)
        p.remove_reservoir(rid)
        lat_p.append(time.monotonic() - (t0 + j.arrival))
    span_p = time.monotonic() - t0
    p.close()
    return {"workload": f"{n_jobs} jobs, Poisson arrivals at {rate:g}/s, "
                        f"{sum(j.workload.n for j in jobs)} particles, {sw.particle_steps:.3e} particle-steps",
            "kinds": {k: sum(1 for j in jobs if j.kind == k) for k in ("relax", "bath", "equil")},
            "recombination": recombination,
            "served_jobs_per_s": n_jobs / span_s, "plain_jobs_per_s": n_jobs / span_p,
            "jobs_speedup": span_p / span_s,
            "served_latency": stats(lat_s), "plain_latency": stats(lat_p),
            "served_queue_wait": stats(queue_s),
            "served_particle_steps_per_s": sw.particle_steps / span_s,
            "plain_particle_steps_per_s": sw.particle_steps / span_p,
            "engine_iterations": int(iters),
            "engine_time_s": timing,
            "engine_note": "engine thread's host time by activity: admit (reservoir set-up and load "
                           "from the job's host copy), step (step launches + synchronisation: the "
                           "device busy with the resident jobs), retire (read-back, release), wait",
            "note": "jobs/s over the span from the first arrival to the last completion; the "
                    "plain loop serves the same arrivals first come first served"}


def _config(kind, w, args, ws):
    per_cell = int(np.bincount(w.cell, minlength=w.n_cells).max())
    return {"workload": WORKLOADS[kind], "cells": w.n_cells * ws, "cells_per_rank": w.n_cells,
            "particles_per_cell": per_cell, "particles": w.n * ws, "T0_K": w.T_tr0, "precision": args.precision,
            "species": [s.name for s in w.species],
            "l2": l2_note(w, 1 if args.precision == "fp32" else 0),
            "parallelism": f"contiguous cell ranges x{ws} (one workload of {ws} x {w.n_cells} cells, "
                           "keyed by global cell index; no data-path collective)"}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    cb = cpu_baseline(args.workload, budget_s=max(3.0, min(20.0, 2.0 * args.steps)))
    w = headline_workload(args.workload)
    cfg = _config(args.workload, w, args, 1)
    cfg["precision"] = "fp64"
    cfg["sample"] = cb["sample"]
    line = {"impl": "reference", "metric": "particle-steps/s", "value": cb["value"],
            "unit": "particle-steps/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line))
    return 0


def composition(ctx, w):
    m = ctx.read_moments(0)
    return {s.name: int(m.n[i]) for i, s in enumerate(w.species)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="exchange", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--batched-res", type=int, default=256, help="reservoirs of the batched run (0: skip)")
    ap.add_argument("--batched-steps", type=int, default=1000)
    ap.add_argument("--served-jobs", type=int, default=48, help="jobs of the served run (0: skip)")
    ap.add_argument("--other-configs", type=int, default=1,
                    help="measure the exchange temperature sweep, the heat bath and the triatomic too")
    ap.add_argument("--served-rate", type=float, default=50.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2606_31548_b300 import hcao

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    prec = hcao.FP32 if args.precision == "fp32" else hcao.FP64
    w = headline_workload(args.workload, rank, ws)
    ctx = hcao.from_workload(w, precision=prec, stream=stream.cuda_stream, device=local)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        ctx.step(1)
    ctx.sync()
    c0 = ctx.read_counters(0)
    comp0 = composition(ctx, w)
    torch.cuda.synchronize()
    _barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    psteps = 0
    do_flush = needs_flush(w, prec)
    with Clocks(local) as clk:
        clk.start()
        t_wall0 = time.perf_counter()
        launches = 0
        for i in range(args.steps):
            n = ctx.count(0)  # particles entering this step (host sync, outside the events)
            psteps += n
            if do_flush:
                flush.zero_()
            l0 = ctx.kernel_launches()
            ev[i][0].record(stream)
            ctx.step(1)
            ev[i][1].record(stream)
            launches += ctx.kernel_launches() - l0  # the step's kernels (not the count's read-out)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        clk.stop()
    _barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ctx.sync()
    c1 = ctx.read_counters(0)
    comp1 = composition(ctx, w)
    ctx.close()
    ctx = None
    # The per-kernel split of the roofline: the same steps of the same
    # workload (a fresh context from the same state, the same warm-up, so the
    # same composition at every step), with CUDA events around every kernel
    # (launched one by one, not as the step's graph); outside the timed region.
    pctx = hcao.from_workload(w, precision=prec, stream=stream.cuda_stream, device=local)
    for _ in range(args.warmup):
        pctx.step(1)
    work0 = pctx.read_work()
    pctx.set_profiling(True)
    psteps_prof = 0
    for i in range(args.steps):
        psteps_prof += pctx.count(0)
        if do_flush:
            flush.zero_()
        pctx.step(1)
    kms, kn = pctx.read_profile()
    pctx.set_profiling(False)
    work_end = pctx.read_work()
    pctx.close()
    # The same steps again, with L2 flushed before each (cold tables at every
    # step start), beside the headline when it runs without flushing.
    l2_flushed = None
    if not do_flush:
        fctx = hcao.from_workload(w, precision=prec, stream=stream.cuda_stream, device=local)
        for _ in range(args.warmup):
            fctx.step(1)
        evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        psf = 0
        for i in range(args.steps):
            psf += fctx.count(0)
            flush.zero_()
            evf[i][0].record(stream)
            fctx.step(1)
            evf[i][1].record(stream)
        torch.cuda.synchronize()
        fctx.close()
        msf = sum(a.elapsed_time(b) for a, b in evf)
        l2_flushed = {"ms_per_step": msf / args.steps, "particle_steps_per_s": psf / (msf / 1e3),
                      "note": "the timed steps again (fresh context, same warm-up), a 256 MiB write "
                              "before each"}
    work = (work_end - work0).astype(np.float64)
    collisions = float(c1[1] - c0[1])
    reactions = float(sum(c1[8:]) - sum(c0[8:]))
    tot_psteps, t = aggregate(float(psteps), ms / 1e3)
    tot_coll = _sum_over_ranks(collisions)
    tot_rx = _sum_over_ranks(reactions)

    # roofline.  HBM view (the algorithmic bytes of the collision phase: one
    # read and one write of each particle's state, 2 S bytes per
    # particle-step, S = 26 B FP32 / 38 B FP64) over the collide-phase kernels'
    # CUDA-event time; the ALU view of the relaxation kernel (counted K5 work x
    # OPS_PER_UNIT lane-operations against 148 SMs x 128 lanes x the maximum
    # SM clock) beside it.
    names = hcao.Context.PROFILE_KERNELS
    per_step = {k: kms[i] / args.steps for i, k in enumerate(names)}
    hbm_peak, sm_mhz_max, peak_kind = _peaks()
    relax_s = kms[2] / 1e3
    lane_ops = float(np.dot(work, OPS_PER_UNIT))
    alu_peak = SMS * LANES_PER_SM * sm_mhz_max * 1e6 / 1e9  # Glane-op/s
    alu_ach = lane_ops / relax_s / 1e9 if relax_s > 0 and lane_ops > 0 else None
    S = 26.0 if prec == hcao.FP32 else 38.0
    fused = int(kn[5]) > 0
    collide_s = (kms[1] + kms[2] + kms[3] + kms[5]) / 1e3
    step_s = float(np.sum(kms)) / 1e3
    if fused:  # the relaxation runs inside the fused kernel
        relax_s = kms[5] / 1e3
        alu_ach = lane_ops / relax_s / 1e9 if relax_s > 0 and lane_ops > 0 else None
    hbm_ach = (2 * S * psteps_prof) / collide_s / 1e9 if collide_s > 0 else None
    tr = _traffic_per_step(args.workload, "fused" if fused else "queue")
    roof = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
            "frac": (hbm_ach / hbm_peak) if hbm_ach else None,
            "traffic": tr["dram_bytes_per_step"] if tr else None,
            "traffic_unit": "DRAM bytes per step of the collide phase (ncu, cold cache), beside "
                            f"{2 * S * psteps / args.steps:.4g} algorithmic bytes per step",
            "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
            "kernel": "k_collide_fused (the whole collision phase, one launch per step)" if fused
                      else "collide phase (select + work-class placement + relax + react kernels)",
            "path": "fused" if fused else "queue",
            "bytes_per_particle_step": 2 * S,
            "step_view": {"achieved_GBps": (2 * S * psteps) / (ms / 1e3) / 1e9 if ms > 0 else None,
                          "frac": (2 * S * psteps) / (ms / 1e3) / 1e9 / hbm_peak if ms > 0 else None,
                          "time": "the timed steps (one CUDA graph per step, all kernels)"},
            "profiled_steps": {"steps": args.steps, "ms_per_step": step_s * 1e3 / args.steps,
                               "note": "kernel_ms_per_step, achieved and alu_view come from these steps, "
                                       "run after the timed ones with events around every kernel"},
            "kernel_ms_per_step": per_step,
            "kernel_launches": {k: int(kn[i]) for i, k in enumerate(names)},
            "alu_view": {"kernel": ("k_collide_fused" if fused else "k_relax_fast") if prec == hcao.FP32
                         else "k_relax",
                         "achieved_Glane_op_s": alu_ach, "peak_Glane_op_s": alu_peak,
                         "frac": (alu_ach / alu_peak) if alu_ach else None,
                         "peak_kind": f"derived: {SMS} SMs x {LANES_PER_SM} lanes x {sm_mhz_max:.0f} MHz",
                         "work_per_step": {"level_evals": work[0] / args.steps,
                                           "mode_draws": work[1] / args.steps,
                                           "samples": work[2] / args.steps, "pairs": work[3] / args.steps},
                         "ops_per_unit": list(OPS_PER_UNIT)}}

    # e2e through the C ABI with host buffers (pinned): load + step + moments
    e2e = None
    if args.e2e_steps > 0:
        vdt = np.float32 if prec == hcao.FP32 else np.float64
        v_h = torch.from_numpy(np.ascontiguousarray(w.v, dtype=vdt)).pin_memory()
        q_h = torch.from_numpy(w.qn0()).pin_memory()
        s_h = torch.from_numpy(w.species_idx).pin_memory()
        c_h = torch.from_numpy(w.cell).pin_memory()
        ectx = hcao.Context(precision=prec, stream=stream.cuda_stream, device=local)
        ectx.set_species(w.species)
        ectx.set_reactions(w.reactions)
        rid = ectx.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
        L = ectx.L
        import ctypes as C
        load = L.hcao_load_particles_f32 if prec == hcao.FP32 else L.hcao_load_particles
        mom = hcao.Moments()

        def one():
            ectx._chk(load(ectx.h, rid, w.n, C.c_void_p(v_h.data_ptr()), C.c_void_p(q_h.data_ptr()),
                           C.c_void_p(s_h.data_ptr()), C.c_void_p(c_h.data_ptr())))
            ectx._chk(L.hcao_step(ectx.h, 1))
            ectx._chk(L.hcao_read_moments(ectx.h, rid, C.byref(mom)))

        one()
        torch.cuda.synchronize()
        _barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            one()
        torch.cuda.synchronize()
        te = _max_over_ranks(time.perf_counter() - t0)
        # where an e2e step goes: each call timed alone (host clock, synchronised),
        # after the timed loop and outside it
        split = {}
        for name, f in (("load", lambda: ectx._chk(load(
                            ectx.h, rid, w.n, C.c_void_p(v_h.data_ptr()), C.c_void_p(q_h.data_ptr()),
                            C.c_void_p(s_h.data_ptr()), C.c_void_p(c_h.data_ptr())))),
                        ("step", lambda: ectx._chk(L.hcao_step(ectx.h, 1))),
                        ("moments", lambda: ectx._chk(L.hcao_read_moments(ectx.h, rid, C.byref(mom))))):
            ts = []
            for _ in range(3):
                ectx.sync()
                t1 = time.perf_counter()
                f()
                ectx.sync()
                ts.append(time.perf_counter() - t1)
            split[name] = 1e3 * sorted(ts)[1]
        e2e = {"value": _sum_over_ranks(float(w.n * args.e2e_steps)) / te, "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(w.n * (3 * v_h.element_size() + 16 + 4 + 4)),
               "d2h_bytes_per_step": int(C.sizeof(hcao.Moments)),
               "split_ms": split,
               "note": "per step: hcao_load_particles (FP32 velocities through hcao_load_particles_f32 "
                       "in FP32 mode) from pinned host memory (state of the "
                       "workload), hcao_step(1), hcao_read_moments; split_ms: the median of 3 "
                       "separate synchronised calls of each, measured after the timed loop"}
        ectx.close()
        del v_h, q_h, s_h, c_h

    others = None
    if args.other_configs and ws == 1:
        others = {}
        if args.workload != "exchange":
            others["ch4_h_exchange_16384x1200_4000K_fp32"] = run_config(
                hcao, torch, stream, W.ch4_h_exchange(T0=4000.0), hcao.FP32, 10, 3, flush)
        for T in (2000.0, 3000.0, 5000.0, 6000.0):
            others[f"ch4_h_exchange_16384x1200_{T:.0f}K_fp32"] = run_config(
                hcao, torch, stream, W.ch4_h_exchange(T0=T), hcao.FP32, 10, 3, flush)
        if args.workload != "heat_bath":
            others["ch4_heat_bath_4096x500_15000K_fp32"] = run_config(
                hcao, torch, stream, W.ch4_heat_bath(), hcao.FP32, 20, 5, flush)
        others["ch4_heat_bath_4096x500_15000K_no_dissociation_fp32"] = run_config(
            hcao, torch, stream, W.ch4_heat_bath(dissociation=False), hcao.FP32, 20, 5, flush)
        # the heat bath in the FP64 parity mode too (its configuration names both)
        others["ch4_heat_bath_4096x500_15000K_fp64"] = run_config(
            hcao, torch, stream, W.ch4_heat_bath(), hcao.FP64, 10, 3, flush)
        others["triatomic_relaxation_20000x1_fp64"] = run_config(
            hcao, torch, stream, W.relaxation_triatomic(), hcao.FP64, 50, 5, flush)
    batched = None
    if args.batched_res > 0 and ws == 1:
        if ctx is not None:
            ctx.close()
            ctx = None
        batched = run_batched(hcao, torch, prec, stream, args.batched_res, args.batched_steps)
    served = None
    if args.served_jobs > 0 and ws == 1:
        served = run_served(hcao, prec, stream, args.served_jobs, args.served_rate, recombination=True)
    cb = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(args.workload)
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": "particle-steps/s", "value": tot_psteps / t, "unit": "particle-steps/s",
            "collisions_per_s": tot_coll / t, "reactions_per_s": tot_rx / t,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == hcao.FP32 else "f64",
            "data": "synthetic",
            "config": _config(args.workload, w, args, ws),
            "composition": {"timed_start": comp0, "timed_end": comp1},
            "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": int(launches),
            "l2_flushed": l2_flushed,
            "clocks": clocks, "wall_s_timed_loop": t_wall, "batched": batched, "served": served,
            "other_configs": others,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if ctx is not None:
        ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
