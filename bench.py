#!/usr/bin/env python3
"""Benchmark of the SMC-X swap sweep on GB300 (one JSON line on rank 0).

Workload (default): BCC 812^3 conventional cells x 2 = 1,070,774,656 sites,
5 species equiatomic, EPI shells 1-3 drawn from N(0, 0.02 eV) (seed 0,
quantised to 2^-32 eV), linear anneal 1200 -> 600 K over 10^4 sweeps, Philox
seed 0, one byte per site.  One step = one MC sweep (the eight checkerboard
colour phases, one trial per site) at that sweep's anneal temperature plus
one Warren-Cowley SRO / energy pair-count reduction, with the pair counts
read back to the host.  Inputs (1.07 GB of occupancy) exceed the 129 MB L2,
so no flush is needed between steps.

Metric: attempted swaps per second (sites x sweeps / device time of the
timed steps, max over ranks).  Multi-GPU: one independent lattice replica
per rank (the sweep of one lattice has no exchange step), value = sum.

--impl reference times the sequential CPU oracle (oracle/) on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2509_20949_gb300 import inputs  # noqa: E402

METRIC = ("attempted MC swaps/sec on 1 GB300 (plain single-lattice sweep; batched and served "
          "forms in the line's batched/served/served_saturated objects)")
UNIT = "swaps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bcc812_k5")
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 generic, 2 tiled")
    ap.add_argument("--tile", type=int, default=-1,
                    help="tile shape of the tiled kernel (-1: the online choice)")
    ap.add_argument("--staging", type=int, default=0,
                    help="tiled kernel staging: 0 bulk (TMA) copies where they fit, 1 cp.async only")
    ap.add_argument("--pack-bits", type=int, default=8)
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--mode", default="plain", choices=["plain", "batch", "serve", "slab", "local", "analysis", "exchange"],
                    help="plain: the single-lattice sweep (default); batch: 256 independent "
                         "lattices batched vs one at a time; serve: Poisson-arrival serving; "
                         "slab: one lattice decomposed along z over the ranks; local: the "
                         "local-energy (nonlinear short-range) model")
    ap.add_argument("--jobs", type=int, default=256)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--rate", type=float, default=5.0)
    ap.add_argument("--window", type=float, default=10.0)
    ap.add_argument("--budget-gb", type=float, default=160.0)
    ap.add_argument("--no-batched", action="store_true",
                    help="plain mode: leave out the batched (256-job) measurement")
    ap.add_argument("--no-served", action="store_true",
                    help="plain mode: leave out the served (Poisson trace) measurement")
    ap.add_argument("--served-rate", type=float, default=1.0)
    ap.add_argument("--served-window", type=float, default=10.0)
    ap.add_argument("--saturated-rate", type=float, default=5.0,
                    help="plain mode: arrival rate of the second, saturating served trace (0 = none)")
    ap.add_argument("--saturated-window", type=float, default=4.0)
    return ap.parse_args()


def workload_config(name):
    w = inputs.workload(name)
    kind = "BCC" if w["kind"] == 0 else "FCC"
    n = w["n"]
    N = inputs.n_sites(w["kind"], n)
    desc = (f"{name}: {kind} {n[0]}x{n[1]}x{n[2]} conventional cells = {N} sites, K={w['K']}, "
            f"EPI shells 1-{w['M']} ~N(0,{w['sigma']} eV) seed {w['epi_seed']}, "
            f"T {w['T_first']:g}->{w['T_last']:g} K over {w['sweeps']} sweeps, Philox seed {w['seed']}")
    return w, N, desc


def sweep_temperature(w, i):
    n = w["sweeps"]
    if n <= 1 or w["T_first"] == w["T_last"]:
        return w["T_first"]
    return w["T_first"] + (w["T_last"] - w["T_first"]) * (i % n) / (n - 1)


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"smcx_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def max_over_ranks(value: float) -> float:
    """Maximum of a per-rank float over all ranks (identity without a process
    group); NCCL reduces on the device, gloo on the host."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank simulates an independent replica of the lattice."""
    return int(base_seed) + int(rank)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_cpu():
    """Host CPU of this machine: logical CPUs and model name (lscpu)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def _oracle_rate(oracle, d, V, scratch, T, cids, seconds, threads):
    """Trials/s of the oracle replaying the listed cells of colour 0 of sweep
    0 in place, on `threads` threads, over about `seconds` of work."""
    n_cal = min(len(cids), 256 * max(1, threads))
    t0 = time.perf_counter()
    oracle.phase_cells_par(d, V, scratch, 0, T, 0, cids[:n_cal], n_threads=threads, inplace=True)
    per_cell = max((time.perf_counter() - t0) / n_cal, 1e-8)
    n = int(min(len(cids) - n_cal, max(64, seconds / per_cell)))
    sel = cids[n_cal:n_cal + n]
    t0 = time.perf_counter()
    _, st = oracle.phase_cells_par(d, V, scratch, 0, T, 0, sel, n_threads=threads, inplace=True)
    dt = time.perf_counter() - t0
    return int(st["attempts"]) / dt, len(sel), int(st["attempts"]), dt


def cpu_baseline(w, N, V, occ, seconds, rank):
    """The oracle as it stands on the host: its OpenMP variant (the cells of
    one colour shared out over every host core; same results as the
    sequential oracle) replaying a bounded sample of link cells of colour 0
    of sweep 0 on the full lattice, and the sequential rate on one core."""
    import oracle

    d = oracle.Desc(w["kind"], w["n"], w["K"], w["M"], seed=w["seed"])
    cids = _colour_cells(oracle, d, 0)
    scratch = np.array(occ, copy=True)
    T = sweep_temperature(w, 0)
    threads = oracle.max_threads()
    half = len(cids) // 2
    v1, n1, a1, t1 = _oracle_rate(oracle, d, V, scratch, T, cids[:half], seconds / 3, 1)
    vp, n_p, ap, tp = _oracle_rate(oracle, d, V, scratch, T, cids[half:], seconds * 2 / 3, threads)
    return {"value": vp, "unit": UNIT, "cores": threads, "kind": "oracle",
            "single_core_value": v1, "host": host_cpu(),
            "sample": f"{n_p} link cells ({ap} trials) of colour 0, sweep 0 of the full lattice, "
                      f"{tp:.1f} s on {threads} threads (cells of one colour in parallel); "
                      f"one core: {n1} cells, {a1} trials, {t1:.1f} s"}


def _colour_cells(oracle, d, colour):
    L, m = oracle.layout(d)
    cx = np.arange(m[0])
    cy = np.arange(m[1])
    cz = np.arange(m[2])
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    col = (X & 1) | ((Y & 1) << 1) | ((Z & 1) << 2)
    cid = (Z * m[1] + Y) * m[0] + X
    return cid[col == colour].astype(np.uint32).ravel()


def run_reference(args):
    world, rank, local = dist_setup()
    if world > 1 and rank != 0:
        return 0
    w, N, desc = workload_config(args.workload)
    V = inputs.epi_table(w["M"], w["K"], w["sigma"], w["epi_seed"])
    occ = inputs.initial_occupancy(w["kind"], w["n"], w["K"], w["occ_seed"], w["fractions"])
    import oracle

    oracle.build()
    d = oracle.Desc(w["kind"], w["n"], w["K"], w["M"], seed=w["seed"])
    cids = _colour_cells(oracle, d, 0)
    threads = oracle.max_threads()
    per_step = min(len(cids), max(64, min(32768 * threads,
                                          len(cids) // max(1, args.steps + args.warmup))))
    scratch = np.array(occ, copy=True)
    pos = 0
    times, atts = [], []
    for s in range(args.warmup + args.steps):
        if pos + per_step > len(cids):  # small lattices: go round the colour's cells again
            pos = 0
        sel = cids[pos:pos + per_step]
        pos += per_step
        t0 = time.perf_counter()
        _, st = oracle.phase_cells_par(d, V, scratch, 0, sweep_temperature(w, 0), 0, sel,
                                       n_threads=threads, inplace=True)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            atts.append(int(st["attempts"]))
    value = sum(atts) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": desc, "sample_per_step": f"{per_step} link cells of colour 0"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "host": host_cpu(),
                             "sample": f"{per_step} link cells per step of colour 0, sweep 0, "
                                       f"full lattice in host memory, {threads} threads "
                                       "(cells of one colour in parallel)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _job_arrays(j):
    V = inputs.epi_table(j["M"], j["K"], j["sigma"], j["epi_seed"])
    occ = inputs.initial_occupancy(j["kind"], j["n"], j["K"], j["occ_seed"], j["fractions"])
    return V, occ


def cpu_baseline_local(w, M, seconds):
    """The oracle's local-energy sweeps, single-threaded on the host, on a
    bounded lattice of the workload's kind, composition and table recipe
    (a full sweep of the benchmark lattice would take hours)."""
    import oracle

    n = 12
    while True:
        d = oracle.Desc(w["kind"], (n, n, n), w["K"], M, seed=w["seed"])
        T = inputs.local_energy_table(w["kind"], M, w["K"], w["sigma"], w["epi_seed"])
        occ = inputs.initial_occupancy(w["kind"], (n, n, n), w["K"], w["occ_seed"], w["fractions"])
        t0 = time.perf_counter()
        _, st = oracle.local_sweeps(d, T, occ, 0, 1, sweep_temperature(w, 0))
        dt = time.perf_counter() - t0
        if dt > seconds / 4 or n >= 48:
            break
        n = int(n * 1.5)
    att = int(st["attempts"].sum())
    return {"value": att / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 sweep of a {n}^3 lattice of the same kind, species, composition "
                      f"and table recipe, {dt:.1f} s single-threaded"}


def run_local(args):
    """The local-energy model (the nonlinear short-range model of Sec. 3): the
    workload's lattice and composition with a synthetic table (pairwise part
    plus a term quadratic in each shell count, shells 1-3); every trial
    recomputes the local energies of its interaction zone.  value = sites x
    sweeps / CUDA-event time of the timed sweeps."""
    import torch

    torch.cuda.set_device(0)
    from paper_2509_20949_gb300.lattice import Lattice

    w, N, desc = workload_config(args.workload)
    M = min(w["M"], 3)
    T = inputs.local_energy_table(w["kind"], M, w["K"], w["sigma"], w["epi_seed"])
    occ = inputs.initial_occupancy(w["kind"], w["n"], w["K"], w["occ_seed"], w["fractions"])
    stream = torch.cuda.current_stream()
    lat = Lattice(w["kind"], w["n"], w["K"], occ, seed=w["seed"], pack_bits=args.pack_bits,
                  stream=stream)
    lat.set_local_model(T)
    for i in range(args.warmup):
        lat.sweep(1, sweep_temperature(w, i), stats=False)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for s in range(args.steps):
        lat.sweep(1, sweep_temperature(w, args.warmup + s), stats=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_ms = ev0.elapsed_time(ev1)
    ts = lat.sweep(1, sweep_temperature(w, args.warmup + args.steps))
    L, m = lat.layout()
    peak, peak_src = measured_peaks()
    phase_ms = t_ms / (args.steps * 8)
    achieved = 2.0 * N / 8 / (phase_ms / 1e3) / 1e9  # 2 B per trial, as the EPI sweep
    cpu = None if args.no_cpu_baseline else cpu_baseline_local(w, M, args.cpu_seconds)
    line = {"metric": "attempted MC swaps/sec on 1 GB300 (local-energy model)",
            "value": N * args.steps / (t_ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "mode": "local",
            "config": {"workload": desc, "model": f"local energies of shells 1-{M}: "
                       "T = c V/2 + U c^2/z per (shell, centre, neighbour species)",
                       "link_cell_edge": L, "cells": m, "step": "1 sweep (8 colour phases)",
                       "pack_bits": args.pack_bits},
            "trial_stats": {"unlike_frac": ts["unlike"] / ts["attempts"],
                            "accepted_frac": ts["accepted"] / ts["attempts"]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "local sweep phase",
                         "kernel_ms_per_launch": phase_ms, "peak_source": peak_src,
                         "limiter": {"unit": "L1/L2 load latency",
                                     "source": "profiles/sweep_local_bcc448_k5.md"}},
            "cpu_baseline": cpu,
            "clocks": clk, "gpu_launches": args.steps * 8}
    print(json.dumps(line), flush=True)
    return 0


def run_slab(args):
    """One lattice swept by all ranks through the z decomposition (strong
    scaling): every rank holds the same lattice, sweeps its share of the link
    cell planes and trades boundary planes (NCCL device buffers under
    torchrun).  value = sites x sweeps / max-over-ranks wall time of the
    timed sweeps (the boundary exchanges are part of each sweep)."""
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2509_20949_gb300.lattice import Lattice
    from paper_2509_20949_gb300.slab import SlabSweep

    w, N, desc = workload_config(args.workload)
    V = inputs.epi_table(w["M"], w["K"], w["sigma"], w["epi_seed"])
    occ = inputs.initial_occupancy(w["kind"], w["n"], w["K"], w["occ_seed"], w["fractions"])
    lat = Lattice(w["kind"], w["n"], w["K"], occ, seed=w["seed"], pack_bits=args.pack_bits)
    if args.kernel:
        lat.set_option(1, args.kernel)
    lat.set_epi(V)
    s = SlabSweep(lat)
    for i in range(args.warmup):
        s.sweep(1, sweep_temperature(w, i))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    tot = 0
    for i in range(args.steps):
        tot += s.sweep(1, sweep_temperature(w, args.warmup + i))["attempts"]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    dt = max_over_ranks(dt)
    p = s.plan(lat.sweep_counter)
    if rank == 0:
        line = {"metric": "attempted MC swaps/sec (one lattice decomposed along z over the GPUs)",
                "value": tot / dt, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "int64", "data": "synthetic", "mode": "slab",
                "config": {"workload": desc, "step": "1 sweep: 2 half sweeps of 4 colour phases on "
                           "this rank's link-cell planes, boundary-plane merges, window moves",
                           "comm": "nccl device buffers" if s.device_comm else "none (one rank)",
                           "planes_per_rank": p["n_own"], "halo": p["halo"],
                           "pack_bits": args.pack_bits},
                "attempts_total": tot, "clocks": clk,
                # 8 colour phases per sweep; with several ranks also the merge
                # kernels (one per row group and run of each boundary region)
                "gpu_launches": args.steps * 8 if world == 1 else None}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def measure_batched(n_jobs=256, chunk=50, sample_stride=8):
    """C4, the 256-job mix (n ~ log-U(8, 64) conventional cells, BCC/FCC,
    K ~ U{3..6}, shells 1-3, T ~ U(300, 1500) K, 200 sweeps each): all jobs
    batched (graph-captured chunks of sweeps over every job) against the same
    jobs one at a time through smcx_sweep, on a 1-in-`sample_stride` sample
    of the jobs (each job's sweeps timed alone, lattices already on the
    device).  Every sampled job ends in the same bits both ways."""
    import torch

    from paper_2509_20949_gb300.batch import Batch
    from paper_2509_20949_gb300.lattice import Lattice

    jobs = inputs.batch_jobs(n_jobs)
    arrays = [_job_arrays(j) for j in jobs]
    attempts = sum(inputs.n_sites(j["kind"], j["n"]) * j["sweeps"] for j in jobs)
    heap = sum(Batch.job_bytes(j["kind"], j["n"], j["K"]) for j in jobs)
    transfer = max(inputs.n_sites(j["kind"], j["n"]) for j in jobs)
    b = Batch(len(jobs), Batch.control_bytes(len(jobs), transfer) + heap + (1 << 20), transfer)
    ids = [b.add(j["kind"], j["n"], j["K"], occ, V, j["T_first"], j["sweeps"], seed=j["seed"])
           for j, (V, occ) in zip(jobs, arrays)]
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t0 = time.perf_counter()
    done = 0
    while done < len(ids):
        b.run(chunk)
        done += len(b.poll())
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    clk = clocks.stop()
    pick = list(range(0, len(jobs), sample_stride))
    t_single, att_single, same = 0.0, 0, True
    for k in pick:
        j, (V, occ) = jobs[k], arrays[k]
        lat = Lattice(j["kind"], j["n"], j["K"], occ, seed=j["seed"])
        lat.set_epi(V)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.sweep(j["sweeps"], j["T_first"], stats=False)
        torch.cuda.synchronize()
        t_single += time.perf_counter() - t0
        att_single += inputs.n_sites(j["kind"], j["n"]) * j["sweeps"]
        r = b.result(ids[k])
        same = same and np.array_equal(r["occ"], lat.occupancy()) and \
            r["energy"] == lat.running_energy() == lat.energy()
        lat.close()
    b.close()
    one = att_single / t_single
    return {"value": attempts / t_batch, "unit": UNIT, "one_at_a_time": one,
            "speedup": (attempts / t_batch) / one, "identical_results": bool(same),
            "jobs": len(jobs), "trials": attempts, "seconds": t_batch,
            "one_at_a_time_sample": f"{len(pick)} of {len(jobs)} jobs (every {sample_stride}th), "
                                    f"{att_single} trials in {t_single:.2f} s",
            "config": f"{len(jobs)} jobs, {sum(inputs.n_sites(j['kind'], j['n']) for j in jobs)} "
                      f"sites, 200 sweeps each, chunk {chunk} sweeps", "clocks": clk}


def fifo_one_at_a_time(trace, deadline_s, chunk=50):
    """Baseline of the served trace: one job at a time in arrival order
    (FIFO), each uploaded as its own lattice when it starts and swept
    through smcx_sweep in chunks of `chunk` sweeps (so the deadline can stop
    it); latency = arrival -> result on the host."""
    import torch

    from paper_2509_20949_gb300.lattice import Lattice

    t0 = time.perf_counter()
    lat_s, swaps, results = [], 0, {}
    for j in sorted(trace, key=lambda j: j["arrival_s"]):
        while time.perf_counter() - t0 < j["arrival_s"]:
            time.sleep(min(0.01, j["arrival_s"] - (time.perf_counter() - t0)))
        if time.perf_counter() - t0 > deadline_s:
            break
        lat = Lattice(j["kind"], j["n"], j["K"], j["occ"], seed=j["seed"])
        lat.set_epi(j["V"])
        sites = inputs.n_sites(j["kind"], j["n"])
        done = 0
        while done < j["sweeps"] and time.perf_counter() - t0 <= deadline_s:
            k = min(chunk, j["sweeps"] - done)
            lat.sweep(k, j["T"], stats=False)
            torch.cuda.synchronize()
            done += k
            swaps += sites * k
        if done == j["sweeps"]:
            results[j["job"]] = lat.occupancy()
            lat_s.append(time.perf_counter() - t0 - j["arrival_s"])
        lat.close()
    elapsed = time.perf_counter() - t0
    lat_a = np.array(lat_s)
    return {"swaps_per_s": swaps / elapsed, "completed": len(lat_s),
            "p50_latency_s": float(np.percentile(lat_a, 50)) if len(lat_a) else None,
            "p99_latency_s": float(np.percentile(lat_a, 99)) if len(lat_a) else None,
            "elapsed_s": elapsed}, results


def measure_served(rate=1.0, window=10.0, budget_gb=160.0, chunk=50, deadline=None, seed=11):
    """C5 at one arrival rate: Poisson arrivals over `window` s of lattices
    with 1e4-1e8 sites and 100-5000 sweeps (log-uniform), composition or
    temperature scans, admitted by the HBM budget into the continuous-
    batching server (state resident between chunks); then the same trace
    FIFO one job at a time.  p50/p99 latency of the completed jobs,
    aggregate swaps/s of all swaps run, and whether every job completed both
    ways ended in the same bits."""
    import torch

    from paper_2509_20949_gb300.server import Server

    deadline = 3.0 * window if deadline is None else deadline
    trace = inputs.served_jobs(rate, window, seed=seed)
    for j in trace:
        j["V"], j["occ"] = _job_arrays(j)
    offered = sum(inputs.n_sites(j["kind"], j["n"]) * j["sweeps"] for j in trace)
    srv = Server(int(budget_gb * (1 << 30)), max_jobs=1024, chunk_sweeps=chunk,
                 transfer_bytes=(1 << 27))
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    m = srv.run_trace(trace, deadline_s=deadline)
    clk = clocks.stop()
    served_occ = {srv.done[t]["job"]: srv.done[t]["occ"] for t in srv.done
                  if "job" in srv.done[t]}
    srv.close()
    del srv
    torch.cuda.empty_cache()
    fifo, fifo_occ = fifo_one_at_a_time(trace, deadline, chunk)
    both = [k for k in fifo_occ if k in served_occ]
    same = all(np.array_equal(served_occ[k], fifo_occ[k]) for k in both)
    return {"value": m["swaps_per_s"], "unit": UNIT,
            "p50_latency_s": m["p50_latency_s"], "p99_latency_s": m["p99_latency_s"],
            "completed": m["completed"], "submitted": m["submitted"],
            "finished_jobs_swaps_per_s": m["finished_swaps_per_s"],
            "offered_trials": offered, "elapsed_s": m["elapsed_s"],
            "fifo_one_at_a_time": fifo,
            "identical_results": {"jobs_compared": len(both), "same": bool(same)},
            "config": f"Poisson {rate}/s over {window} s ({len(trace)} jobs), sites "
                      f"log-U(1e4,1e8), sweeps log-U(100,5000), budget {budget_gb} GB, chunk "
                      f"{chunk} sweeps, deadline {deadline} s", "clocks": clk}


def run_batch(args):
    """256 independent lattices (n ~ log-U(8, 64) conventional cells, BCC/FCC,
    K ~ U{3..6}, shells 1-3, T ~ U(300, 1500) K, 200 sweeps each): batched
    (one graph-captured chunk of sweeps for all jobs) vs one job at a time
    through smcx_sweep.  Both with the lattices already on the device."""
    import torch

    from paper_2509_20949_gb300.batch import Batch
    from paper_2509_20949_gb300.lattice import Lattice

    torch.cuda.set_device(0)
    jobs = inputs.batch_jobs(args.jobs)
    arrays = [_job_arrays(j) for j in jobs]
    total_sites = sum(inputs.n_sites(j["kind"], j["n"]) for j in jobs)
    attempts = sum(inputs.n_sites(j["kind"], j["n"]) * j["sweeps"] for j in jobs)
    heap = sum(Batch.job_bytes(j["kind"], j["n"], j["K"]) for j in jobs)
    transfer = max(inputs.n_sites(j["kind"], j["n"]) for j in jobs)
    b = Batch(len(jobs), Batch.control_bytes(len(jobs), transfer) + heap + (1 << 20), transfer)
    ids = [b.add(j["kind"], j["n"], j["K"], occ, V, j["T_first"], j["sweeps"], seed=j["seed"])
           for j, (V, occ) in zip(jobs, arrays)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    while done < len(ids):
        b.run(args.chunk)
        done += len(b.poll())
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    # one job at a time (device-resident lattices, each job's sweeps timed)
    lats = []
    for j, (V, occ) in zip(jobs, arrays):
        lat = Lattice(j["kind"], j["n"], j["K"], occ, seed=j["seed"])
        lat.set_epi(V)
        lats.append(lat)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j, lat in zip(jobs, lats):
        lat.sweep(j["sweeps"], j["T_first"], stats=False)
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    same = all(np.array_equal(b.result(i)["occ"], lat.occupancy())
               for i, lat in list(zip(ids, lats))[:: max(1, len(ids) // 16)])
    line = {"metric": "attempted MC swaps/sec on 1 GB300 (batched, 256 independent lattices)",
            "value": attempts / t_batch, "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "one_at_a_time": attempts / t_single, "speedup": t_single / t_batch,
            "identical_results_sampled": bool(same),
            "config": {"workload": f"{len(jobs)} jobs, {total_sites} sites, {attempts} trials, "
                                   f"chunk {args.chunk} sweeps", "dtype": "int64"}}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Poisson arrivals (rate per s, window s) of lattices with 1e4-1e8 sites
    and 100-5000 sweeps (log-uniform), composition or temperature scans,
    admitted by an HBM budget, continuous batching; p50/p99 latency of the
    completed jobs and aggregate swaps/s."""
    import torch

    from paper_2509_20949_gb300.server import Server

    torch.cuda.set_device(0)
    trace = inputs.served_jobs(args.rate, args.window, seed=11)
    for j in trace:
        j["V"], j["occ"] = _job_arrays(j)
    budget = int(args.budget_gb * (1 << 30))
    srv = Server(budget, max_jobs=1024, chunk_sweeps=args.chunk, transfer_bytes=(1 << 27))
    m = srv.run_trace(trace, deadline_s=args.window * 3)
    line = {"metric": "attempted MC swaps/sec on 1 GB300 (served, continuous batching)",
            "value": m["swaps_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "finished_jobs_swaps_per_s": m["finished_swaps_per_s"],
            "p50_latency_s": m["p50_latency_s"], "p99_latency_s": m["p99_latency_s"],
            "completed": m["completed"], "submitted": m["submitted"],
            "completed_fraction": m["completed_fraction"], "elapsed_s": m["elapsed_s"],
            "config": {"workload": f"Poisson {args.rate}/s over {args.window} s, sites log-U(1e4,1e8), "
                                   f"sweeps log-U(100,5000), budget {args.budget_gb} GB, "
                                   f"chunk {args.chunk}", "dtype": "int64"}}
    print(json.dumps(line), flush=True)
    return 0


def run_analysis(args):
    """The analyses of Sec. 3.2 on the workload lattice after its warm-up
    sweeps: the composition profile along a cylinder (one pass over the
    lattice: 1 B/site of algorithmic traffic, against the HBM roofline) and
    the first-shell clusters of the last species (union-find over all
    sites).  Each timed `steps` times after `warmup` untimed calls; median."""
    import torch

    torch.cuda.set_device(0)
    from paper_2509_20949_gb300.lattice import Lattice

    w, N, desc = workload_config(args.workload)
    V = inputs.epi_table(w["M"], w["K"], w["sigma"], w["epi_seed"])
    occ = inputs.initial_occupancy(w["kind"], w["n"], w["K"], w["occ_seed"], w["fractions"])
    lat = Lattice(w["kind"], w["n"], w["K"], occ, seed=w["seed"])
    lat.set_epi(V)
    lat.sweep(2, w["T_first"], stats=False)
    n = w["n"]
    origin = (n[0], n[1], 0)                      # the lattice's centre line (half units)
    radius2 = (n[0] // 2) ** 2                    # a cylinder of radius n_x / 4 cells
    length, n_bins = 2 * n[2], 64

    def timed(f, k):
        ts = []
        for _ in range(k):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = f()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts)), r

    for _ in range(args.warmup):
        lat.composition_profile(2, origin, radius2, length, n_bins)
    clocks = ClockSampler(0)
    clocks.start()
    t_prof, prof = timed(lambda: lat.composition_profile(2, origin, radius2, length, n_bins),
                         max(args.steps, 3))
    species = [w["K"] - 1]
    lat.clusters(species, cap=64)
    t_cl, sizes = timed(lambda: lat.clusters(species, cap=64), 3)
    clk = clocks.stop()
    peak, peak_src = measured_peaks()
    gbs = N / t_prof / 1e9
    line = {"metric": "composition-profile pass over the lattice (Sec. 3.2), GB/s of site bytes read",
            "value": gbs, "unit": "GB/s", "n_gpus": 1, "steps": max(args.steps, 3),
            "warmup": args.warmup, "ms_per_step": 1e3 * t_prof, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "mode": "analysis",
            "config": {"workload": desc, "profile": f"axis z, radius^2 {radius2} half units^2, "
                       f"length {length}, {n_bins} bins", "clusters": f"species {species}, first shell"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "traffic": None, "kernel": "k_profile",
                         "peak_source": peak_src},
            "profile_sites_counted": int(prof.sum()),
            "clusters": {"ms": 1e3 * t_cl, "sites_per_s": N / t_cl,
                         "largest": [int(v) for v in sizes[:8]],
                         "sites_of_species": int(np.count_nonzero(lat.occupancy() == species[0]))},
            "clocks": clk, "gpu_launches": max(args.steps, 3)}
    print(json.dumps(line), flush=True)
    lat.close()
    return 0


def run_exchange(args):
    """Replica exchange (parallel tempering, Sec. 2.2, Eqs. 6-7) through the
    batch.  Throughput ladder: `--jobs` replicas (32 unless given) of one
    system (BCC 128^3 x 2, K = 5, shells 1-3) on a geometric ladder of
    600-1500 K; each round runs `--chunk` sweeps of every replica (one
    graph-captured chunk), then one exchange round over the ladder (even and
    odd neighbour pairs alternately).  value = attempted swaps / wall time of
    `steps` rounds, exchanges included.  Mixing ladder: 64 replicas of BCC
    16^3 x 2 on 800-1200 K, where neighbouring replicas' energies overlap,
    for the acceptance of the exchanges."""
    import torch

    torch.cuda.set_device(0)
    from paper_2509_20949_gb300.batch import Batch

    def ladder_run(R, n, T0, T1):
        kind, K, M = 0, 5, 3
        V = inputs.epi_table(M, K, 0.02, 0)
        occ = inputs.initial_occupancy(kind, n, K, 0)
        sites = inputs.n_sites(kind, n)
        temps = [T0 * (T1 / T0) ** (k / (R - 1)) for k in range(R)]
        rounds = args.warmup + args.steps
        b = Batch(R, Batch.control_bytes(R, sites) + R * Batch.job_bytes(kind, n, K) + (1 << 20),
                  sites)
        ladder = [b.add(kind, n, K, occ, V, T, rounds * args.chunk, seed=k)
                  for k, T in enumerate(temps)]
        acc_total, pairs_total, t_ex = 0, 0, []
        torch.cuda.synchronize()
        for r in range(args.warmup):
            b.run(args.chunk)
            ladder, _ = b.exchange(ladder, 7, r)
        clocks = ClockSampler(0)
        clocks.start()
        t0 = time.perf_counter()
        for r in range(args.warmup, rounds):
            b.run(args.chunk)
            te = time.perf_counter()
            ladder, acc = b.exchange(ladder, 7, r)
            t_ex.append(time.perf_counter() - te)
            acc_total += acc
            pairs_total += (R - (r & 1)) // 2
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        clk = clocks.stop()
        b.close()
        return {"replicas": R, "sites_each": sites, "T": [T0, T1],
                "swaps_per_s": R * sites * args.chunk * args.steps / dt,
                "ms_per_round": 1e3 * dt / args.steps,
                "exchange_ms_per_round": 1e3 * float(np.median(t_ex)), "accepted": acc_total,
                "attempted_pairs": pairs_total, "acceptance": acc_total / max(1, pairs_total),
                "clocks": clk}

    R = args.jobs if args.jobs != 256 else 32
    big = ladder_run(R, (128, 128, 128), 600.0, 1500.0)
    mix = ladder_run(64, (16, 16, 16), 800.0, 1200.0)
    line = {"metric": "attempted MC swaps/sec of a replica-exchange ladder (batched, exchanges included)",
            "value": big["swaps_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": big["ms_per_round"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "mode": "exchange",
            "config": {"workload": f"{R} replicas of BCC 128^3 x 2 = {big['sites_each']} sites, K=5, "
                       "shells 1-3, T geometric 600-1500 K",
                       "step": f"{args.chunk} sweeps of every replica + one exchange round"},
            "throughput_ladder": big, "mixing_ladder": mix, "clocks": big["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "slab":
        return run_slab(args)
    if args.mode == "local":
        return run_local(args)
    if args.mode == "analysis":
        return run_analysis(args)
    if args.mode == "exchange":
        return run_exchange(args)
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2509_20949_gb300.lattice import Lattice

    w, N, desc = workload_config(args.workload)
    V = inputs.epi_table(w["M"], w["K"], w["sigma"], w["epi_seed"])
    occ = inputs.initial_occupancy(w["kind"], w["n"], w["K"], w["occ_seed"], w["fractions"])
    seed = replica_seed(w["seed"], rank)
    stream = torch.cuda.current_stream()
    lat = Lattice(w["kind"], w["n"], w["K"], occ, seed=seed, pack_bits=args.pack_bits,
                  stream=stream)
    if args.kernel:
        lat.set_option(1, args.kernel)
    if args.tile >= 0:
        lat.set_option(2, args.tile)
    if args.staging:
        lat.set_option(3, args.staging)
    lat.set_epi(V)
    M = w["M"]

    def step(i):
        lat.sweep(1, sweep_temperature(w, i), stats=False)

    # warm-up (also where the online kernel choice times its candidates)
    for i in range(args.warmup):
        step(i)
        lat.sro(M)
    torch.cuda.synchronize()
    names = {1: "generic", 2: "tiled", 3: "cell"}
    kt = lat.kernel_tuning()
    kern, shape = lat.kernel_in_use()
    kernel_choice = {"kernel": names.get(kern, str(kern)), "tile_shape": shape,
                     "tuned": kt["done"],
                     "candidates_ms": {f"{names.get(c['kernel'])}{'' if c['shape'] < 0 else c['shape']}":
                                       round(c["best_ms"], 4) for c in kt["candidates"]}}
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev_sweep = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
    ev_step = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev0 = ev_step[0]
    ev0.record(stream)
    for s in range(args.steps):
        a, b = ev_sweep[s]
        a.record(stream)
        step(args.warmup + s)
        b.record(stream)
        lat.sro(M)  # pair counts -> host (the step's result)
        ev_step[s + 1].record(stream)
    ev1 = ev_step[-1]
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_ms = ev0.elapsed_time(ev1)
    sweep_ms = sum(a.elapsed_time(b) for a, b in ev_sweep)
    step_ms = [ev_step[s].elapsed_time(ev_step[s + 1]) for s in range(args.steps)]
    t_ms = max_over_ranks(t_ms)
    total_attempts = N * args.steps * world
    value = total_attempts / (t_ms / 1e3)
    launches_per_sweep = 8
    kernel_ms = sweep_ms / (args.steps * launches_per_sweep)
    alg_bytes_per_launch = 2.0 * N / launches_per_sweep * (0.5 if args.pack_bits == 4 else 1.0)
    peak, peak_src = measured_peaks()
    achieved = alg_bytes_per_launch / (kernel_ms / 1e3) / 1e9

    # end to end through the public API with host buffers
    h_in = torch.empty(N, dtype=torch.uint8, pin_memory=True)
    h_in.numpy()[:] = lat.occupancy()
    h_out = torch.empty(N, dtype=torch.uint8, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_step_s = []
    for s in range(args.e2e_steps):
        ts = time.perf_counter()
        lat.set_occupancy(h_in.numpy())
        step(args.warmup + args.steps + s)
        # the read-back of the swept occupancy (straight into pinned memory)
        # overlaps the pair count, which only reads the lattice
        lat.occupancy_async(h_out.numpy())
        cnt, _ = lat.sro(M)
        lat.wait_occupancy()
        e2e_step_s.append(time.perf_counter() - ts)
        h_in, h_out = h_out, h_in
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = N * args.e2e_steps / e2e_s
    if world > 1:
        e2e_value = N * args.e2e_steps * world / max_over_ranks(e2e_s)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, N, V, occ, args.cpu_seconds, rank)
    rec = (_recorded_profile(N) if args.workload in ("bcc812_k5", "bcc448_k5") and args.pack_bits == 8
           and args.staging == 0 else None)
    traffic = rec["dram_bytes_per_launch"] if rec else None
    # unlike and accepted fractions of the trials of one more sweep (outside the timed region)
    ts = lat.sweep(1, sweep_temperature(w, args.warmup + args.steps + args.e2e_steps))
    trial_stats = {"unlike_frac": ts["unlike"] / ts["attempts"],
                   "accepted_frac": ts["accepted"] / ts["attempts"],
                   "accepted_per_unlike": ts["accepted"] / max(1, ts["unlike"])}
    batched = served = saturated = None
    if world == 1 and (not args.no_batched or not args.no_served):
        lat.close()
        del lat
        torch.cuda.empty_cache()
        if not args.no_batched:
            batched = measure_batched(args.jobs, args.chunk)
        if not args.no_served:
            # below saturation (latency), then a trace the device cannot keep up
            # with alone (aggregate rate against FIFO one job at a time)
            served = measure_served(args.served_rate, args.served_window, args.budget_gb,
                                    args.chunk)
            if args.saturated_rate > 0:
                saturated = measure_served(args.saturated_rate, args.saturated_window,
                                           args.budget_gb, args.chunk, seed=12)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": desc, "step": "1 sweep (8 colour phases) + 1 SRO/energy pair count",
                       "l2": "no flush: 1.07 GB occupancy > 129 MB L2",
                       "pack_bits": args.pack_bits, "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": N,
                    "d2h_bytes_per_step": N + 8 * M * w["K"] * w["K"], "steps": args.e2e_steps,
                    "step_ms": {"median": 1e3 * float(np.median(e2e_step_s)),
                                "min": 1e3 * min(e2e_step_s), "max": 1e3 * max(e2e_step_s)},
                    "value_median": N / float(np.median(e2e_step_s))},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "sweep phase", "kernel_ms_per_launch": kernel_ms,
                         "peak_source": peak_src,
                         "limiter": rec.get("limiter") if rec else None},
            "step_ms": {"median": statistics.median(step_ms), "min": min(step_ms),
                        "max": max(step_ms), "repeats": len(step_ms)},
            "value_median": N * world / (statistics.median(step_ms) / 1e3),
            "kernel_choice": kernel_choice,
            "trial_stats": trial_stats,
            "batched": batched,
            "served": served,
            "served_saturated": saturated,
            "cpu_baseline": cpu,
            "clocks": clk,
            # per step: 8 colour phases + the pair count (K <= 6: bit-mask
            # kernel + its one-thread finishing kernel)
            "gpu_launches": args.steps * (launches_per_sweep + (2 if w["K"] <= 6 else 1)),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _recorded_profile(n_sites):
    """Figures of the committed ncu summary of the tiled sweep phase, if it
    was taken on the current kernel source (else None): the DRAM bytes of
    one phase scaled from the profiled lattice to n_sites sites (a phase
    stages the whole lattice with its halos once, so the traffic grows with
    the sites), and the shared-memory-pipe and issue utilisation."""
    import hashlib
    import re

    prof = os.path.join(ROOT, "profiles", "sweep_tiled_bcc448_k5.md")
    src = os.path.join(ROOT, "paper_2509_20949_gb300", "csrc", "kernels_tiled.cuh")
    try:
        text = open(prof).read()
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    except OSError:
        return None
    m_sha = re.search(r"source_sha1 \(.*?\): ([0-9a-f]+)", text)
    m_b = re.search(r"dram_bytes_per_launch: ([0-9]+)", text)
    m_n = re.search(r"^sites: ([0-9]+)", text, re.M)
    if not m_sha or not m_b or not m_n or m_sha.group(1) != sha:
        return None
    out = {"dram_bytes_per_launch": int(m_b.group(1)) * n_sites // int(m_n.group(1)),
           "profiled_sites": int(m_n.group(1))}
    m_s = re.search(r"shared wavefronts \| [0-9.]+M \(([0-9.]+)% of the shared pipe", text)
    m_i = re.search(r"\| issue active \| ([0-9.]+)%", text)
    if m_s and m_i:
        out["limiter"] = {"unit": "latency of the trial's dependent chain (shared pipe and issue "
                                  "both below saturation)",
                          "shared_pipe_frac": float(m_s.group(1)) / 100.0,
                          "issue_active_frac": float(m_i.group(1)) / 100.0,
                          "source": "profiles/sweep_tiled_bcc448_k5.md"}
    return out




if __name__ == "__main__":
    sys.exit(main())
