"""Continuous-batching simulation server over one GPU.

Jobs (lattice, EPI, temperature, sweeps) arrive over time; the server admits
waiting jobs whenever a job slot and room in the device arena (the HBM
budget) are free, keeps every admitted lattice resident on the device
between chunks, runs one graph-captured chunk of sweeps for all resident
jobs at a time (new arrivals join at the next chunk boundary), returns each
finished job's result to the host and frees its space.  Host work overlaps
the device: while a chunk runs, arrivals are admitted (their uploads and
initial energies on the batch's side stream) and the jobs finished by the
previous chunk are read back, so the next chunk starts as soon as this one
ends.  Each job's result is bit-identical to the same lattice run alone (the
batch runtime guarantees it).  Latency = time from arrival to the result on
the host.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from .batch import Batch


def _sites(job) -> int:
    return (2 if job["kind"] == 0 else 4) * int(np.prod(job["n"]))


class Server:
    def __init__(self, budget_bytes: int, max_jobs: int = 1024, chunk_sweeps: int = 50,
                 transfer_bytes: int = 1 << 27, clock=time.perf_counter, device=None):
        ctrl = Batch.control_bytes(max_jobs, transfer_bytes)
        self.batch = Batch(max_jobs, ctrl + int(budget_bytes), transfer_bytes, device=device)
        self.chunk = int(chunk_sweeps)
        self.clock = clock
        self.queue = collections.deque()  # waiting jobs: (ticket, job, arrival)
        self.running = {}                  # batch id -> (ticket, job, arrival)
        self.done = {}                     # ticket -> result dict
        self.next_ticket = 0
        self.swaps = 0                     # attempted swaps run on the GPU (all jobs)
        self.swaps_finished = 0            # of which in jobs that have finished
        self.progress = {}                 # batch id -> sweeps done
        self.chunks = 0
        self.max_bypass = 64               # how many later jobs may overtake a waiting head

    def submit(self, job: dict, arrival: float | None = None) -> int:
        """job: kind, n, K, occ, V, T, sweeps, seed (see inputs.served_jobs)."""
        t = self.clock() if arrival is None else arrival
        ticket = self.next_ticket
        self.next_ticket += 1
        self.queue.append((ticket, job, t, 0))
        return ticket

    def _admit(self):
        """FIFO admission; a job that does not fit yet may be overtaken by
        later ones, at most max_bypass times (then admission waits for it)."""
        remaining = collections.deque()
        starving = False
        while self.queue:
            item = self.queue.popleft()
            ticket, job, arr, bypassed = item
            if starving:
                remaining.append(item)
                continue
            jid = self.batch.try_add(job["kind"], job["n"], job["K"], job["occ"], job["V"],
                                     job["T"], job["sweeps"], seed=job["seed"])
            if jid is None:
                remaining.append(item)
                starving = bypassed >= self.max_bypass
                continue
            self.running[jid] = (ticket, job, arr)
            self.progress[jid] = 0
            # every job still waiting ahead of this one has been overtaken once
            # more; one that has reached the limit stops the later ones
            remaining = collections.deque((t, j, a, b + 1) for (t, j, a, b) in remaining)
            starving = any(b >= self.max_bypass for (_, _, _, b) in remaining)
        self.queue = remaining

    def _account(self, jids):
        """Advances the progress (sweeps launched) of the jobs of a chunk as it
        is launched: a job whose last chunk is on the device is not active."""
        for jid in jids:
            _, job, _ = self.running[jid]
            ran = min(self.chunk, job["sweeps"] - self.progress[jid])
            self.progress[jid] += ran
            self.swaps += _sites(job) * ran

    def _collect(self):
        """Reads back, frees and records every job finished by a completed
        chunk (through the side stream while a chunk runs)."""
        for jid in self.batch.poll():
            ticket, job, arr = self.running.pop(jid)
            r = self.batch.result(jid)
            self.batch.remove(jid)
            now = self.clock()
            r["job"] = job.get("job", ticket)
            r["latency_s"] = now - arr
            r["arrival_s"] = arr
            r["finish_s"] = now
            self.done[ticket] = r
            self.progress.pop(jid, None)
            self.swaps_finished += _sites(job) * job["sweeps"]

    def _active(self):
        return [jid for jid, (_, job, _) in self.running.items()
                if self.progress[jid] < job["sweeps"]]

    def step(self) -> int:
        """Admit, run one chunk to completion, collect finished jobs.
        Returns the jobs finished."""
        self._admit()
        jids = self._active()
        if not jids:
            return 0
        self.batch.run(self.chunk)
        self.chunks += 1
        self._account(jids)
        before = len(self.done)
        self._collect()
        return len(self.done) - before

    def idle(self) -> bool:
        return not self.queue and not self.running

    def run_trace(self, jobs: list, window_s: float | None = None, drain: bool = True,
                  deadline_s: float | None = None):
        """Replays an arrival trace (each job has arrival_s) in real time,
        overlapping each chunk with the admissions and read-backs around it.
        Returns the metrics of the completed jobs."""
        t0 = self.clock()
        pending = sorted(jobs, key=lambda j: j["arrival_s"])
        k = 0
        flight = None  # job ids of the chunk on the device

        def arrive():
            nonlocal k
            now = self.clock() - t0
            while k < len(pending) and pending[k]["arrival_s"] <= now:
                self.submit(pending[k], arrival=t0 + pending[k]["arrival_s"])
                k += 1

        while True:
            arrive()
            if flight is not None:
                # while the chunk runs: admit arrivals for the next chunk and
                # read back the jobs finished by the previous one
                self._admit()
                self._collect()
                self.batch.wait()
                flight = None
            self._admit()
            jids = self._active()
            if jids:
                self.batch.launch(self.chunk)
                self._account(jids)
                self.chunks += 1
                flight = jids
            else:
                self._collect()
                if k < len(pending) and not self.running:
                    time.sleep(max(0.0, min(0.01, pending[k]["arrival_s"] - (self.clock() - t0))))
            if flight is None and k >= len(pending) and (not drain or self.idle()):
                break
            if deadline_s is not None and self.clock() - t0 > deadline_s:
                if flight is not None:
                    self.batch.wait()
                break
        elapsed = self.clock() - t0
        return self.metrics(elapsed, submitted=k)

    def metrics(self, elapsed_s: float, submitted: int | None = None) -> dict:
        lat = np.array([r["latency_s"] for r in self.done.values()], dtype=np.float64)
        sub = self.next_ticket if submitted is None else submitted
        return {
            "completed": len(self.done), "submitted": sub,
            "completed_fraction": (len(self.done) / sub) if sub else 0.0,
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "swaps_per_s": self.swaps / elapsed_s if elapsed_s > 0 else 0.0,
            "finished_swaps_per_s": self.swaps_finished / elapsed_s if elapsed_s > 0 else 0.0,
            "elapsed_s": elapsed_s, "chunks": self.chunks,
        }

    def close(self):
        self.batch.close()
