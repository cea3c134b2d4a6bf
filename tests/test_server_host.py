"""Host logic of the continuous-batching server (not gpu): admission order
and its bypass limit, the per-chunk accounting of sweeps and swaps, the
pipelined trace loop (admissions and read-backs while a chunk is in
flight) and the metrics, against a fake batch that advances jobs the way
the batch runtime does (every active job by min(chunk, sweeps left) per
chunk; a job is reported by poll() once the chunk that finished it has
completed) and a fake clock."""
import collections

import numpy as np
import pytest

from paper_2509_20949_gb300.server import Server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBatch:
    """Slots and a byte budget (1 byte per site); chunks take `sec_per_chunk`
    on the fake clock, advanced when the chunk completes."""

    def __init__(self, clock, slots, budget, sec_per_chunk=1.0):
        self.clock, self.slots, self.budget = clock, slots, budget
        self.sec = sec_per_chunk
        self.jobs = {}            # id -> dict(sites, sweeps, done)
        self.next_id = 0
        self.flight = None        # (chunk, ids) of the chunk on the device
        self.finished = collections.deque()
        self.removed = []
        self.launches = 0

    def used(self):
        return sum(j["sites"] for j in self.jobs.values())

    def try_add(self, kind, n, K, occ, V, T, sweeps, seed=0):
        sites = (2 if kind == 0 else 4) * int(np.prod(n))
        if len(self.jobs) >= self.slots or self.used() + sites > self.budget:
            return None
        jid = self.next_id
        self.next_id += 1
        self.jobs[jid] = dict(sites=sites, sweeps=sweeps, done=0, seed=seed)
        return jid

    def _active(self):
        return [j for j, v in self.jobs.items() if v["done"] < v["sweeps"]]

    def launch(self, chunk):
        assert self.flight is None
        self.launches += 1
        self.flight = (chunk, self._active())

    def wait(self):
        if self.flight is None:
            return 0
        chunk, ids = self.flight
        self.flight = None
        self.clock.t += self.sec
        fin = 0
        for j in ids:
            v = self.jobs[j]
            v["done"] += min(chunk, v["sweeps"] - v["done"])
            if v["done"] == v["sweeps"]:
                self.finished.append(j)
                fin += 1
        return fin

    def run(self, chunk):
        self.launch(chunk)
        return self.wait()

    def poll(self, cap=4096):
        out = []
        while self.finished and len(out) < cap:
            out.append(self.finished.popleft())
        return out

    def result(self, jid):
        v = self.jobs[jid]
        return dict(occ=np.full(4, v["seed"], np.uint8), stats={}, energy=0, sweeps=v["done"])

    def remove(self, jid):
        self.removed.append(jid)
        del self.jobs[jid]

    def close(self):
        pass


def _server(slots=4, budget=10_000, chunk=10, sec=1.0):
    clock = FakeClock()
    srv = Server.__new__(Server)
    srv.batch = FakeBatch(clock, slots, budget, sec)
    srv.chunk = chunk
    srv.clock = clock
    srv.queue = collections.deque()
    srv.running = {}
    srv.done = {}
    srv.next_ticket = 0
    srv.swaps = 0
    srv.swaps_finished = 0
    srv.progress = {}
    srv.chunks = 0
    srv.max_bypass = 64
    return srv, clock


def _job(n, sweeps, seed, arrival=0.0, kind=0):
    return dict(kind=kind, n=(n, n, n), K=2, occ=None, V=None, T=1000.0, sweeps=sweeps,
                seed=seed, job=seed, arrival_s=arrival)


def test_step_accounting_and_results():
    srv, clock = _server(chunk=10)
    a, b = _job(4, 25, 1), _job(5, 10, 2)          # 128 and 250 sites
    ta, tb = srv.submit(a), srv.submit(b)
    assert srv.step() == 1                         # b finishes in its first chunk
    assert srv.swaps == 128 * 10 + 250 * 10
    assert srv.step() == 0
    assert srv.step() == 1                         # a: 10 + 10 + 5 sweeps
    assert srv.swaps == 128 * 25 + 250 * 10 == srv.swaps_finished
    assert srv.idle() and srv.chunks == 3
    assert srv.done[ta]["latency_s"] == pytest.approx(3.0)
    assert srv.done[tb]["latency_s"] == pytest.approx(1.0)
    assert srv.done[ta]["sweeps"] == 25 and srv.done[ta]["job"] == 1
    assert sorted(srv.batch.removed) == [0, 1]     # every finished job freed
    assert srv.step() == 0                         # nothing left: no launch
    assert srv.batch.launches == 3


def test_admission_is_fifo_with_a_bounded_bypass():
    srv, clock = _server(slots=8, budget=1000, chunk=5)
    srv.max_bypass = 2
    big = _job(6, 5, 100)                          # 432 sites
    srv.submit(_job(6, 50, 1))                     # 432: admitted
    srv.submit(big)                                # 432 more would be 864 <= 1000: admitted
    srv.submit(_job(6, 5, 101))                    # does not fit (1296)
    for k in range(4):
        srv.submit(_job(2, 5, 200 + k))            # 16 sites each: may overtake it twice
    srv._admit()
    seeds = sorted(v[1]["seed"] for v in srv.running.values())
    assert seeds == [1, 100, 200, 201]             # the waiting head was overtaken twice, then starves
    assert [q[1]["seed"] for q in srv.queue] == [101, 202, 203]
    # the next pass still holds the later jobs back behind the head
    srv._admit()
    assert [q[1]["seed"] for q in srv.queue] == [101, 202, 203]
    srv.step()                                      # big and the two small ones finish
    assert sorted(v[1]["seed"] for v in srv.running.values()) == [1]
    srv._admit()                                    # room again: the head first, then the rest
    assert sorted(v[1]["seed"] for v in srv.running.values()) == [1, 101, 202, 203]
    assert not srv.queue


def test_pipelined_trace_runs_every_job_and_accounts_every_swap(monkeypatch):
    import paper_2509_20949_gb300.server as server_mod
    jobs = [_job(3 + (k % 4), 7 + 9 * (k % 5), k, arrival=0.4 * k) for k in range(12)]
    srv, clock = _server(slots=3, budget=600, chunk=8, sec=0.5)
    # the fake clock moves when a chunk completes and when the loop idles
    # until the next arrival
    monkeypatch.setattr(server_mod.time, "sleep", lambda dt: setattr(clock, "t", clock.t + max(dt, 0.01)))
    m = srv.run_trace(jobs)
    assert m["completed"] == m["submitted"] == 12
    assert srv.idle()
    want = sum((2 * int(np.prod(j["n"]))) * j["sweeps"] for j in jobs)
    assert srv.swaps == srv.swaps_finished == want
    for t, r in srv.done.items():
        assert r["sweeps"] == jobs[r["job"]]["sweeps"]
        assert r["latency_s"] > 0 and r["finish_s"] >= r["arrival_s"]
    assert m["p50_latency_s"] <= m["p99_latency_s"]
    assert m["swaps_per_s"] == pytest.approx(want / m["elapsed_s"])
