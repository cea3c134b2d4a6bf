"""Python handle over a batch of independent lattices (smcx_batch_* C ABI).

PyTorch owns the device arena and the stream; admission, the work queue of
the persistent sweep kernel, its online tuning, the graph-captured chunks and
all computation run in libsmcx.so.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import SweepStats, check
from .lattice import make_desc


class Batch:
    def __init__(self, max_jobs: int, arena_bytes: int, transfer_bytes: int, device=None,
                 stream=None):
        import torch

        self.L = _lib.lib()
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.Stream(dev)
        ctrl = self.L.smcx_batch_control_bytes(int(max_jobs), int(transfer_bytes))
        if ctrl == 0 or arena_bytes < ctrl:
            raise _lib.SmcxError(_lib.SMCX_ENOMEM, f"arena needs at least {ctrl} bytes")
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=dev)
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            check(self.L.smcx_batch_create(int(max_jobs), ctypes.c_void_p(self.arena.data_ptr()),
                                           int(arena_bytes), int(transfer_bytes),
                                           ctypes.c_void_p(self.stream.cuda_stream),
                                           ctypes.byref(h)))
        self.h = h
        self.meta = {}

    @staticmethod
    def control_bytes(max_jobs: int, transfer_bytes: int) -> int:
        return int(_lib.lib().smcx_batch_control_bytes(int(max_jobs), int(transfer_bytes)))

    @staticmethod
    def job_bytes(kind, n, K, pack_bits=8) -> int:
        d = make_desc(kind, n, K, pack_bits)
        return int(_lib.lib().smcx_batch_job_bytes(ctypes.byref(d)))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.smcx_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, kind, n, K, occ, V, T, sweeps, seed=0, flags=0, min_cell=0) -> int:
        """Admits a job; raises SmcxError (status EBUDGET when full)."""
        d = make_desc(kind, n, K, 8, min_cell, flags, seed)
        occ = np.ascontiguousarray(occ, dtype=np.uint8)
        V = np.ascontiguousarray(V, dtype=np.int64)
        jid = ctypes.c_uint32()
        check(self.L.smcx_batch_add(self.h, ctypes.byref(d), ctypes.c_void_p(occ.ctypes.data),
                                    V.shape[0], ctypes.c_void_p(V.ctypes.data), float(T),
                                    int(sweeps), ctypes.byref(jid)))
        j = int(jid.value)
        self.meta[j] = dict(kind=int(kind), n=tuple(int(v) for v in n), K=int(K))
        return j

    def try_add(self, *args, **kw):
        """add() that returns None instead of raising when the budget is full."""
        try:
            return self.add(*args, **kw)
        except _lib.SmcxError as e:
            if e.status == _lib.SMCX_EBUDGET:
                return None
            raise

    def run(self, chunk_sweeps: int) -> int:
        fin = ctypes.c_uint32()
        check(self.L.smcx_batch_run(self.h, int(chunk_sweeps), ctypes.byref(fin)))
        return int(fin.value)

    def launch(self, chunk_sweeps: int):
        """Enqueues one chunk for every active job and returns at once
        (smcx_batch_launch); wait() completes it."""
        check(self.L.smcx_batch_launch(self.h, int(chunk_sweeps)))

    def wait(self) -> int:
        """Completes the launched chunk; the number of jobs finished since the
        last report (smcx_batch_wait)."""
        fin = ctypes.c_uint32()
        check(self.L.smcx_batch_wait(self.h, ctypes.byref(fin)))
        return int(fin.value)

    def poll(self, cap: int = 4096):
        ids = (ctypes.c_uint32 * cap)()
        n = ctypes.c_uint32()
        check(self.L.smcx_batch_poll(self.h, ids, cap, ctypes.byref(n)))
        return [int(ids[i]) for i in range(n.value)]

    def result(self, job_id: int, occupancy: bool = True):
        m = self.meta[job_id]
        N = (2 if m["kind"] == 0 else 4) * m["n"][0] * m["n"][1] * m["n"][2]
        out = np.empty(N, dtype=np.uint8) if occupancy else None
        st = SweepStats()
        e = ctypes.c_int64()
        sw = ctypes.c_uint32()
        check(self.L.smcx_batch_result(self.h, int(job_id),
                                       ctypes.c_void_p(out.ctypes.data) if occupancy else None,
                                       ctypes.byref(st), ctypes.byref(e), ctypes.byref(sw)))
        return dict(occ=out, stats=st.as_dict(), energy=int(e.value), sweeps=int(sw.value))

    def remove(self, job_id: int):
        check(self.L.smcx_batch_remove(self.h, int(job_id)))
        self.meta.pop(job_id, None)

    def info(self):
        a, f = ctypes.c_uint32(), ctypes.c_uint32()
        fb, lb = ctypes.c_size_t(), ctypes.c_size_t()
        check(self.L.smcx_batch_info(self.h, ctypes.byref(a), ctypes.byref(f), ctypes.byref(fb),
                                     ctypes.byref(lb)))
        return dict(active=int(a.value), free_slots=int(f.value), free_bytes=int(fb.value),
                    largest_free=int(lb.value))

    # tuning (never changes results) ---------------------------------------
    OPT_TILE, OPT_OCCUPANCY, OPT_SCHEDULE, OPT_TEST_WAIT_TIMEOUT = 1, 2, 3, 4

    def set_option(self, key: int, value: int):
        """key OPT_TILE (work-item shape index), OPT_SCHEDULE (0 persistent
        plan, 1 one launch per colour phase) or OPT_OCCUPANCY (register
        budget index); value -1 = tuned online."""
        check(self.L.smcx_batch_set_option(self.h, int(key), int(value)))

    def tuning(self):
        t, sc, o, d = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint32()
        check(self.L.smcx_batch_tuning(self.h, ctypes.byref(t), ctypes.byref(sc), ctypes.byref(o),
                                       ctypes.byref(d)))
        return dict(tile=int(t.value), schedule=int(sc.value), occupancy=int(o.value),
                    tuned=bool(d.value))

    @staticmethod
    def tile_shape(i: int):
        c = (ctypes.c_uint32 * 3)()
        check(_lib.lib().smcx_batch_tile_shape(int(i), c))
        return tuple(int(v) for v in c)

    def queue_stats(self):
        """Item ranges of the persistent schedule that waited for their job's
        previous phase, their polls and the nanoseconds waited (summed over
        warps), since creation."""
        out = (ctypes.c_uint64 * 3)()
        check(self.L.smcx_batch_queue_stats(self.h, out))
        return dict(waited_items=int(out[0]), polls=int(out[1]), wait_ns=int(out[2]))

    # replica exchange ------------------------------------------------------
    def exchange(self, ladder, seed: int, rnd: int):
        """One replica-exchange round (Sec. 2.2, Eqs. 6-7) over `ladder`
        (job ids, ladder[k] = the job at the k-th temperature).  Returns the
        new ladder and the number of accepted pairs."""
        lad = (ctypes.c_uint32 * len(ladder))(*[int(j) for j in ladder])
        acc = ctypes.c_uint32()
        check(self.L.smcx_batch_exchange(self.h, lad, len(ladder), int(seed), int(rnd),
                                         ctypes.byref(acc)))
        return [int(v) for v in lad], int(acc.value)

    def temperature(self, job_id: int) -> float:
        t = ctypes.c_double()
        check(self.L.smcx_batch_temperature(self.h, int(job_id), ctypes.byref(t)))
        return float(t.value)
