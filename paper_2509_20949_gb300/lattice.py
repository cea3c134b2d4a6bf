"""Python handle over one lattice of the C ABI (include/smcx.h).

PyTorch provides the device buffers (occupancy, workspace) and the CUDA
stream; every computation runs inside libsmcx.so.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import LatticeDesc, SweepStats, check

BCC, FCC = 0, 1
NO_SHIFT, SINGLE_CELL = 1, 2
OPT_KERNEL, OPT_TILE = 1, 2
KERNEL_AUTO, KERNEL_GENERIC, KERNEL_TILED, KERNEL_CELL, KERNEL_LOCAL = 0, 1, 2, 3, 4


def make_desc(kind, n, n_species, pack_bits=8, min_cell=0, flags=0, seed=0) -> LatticeDesc:
    d = LatticeDesc()
    d.kind = int(kind)
    d.n[0], d.n[1], d.n[2] = (int(v) for v in n)
    d.n_species = int(n_species)
    d.pack_bits = int(pack_bits)
    d.min_cell = int(min_cell)
    d.flags = int(flags)
    d.seed = int(seed)
    return d


def local_model_width(kind, n_shells) -> int:
    """Count-axis length of a local-energy table (1 + max z_m), 0 if invalid."""
    return int(_lib.lib().smcx_local_model_width(int(kind), int(n_shells)))


def _host_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class Lattice:
    """One simulated lattice.  occ: canonical uint8 occupancy (host array)."""

    def __init__(self, kind, n, n_species, occ, seed=0, pack_bits=8, min_cell=0, flags=0,
                 device=None, stream=None):
        import torch

        self._torch = torch
        self.L = _lib.lib()
        self.desc = make_desc(kind, n, n_species, pack_bits, min_cell, flags, seed)
        self.kind, self.n, self.K = int(kind), tuple(int(v) for v in n), int(n_species)
        self.N = (2 if self.kind == BCC else 4) * self.n[0] * self.n[1] * self.n[2]
        occ = np.ascontiguousarray(occ, dtype=np.uint8)
        if occ.size != self.N:
            raise ValueError(f"occupancy has {occ.size} sites, lattice needs {self.N}")
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        ob = self.L.smcx_occupancy_bytes(ctypes.byref(self.desc))
        wb = self.L.smcx_workspace_bytes(ctypes.byref(self.desc))
        if ob == 0 or wb == 0:
            raise _lib.SmcxError(_lib.SMCX_EINVAL, "invalid lattice descriptor")
        # torch's caching allocator returns 512-byte aligned blocks
        self.d_occ = torch.empty(ob, dtype=torch.uint8, device=dev)
        self.d_work = torch.empty(wb, dtype=torch.uint8, device=dev)
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            check(self.L.smcx_create_lattice(ctypes.byref(self.desc),
                                             ctypes.c_void_p(self.d_occ.data_ptr()),
                                             ctypes.c_void_p(self.d_work.data_ptr()),
                                             _host_ptr(occ), ctypes.c_void_p(self.stream.cuda_stream),
                                             ctypes.byref(h)))
        self.h = h
        self.M = 0
        self.local_model = False

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.smcx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_epi(self, V):
        V = np.ascontiguousarray(V, dtype=np.int64)
        if V.ndim != 3 or V.shape[1] != self.K or V.shape[2] != self.K:
            raise ValueError("EPI table must be [M][K][K]")
        check(self.L.smcx_set_epi(self.h, V.shape[0], _host_ptr(V)))
        self.M = V.shape[0]
        self.local_model = False

    def set_local_model(self, T):
        """Local-energy model (the nonlinear short-range model of Sec. 3):
        T is [M][K][K][zt] int64 q units, T[m][a][s][c] = energy of a site of
        species a whose shell m+1 holds c sites of species s
        (zt = local_model_width(kind, M))."""
        T = np.ascontiguousarray(T, dtype=np.int64)
        if T.ndim != 4 or T.shape[1] != self.K or T.shape[2] != self.K:
            raise ValueError("local-energy table must be [M][K][K][zt]")
        if T.shape[3] != local_model_width(self.kind, T.shape[0]):
            raise ValueError("local-energy table: wrong count axis length")
        check(self.L.smcx_set_local_model(self.h, T.shape[0], _host_ptr(T)))
        self.M = T.shape[0]
        self.local_model = True

    def set_option(self, key, value):
        check(self.L.smcx_set_option(self.h, int(key), int(value)))

    def sweep(self, n_sweeps=1, T_first=1000.0, T_last=None, stats=True):
        T_last = T_first if T_last is None else T_last
        st = SweepStats()
        check(self.L.smcx_sweep(self.h, int(n_sweeps), float(T_first), float(T_last),
                                ctypes.byref(st) if stats else None))
        return st.as_dict() if stats else None

    def run_colour(self, colour, T):
        st = SweepStats()
        check(self.L.smcx_run_colour(self.h, int(colour), float(T), ctypes.byref(st)))
        return st.as_dict()

    def run_colour_planes(self, colour, T, c_lo, c_hi):
        """One colour phase of the current sweep over the link cells whose z
        index lies in [c_lo, c_hi) (a rank's share of a z decomposition)."""
        st = SweepStats()
        check(self.L.smcx_run_colour_planes(self.h, int(colour), float(T), int(c_lo), int(c_hi),
                                            ctypes.byref(st)))
        return st.as_dict()

    def planes_buffer(self, nz):
        """A device buffer for nz conventional z planes in storage order."""
        return self._torch.empty(int(self.L.smcx_planes_bytes(self.h, int(nz))),
                                 dtype=self._torch.uint8, device=self.device)

    def get_planes(self, z0, nz, buf):
        check(self.L.smcx_get_planes(self.h, int(z0), int(nz), ctypes.c_void_p(buf.data_ptr())))
        return buf

    def put_planes(self, z0, nz, buf):
        check(self.L.smcx_put_planes(self.h, int(z0), int(nz), ctypes.c_void_p(buf.data_ptr())))

    def merge_planes(self, z0, nz, theirs, before):
        check(self.L.smcx_merge_planes(self.h, int(z0), int(nz), ctypes.c_void_p(theirs.data_ptr()),
                                       ctypes.c_void_p(before.data_ptr())))

    def synchronize(self):
        self.stream.synchronize()

    def energy(self) -> int:
        e = ctypes.c_int64()
        check(self.L.smcx_energy(self.h, ctypes.byref(e)))
        return int(e.value)

    def running_energy(self) -> int:
        e = ctypes.c_int64()
        check(self.L.smcx_running_energy(self.h, ctypes.byref(e)))
        return int(e.value)

    def sro(self, n_shells):
        cnt = np.zeros((n_shells, self.K, self.K), dtype=np.uint64)
        alpha = np.zeros((n_shells, self.K, self.K), dtype=np.float64)
        check(self.L.smcx_warren_cowley_sro(self.h, int(n_shells), _host_ptr(cnt), _host_ptr(alpha)))
        return cnt, alpha

    def occupancy(self, out: np.ndarray | None = None) -> np.ndarray:
        """Canonical occupancy (N bytes).  `out`: a contiguous uint8 array
        of N bytes to fill (e.g. a view of pinned host memory, which the
        device-to-host copy then reaches directly)."""
        if out is None:
            out = np.empty(self.N, dtype=np.uint8)
        elif out.dtype != np.uint8 or out.size != self.N or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a contiguous uint8 array of N bytes")
        check(self.L.smcx_get_occupancy(self.h, _host_ptr(out)))
        return out

    def occupancy_async(self, out: np.ndarray) -> np.ndarray:
        """Starts copying the occupancy as it is at this point of the stream
        into `out` (a contiguous uint8 array of N bytes, best a view of
        pinned host memory) and returns at once; the copy overlaps what is
        enqueued next.  `out` is complete after wait_occupancy()."""
        if out.dtype != np.uint8 or out.size != self.N or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a contiguous uint8 array of N bytes")
        check(self.L.smcx_get_occupancy_async(self.h, _host_ptr(out)))
        self._pending_out = out  # kept alive until the copy has landed
        return out

    def wait_occupancy(self):
        """Waits for the copy started by the last occupancy_async()."""
        check(self.L.smcx_wait_occupancy(self.h))
        self._pending_out = None

    def set_occupancy(self, occ):
        occ = np.ascontiguousarray(occ, dtype=np.uint8)
        if occ.size != self.N:
            raise ValueError("wrong occupancy size")
        check(self.L.smcx_set_occupancy(self.h, _host_ptr(occ)))

    @property
    def sweep_counter(self) -> int:
        t = ctypes.c_uint32()
        check(self.L.smcx_get_sweep_counter(self.h, ctypes.byref(t)))
        return int(t.value)

    @sweep_counter.setter
    def sweep_counter(self, t):
        check(self.L.smcx_set_sweep_counter(self.h, int(t)))

    def layout(self):
        L = ctypes.c_uint32()
        m = (ctypes.c_uint32 * 3)()
        check(self.L.smcx_get_layout(self.h, ctypes.byref(L), m))
        return int(L.value), tuple(int(v) for v in m)

    def kernel_in_use(self):
        k = ctypes.c_uint32()
        sh = ctypes.c_int32()
        check(self.L.smcx_kernel_in_use(self.h, ctypes.byref(k), ctypes.byref(sh)))
        return int(k.value), int(sh.value)

    def kernel_tuning(self):
        """Online kernel choice: done flag and, per candidate (kernel, tile
        shape), the fastest timed colour phase in ms (-1 if not timed)."""
        done, n = ctypes.c_uint32(), ctypes.c_uint32(8)
        k = (ctypes.c_uint32 * 8)()
        sh = (ctypes.c_int32 * 8)()
        ms = (ctypes.c_float * 8)()
        check(self.L.smcx_kernel_tuning(self.h, ctypes.byref(done), ctypes.byref(n), k, sh, ms))
        cands = [dict(kernel=int(k[c]), shape=int(sh[c]), best_ms=float(ms[c]))
                 for c in range(min(int(n.value), 8))]
        return dict(done=bool(done.value), candidates=cands)

    def composition_profile(self, axis, origin_h, radius2_h, length_h, n_bins):
        """Species counts [n_bins][K] along a cylinder (see smcx.h); positions
        in half lattice-constant units."""
        counts = np.zeros((int(n_bins), self.K), dtype=np.uint64)
        o = (ctypes.c_int32 * 3)(*[int(v) for v in origin_h])
        check(self.L.smcx_composition_profile(self.h, int(axis), o, int(radius2_h), int(length_h),
                                              int(n_bins), _host_ptr(counts)))
        return counts

    def clusters(self, species, cap=None):
        """Sizes (descending) of the first-shell-connected clusters of the
        sites whose species is in `species` (precipitates, Sec. 3.2)."""
        torch = self._torch
        mask = 0
        for sp in species:
            mask |= 1 << int(sp)
        scratch = torch.empty(8 * self.N, dtype=torch.uint8, device=self.device)
        n = ctypes.c_uint64()
        cap = self.N if cap is None else int(cap)
        sizes = np.zeros(max(cap, 1), dtype=np.uint64)
        check(self.L.smcx_clusters(self.h, mask, ctypes.c_void_p(scratch.data_ptr()),
                                   8 * self.N, ctypes.byref(n), _host_ptr(sizes), cap))
        return sizes[: min(cap, int(n.value))]

    def sro_average(self, n_shells, n_samples, sweeps_between, T):
        """Warren-Cowley parameters averaged over configurations (Sec. 3.2,
        Eq. 9): n_samples snapshots, each after sweeps_between sweeps at T.
        The species counts are conserved by swaps, so alpha is linear in the
        pair counts and the average of alpha is alpha of the summed counts.
        Returns (summed pair counts, mean alpha)."""
        total = None
        alphas = []
        for _ in range(int(n_samples)):
            self.sweep(int(sweeps_between), float(T), stats=False)
            cnt, alpha = self.sro(n_shells)
            total = cnt.copy() if total is None else total + cnt
            alphas.append(alpha)
        return total, np.mean(np.stack(alphas), axis=0)

    def checkpoint(self) -> bytes:
        n = ctypes.c_size_t()
        check(self.L.smcx_checkpoint(self.h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        check(self.L.smcx_checkpoint(self.h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        check(self.L.smcx_restore(self.h, buf, len(blob)))
