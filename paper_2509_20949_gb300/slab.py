"""Lattice decomposition along z (Sec. 2.2, lattice parallelism).

One lattice is swept by several ranks (one per GPU).  In every sweep each rank
runs the link cells of its range of z planes of that sweep's moving cell grid,
and ranks trade boundary planes so that the trajectory is the single-lattice
one, bit for bit:

* colours 0-3 are the even link-cell planes and 4-7 the odd ones.  Two cells of
  one z parity never interact, so within a half sweep no rank reads a site
  that another writes, and no site is written by two ranks;
* after each half sweep the two ranks at an ownership boundary trade the
  2 x halo planes around it and merge them as mine ^ theirs ^ before;
* when the grid moves for the next sweep, each rank fetches the planes of its
  new window from their previous owners;
* computation-communication overlap (Sec. 3.1): link-cell planes of one z
  parity never interact either, so a half sweep may run plane by plane.  A
  rank sweeps (all four colours of the half) its first and last plane of
  that parity -- the only ones that write or read the boundary regions --
  sends those regions, and sweeps its interior planes while they travel;
  the merge waits for them.  The trajectory is the same.

Every rank keeps a whole-lattice buffer (one byte per site: a 1e10-site
lattice is 10 GB of a GPU's HBM) that is current on its window only.

The plan arithmetic is libsmcx.so's smcx_slab_plan / smcx_slab_transfer, and
the sweeps, plane copies and merges run in its kernels.  This module orders
those calls and moves plane buffers with torch.distributed: device buffers
over NCCL, host-staged over gloo.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import Slab, check

_TAG_UP, _TAG_DOWN, _TAG_MOVE = 1, 2, 10


def plan(desc, n_shells, world, rank, t) -> dict:
    """smcx_slab_plan: the link-cell z range [c_lo, c_hi) rank `rank` sweeps
    in sweep t, its owned planes [z_lo, z_lo + n_own) (mod n_z), halo, m_z."""
    out = Slab()
    check(_lib.lib().smcx_slab_plan(ctypes.byref(desc), int(n_shells), int(world), int(rank),
                                    int(t), ctypes.byref(out)))
    return out.as_dict()


def transfer(desc, n_shells, world, src, dst, t) -> list:
    """smcx_slab_transfer: runs (z0, nz) of planes that rank src owned in
    sweep t and rank dst reads in sweep t + 1."""
    runs = (ctypes.c_int32 * 4)()
    n = ctypes.c_uint32()
    check(_lib.lib().smcx_slab_transfer(ctypes.byref(desc), int(n_shells), int(world), int(src),
                                        int(dst), int(t), runs, ctypes.byref(n)))
    return [(int(runs[2 * i]), int(runs[2 * i + 1])) for i in range(n.value)]


class SlabSweep:
    """This rank's share of one lattice decomposed along z.

    `lattice` is this rank's whole-lattice handle (a Lattice with its EPI
    set; every rank starts from the same occupancy, EPI and seed).  `group`:
    a torch.distributed process group (default: the world, or one rank when
    torch.distributed is not initialised)."""

    def __init__(self, lattice, group=None, overlap=True):
        import torch
        import torch.distributed as dist

        self._torch = torch
        self._dist = dist
        self.lat = lattice
        self.group = group
        if dist.is_available() and dist.is_initialized():
            self.world = dist.get_world_size(group)
            self.rank = dist.get_rank(group)
            self.device_comm = dist.get_backend(group) == "nccl"
        else:
            self.world, self.rank, self.device_comm = 1, 0, False
        if not lattice.M:
            raise ValueError("set the lattice's EPI before decomposing it")
        if getattr(lattice, "local_model", False):
            raise ValueError("the z decomposition plans EPI link cells; the local-energy "
                             "model's cells are larger")
        self.n_z = int(lattice.desc.n[2])
        self.overlap = bool(overlap)
        plan(lattice.desc, lattice.M, self.world, self.rank, 0)  # raises if the split is invalid

    # ------------------------------------------------------------------
    def plan(self, t, rank=None) -> dict:
        return plan(self.lat.desc, self.lat.M, self.world, self.rank if rank is None else rank, t)

    def _global(self, r):
        """Rank r of the group as a global rank (what P2POp wants)."""
        if self.group is None:
            return r
        return self._dist.get_global_rank(self.group, r)

    def _wire(self, buf):
        """What goes over the backend: the device buffer (NCCL) or a host copy."""
        return buf if self.device_comm else buf.cpu()

    def _wire_empty(self, nz):
        buf = self.lat.planes_buffer(nz)
        return buf if self.device_comm else self._torch.empty_like(buf, device="cpu")

    def _to_lattice(self, host_buf, nz):
        """A received host buffer copied to a lattice buffer on the lattice's
        own stream, so that the library calls that follow on that stream see
        the copy complete."""
        dev = self.lat.planes_buffer(nz)
        stream = getattr(self.lat, "stream", None)
        if stream is not None and dev.is_cuda:
            with self._torch.cuda.stream(stream):
                dev.copy_(host_buf)
        else:
            dev.copy_(host_buf)
        return dev

    def _p2p(self, sends, recvs):
        """sends: [(peer, tensor, tag)], recvs: [(peer, tensor, tag)], posted
        as one batch (NCCL groups them, so no pair waits on the other's order)."""
        self._p2p_wait(self._p2p_post(sends, recvs))

    def _p2p_post(self, sends, recvs):
        dist = self._dist
        ops = [dist.P2POp(dist.isend, t, self._global(p), self.group, tag) for p, t, tag in sends]
        ops += [dist.P2POp(dist.irecv, t, self._global(p), self.group, tag) for p, t, tag in recvs]
        return dist.batch_isend_irecv(ops) if ops else []

    def _p2p_wait(self, works):
        if works:
            for w in works:
                w.wait()
            self._after_comm()

    def _after_comm(self):
        """NCCL's completion orders PyTorch's current stream only: the lattice's
        stream waits for it before the library reads received buffers."""
        stream = getattr(self.lat, "stream", None)
        if self.device_comm and stream is not None:
            stream.wait_stream(self._torch.cuda.current_stream(self.lat.device))

    def _regions(self, p):
        h = p["halo"]
        lo = (p["z_lo"] - h) % self.n_z
        hi = (p["z_lo"] + p["n_own"] - h) % self.n_z
        return lo, hi, 2 * h

    def _merge_boundaries(self, p, before, overlapped=None):
        """Trades the planes around both ownership boundaries with the two
        neighbours and merges them (each site changed on one side at most).
        overlapped(): work to run while the planes travel (no part of it may
        read or write them)."""
        lo, hi, nb = self._regions(p)
        lat = self.lat
        mine_lo = lat.get_planes(lo, nb, lat.planes_buffer(nb))
        mine_hi = lat.get_planes(hi, nb, lat.planes_buffer(nb))
        lat.synchronize()
        up, down = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        theirs_lo, theirs_hi = self._wire_empty(nb), self._wire_empty(nb)
        # my upper region goes up (the upper rank's lower one), my lower one down
        works = self._p2p_post(
            [(up, self._wire(mine_hi), _TAG_UP), (down, self._wire(mine_lo), _TAG_DOWN)],
            [(down, theirs_lo, _TAG_UP), (up, theirs_hi, _TAG_DOWN)])
        if overlapped is not None:
            overlapped()
        self._p2p_wait(works)
        if not self.device_comm:
            theirs_lo = self._to_lattice(theirs_lo, nb)
            theirs_hi = self._to_lattice(theirs_hi, nb)
        lat.merge_planes(lo, nb, theirs_lo, before[0])
        lat.merge_planes(hi, nb, theirs_hi, before[1])

    @staticmethod
    def _half_planes(c_lo, c_hi, half):
        """This rank's link-cell planes of z parity `half` in [c_lo, c_hi) as
        (boundary runs, interior run or None): the first and the last plane
        are the boundary ones, the planes between them the interior."""
        first = c_lo if c_lo % 2 == half else c_lo + 1
        last = c_hi - 1 if (c_hi - 1) % 2 == half else c_hi - 2
        if last < first:
            return [], None
        runs = [(first, first + 1)] + ([(last, last + 1)] if last > first else [])
        return runs, ((first + 1, last) if last - first >= 4 else None)

    def _move(self, t):
        """After sweep t: every rank fetches the planes of its sweep-(t+1)
        window from their sweep-t owners."""
        lat = self.lat
        sends, recvs, puts = [], [], []
        for src in range(self.world):
            for dst in range(self.world):
                if src == dst or self.rank not in (src, dst):
                    continue
                for k, (z0, nz) in enumerate(transfer(lat.desc, lat.M, self.world, src, dst, t)):
                    if self.rank == src:
                        sends.append((dst, lat.get_planes(z0, nz, lat.planes_buffer(nz)),
                                      _TAG_MOVE + k))
                    else:
                        buf = self._wire_empty(nz)
                        recvs.append((src, buf, _TAG_MOVE + k))
                        puts.append((z0, nz, buf))
        lat.synchronize()
        self._p2p([(p, self._wire(b), tag) for p, b, tag in sends], recvs)
        for z0, nz, buf in puts:
            if not self.device_comm:
                buf = self._to_lattice(buf, nz)
            lat.put_planes(z0, nz, buf)
        lat.synchronize()

    def _allreduce(self, v):
        if self.world == 1:
            return v
        torch = self._torch
        t = torch.tensor(v, dtype=torch.int64)
        if self.device_comm:
            t = t.to(self.lat.device)
        self._dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    # ------------------------------------------------------------------
    def sweep(self, n_sweeps=1, T_first=1000.0, T_last=None) -> dict:
        """n_sweeps MC steps of the whole lattice, temperature linear from
        T_first to T_last as smcx_sweep; returns the trial statistics summed
        over every rank (the single-lattice numbers)."""
        T_last = T_first if T_last is None else T_last
        lat = self.lat
        tot = np.zeros(4, dtype=np.int64)
        for i in range(int(n_sweeps)):
            T = T_first
            if n_sweeps > 1 and T_first != T_last:
                T = T_first + (T_last - T_first) * i / (n_sweeps - 1)
            t = lat.sweep_counter
            p = self.plan(t)
            def run(c0, c1, colours):
                nonlocal tot
                for colour in colours:
                    st = lat.run_colour_planes(colour, T, c0, c1)
                    tot += np.array([st["attempts"], st["unlike"], st["accepted"], st["sum_dE"]],
                                    dtype=np.int64)

            for half in (0, 1):
                colours = range(4 * half, 4 * half + 4)
                if self.world == 1:
                    run(p["c_lo"], p["c_hi"], colours)
                    continue
                lo, hi, nb = self._regions(p)
                before = (lat.get_planes(lo, nb, lat.planes_buffer(nb)),
                          lat.get_planes(hi, nb, lat.planes_buffer(nb)))
                if not self.overlap:
                    run(p["c_lo"], p["c_hi"], colours)
                    self._merge_boundaries(p, before)
                    continue
                bounds, inner = self._half_planes(p["c_lo"], p["c_hi"], half)
                for c0, c1 in bounds:
                    run(c0, c1, colours)
                self._merge_boundaries(p, before,
                                       (lambda: run(inner[0], inner[1], colours)) if inner else None)
            lat.sweep_counter = t + 1
            if self.world > 1:
                self._move(t)
        tot = self._allreduce(tot)
        return dict(attempts=int(tot[0]), unlike=int(tot[1]), accepted=int(tot[2]),
                    sum_dE=int(tot[3]))

    def gather(self):
        """Makes every rank's whole-lattice copy current everywhere (each rank
        broadcasts the planes it owns in the next sweep), so that occupancy,
        energy and SRO can be read on any rank."""
        if self.world == 1:
            return
        lat = self.lat
        t = lat.sweep_counter
        for src in range(self.world):
            p = self.plan(t, src)
            z0, nz = p["z_lo"], p["n_own"]
            if self.rank == src:
                buf = self._wire(lat.get_planes(z0, nz, lat.planes_buffer(nz)))
                lat.synchronize()
                self._dist.broadcast(buf, src=self._global(src), group=self.group)
            else:
                buf = self._wire_empty(nz)
                self._dist.broadcast(buf, src=self._global(src), group=self.group)
                self._after_comm()
                if not self.device_comm:
                    buf = self._to_lattice(buf, nz)
                lat.put_planes(z0, nz, buf)
        lat.synchronize()
