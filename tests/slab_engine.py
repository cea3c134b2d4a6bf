"""A CPU stand-in for one rank's whole-lattice copy in the z decomposition
tests: the oracle's colour-phase replay on a canonical numpy occupancy, with
the plane calls SlabSweep makes (planes are whole canonical z slices here)."""
import numpy as np
import torch

from paper_2509_20949_gb300.lattice import make_desc


class OracleRankLattice:
    def __init__(self, orc, case):
        self.orc = orc
        self.d = orc.Desc(case["kind"], case["n"], case["K"], case["M"], seed=case["seed"],
                          flags=case["flags"], min_cell=case["min_cell"])
        self.desc = make_desc(case["kind"], case["n"], case["K"], min_cell=case["min_cell"],
                              flags=case["flags"], seed=case["seed"])
        self.M = case["M"]
        self.V = case["V"]
        self.occ = np.array(case["occ"], dtype=np.uint8, copy=True)
        n = case["n"]
        self.n = n
        self.plane = n[0] * n[1] * (2 if case["kind"] == 0 else 4)
        self.t = 0
        _, self.m = orc.layout(self.d)
        self.device = torch.device("cpu")

    @property
    def sweep_counter(self):
        return self.t

    @sweep_counter.setter
    def sweep_counter(self, t):
        self.t = int(t)

    def run_colour_planes(self, colour, T, c_lo, c_hi):
        mx, my, mz = self.m
        cids = [c for c in range(mx * my * mz)
                if ((c % mx) & 1) | (((c // mx) % my & 1) << 1) | (((c // (mx * my)) & 1) << 2) == colour
                and c_lo <= c // (mx * my) < c_hi]
        _, st = self.orc.phase_cells(self.d, self.V, self.occ, self.t, T, colour, cids, inplace=True)
        return st

    def _idx(self, z0, nz):
        zs = (np.arange(nz) + z0) % self.n[2]
        return (zs[:, None] * self.plane + np.arange(self.plane)[None, :]).ravel()

    def planes_buffer(self, nz):
        return torch.empty(nz * self.plane, dtype=torch.uint8)

    def get_planes(self, z0, nz, buf):
        buf.numpy()[:] = self.occ[self._idx(z0, nz)]
        return buf

    def put_planes(self, z0, nz, buf):
        self.occ[self._idx(z0, nz)] = buf.numpy()

    def merge_planes(self, z0, nz, theirs, before):
        i = self._idx(z0, nz)
        self.occ[i] ^= theirs.numpy() ^ before.numpy()

    def synchronize(self):
        pass
