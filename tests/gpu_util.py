"""Helpers of the gpu tests: build both sides of a parity case from the same
seeded inputs.  The CUDA side is reached only through the C ABI (via the
ctypes binding); the oracle only through oracle/."""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs


def require_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu test run without a CUDA device")
    return torch


def make_case(kind, n, K, M, seed=0, sigma=0.03, epi_seed=1, occ_seed=17, fractions=None,
              flags=0, min_cell=0):
    V = inputs.epi_table(M, K, sigma, epi_seed)
    occ = inputs.initial_occupancy(kind, n, K, occ_seed, fractions)
    return dict(kind=kind, n=tuple(n), K=K, M=M, seed=seed, flags=flags, min_cell=min_cell,
                V=V, occ=occ)


def gpu_lattice(case, pack_bits=8, kernel=0):
    from paper_2509_20949_gb300.lattice import Lattice
    lat = Lattice(case["kind"], case["n"], case["K"], case["occ"], seed=case["seed"],
                  pack_bits=pack_bits, min_cell=case["min_cell"], flags=case["flags"])
    if kernel:
        lat.set_option(1, kernel)
    lat.set_epi(case["V"])
    return lat


def oracle_desc(orc, case):
    return orc.Desc(case["kind"], case["n"], case["K"], case["M"], seed=case["seed"],
                    flags=case["flags"], min_cell=case["min_cell"])


def write_region_sites(orc, desc, t, cids):
    """Canonical site indices of the conventional cells within one
    conventional cell of each listed link cell (the sites its trials can
    change), for sweep t's origin."""
    L, m = orc.layout(desc)
    shift = orc.sweep_shift(desc, t)
    nb = orc.nb_of(desc.kind)
    n = desc.n
    out = []
    for cid in cids:
        cid = int(cid)
        c = (cid % m[0], (cid // m[0]) % m[1], cid // (m[0] * m[1]))
        rng = []
        for d in range(3):
            lo = c[d] * n[d] // m[d]
            hi = (c[d] + 1) * n[d] // m[d]
            vals = sorted({(v + shift[d]) % n[d] for v in range(lo - 1, hi + 1)})
            rng.append(np.array(vals, dtype=np.int64))
        X, Y, Z = np.meshgrid(rng[0], rng[1], rng[2], indexing="ij")
        base = ((Z * n[1] + Y) * n[0] + X).ravel() * nb
        out.append((base[:, None] + np.arange(nb)[None, :]).ravel())
    return np.unique(np.concatenate(out)) if out else np.zeros(0, dtype=np.int64)


def colour_cells(orc, desc, colour):
    """Ascending ids of the link cells of one colour."""
    L, m = orc.layout(desc)
    axes = []
    for d in range(3):
        bit = (colour >> d) & 1
        if m[d] == 1:
            if bit:
                return np.zeros(0, dtype=np.uint32)
            axes.append(np.zeros(1, dtype=np.int64))
        else:
            axes.append(np.arange(bit, m[d], 2, dtype=np.int64))
    cid = (axes[2][:, None, None] * m[1] + axes[1][None, :, None]) * m[0] + axes[0][None, None, :]
    return cid.ravel().astype(np.uint32)
