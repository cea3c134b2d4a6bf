"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds none of the method's arithmetic (no energies, no random
numbers of the sweep, no schedule): it only draws the problem instances both
sides consume.  The fitted FeCoNiAlTi interactions of the paper (Sec. 3) are
not published, so effective pair interactions are drawn from N(0, sigma) and
quantised to units of q = 2^-32 eV.

Recipes:
  epi_table           V_m(p, q) for p <= q ~ N(0, sigma_eV) from
                      numpy Generator(PCG64(seed)), drawn in the order
                      m -> p -> q >= p, quantised by rint(V * 2^32) (half-even),
                      mirrored to a symmetric int64 [M][K][K] table.
  composition_counts  equiatomic: floor(N/K) each, remainder to the lowest ids;
                      or fractions -> largest-remainder rounding, ties to the
                      lower id.
  dirichlet_fractions Dirichlet(alpha,...,alpha) from PCG64(seed).
  initial_occupancy   those exact counts at random sites (PCG64(seed)
                      shuffle up to 2^26 sites, i.i.d. draw + random
                      rebalancing above); canonical site order
                      ((z*ny + y)*nx + x)*nb + b.
"""
from __future__ import annotations

import math

import numpy as np

BCC, FCC = 0, 1
Q_PER_EV = float(2 ** 32)


def nb_of(kind: int) -> int:
    return 2 if kind == BCC else 4


def n_sites(kind: int, n) -> int:
    return nb_of(kind) * int(n[0]) * int(n[1]) * int(n[2])


def epi_table(n_shells: int, K: int, sigma_ev: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    V = np.zeros((n_shells, K, K), dtype=np.int64)
    for m in range(n_shells):
        for p in range(K):
            for q in range(p, K):
                v = rng.normal(0.0, sigma_ev)
                iv = int(np.rint(v * Q_PER_EV))
                V[m, p, q] = iv
                V[m, q, p] = iv
    return V


# coordination numbers of shells 1-3 (BCC 8, 6, 12; FCC 12, 6, 24)
_Z = {0: (8, 6, 12), 1: (12, 6, 24)}


def local_energy_table(kind: int, n_shells: int, K: int, sigma_ev: float, seed: int) -> np.ndarray:
    """Synthetic table of the local-energy model: T[m][a][s][c] = c V_m(a,s) / 2
    + U_m(a,s) c^2 / z_m (q units, [M][K][K][1 + max z_m]), V from epi_table
    and U ~ N(0, sigma/4) per (m, a, s) from the same seed: a pairwise part
    plus a term quadratic in each shell count, so the energy is a nonlinear
    function of the local order around every site."""
    z = _Z[kind][:n_shells]
    zt = 1 + max(z)
    V = epi_table(n_shells, K, sigma_ev, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    U = rng.normal(0.0, sigma_ev / 4.0, (n_shells, K, K))
    c = np.arange(zt, dtype=np.float64)
    T = np.zeros((n_shells, K, K, zt), dtype=np.int64)
    for m in range(n_shells):
        quad = U[m][:, :, None] * c[None, None, :] ** 2 / z[m]
        T[m] = (V[m][:, :, None] // 2) * np.arange(zt, dtype=np.int64)[None, None, :] + \
            np.rint(quad * Q_PER_EV).astype(np.int64)
    return T


def composition_counts(N: int, K: int, fractions=None) -> np.ndarray:
    if fractions is None:
        base = N // K
        counts = np.full(K, base, dtype=np.int64)
        counts[: N - base * K] += 1
        return counts
    f = np.asarray(fractions, dtype=np.float64)
    f = f / f.sum()
    raw = f * N
    counts = np.floor(raw).astype(np.int64)
    rem = N - int(counts.sum())
    frac = raw - counts
    # largest remainder first; ties go to the lower id (stable sort on -frac)
    order = np.argsort(-frac, kind="stable")
    counts[order[:rem]] += 1
    return counts


def dirichlet_fractions(K: int, alpha: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.dirichlet(np.full(K, float(alpha)))


def initial_occupancy(kind: int, n, K: int, seed: int, fractions=None) -> np.ndarray:
    """Exact composition counts at random positions.  Up to 2^26 sites: the
    species-sorted array shuffled by PCG64(seed).  Larger lattices (where a
    full shuffle takes minutes): species drawn i.i.d. with the target
    fractions, then the surplus sites of over-represented species, picked at
    random, are reassigned to under-represented ones until the counts are
    exact."""
    N = n_sites(kind, n)
    counts = composition_counts(N, K, fractions)
    rng = np.random.Generator(np.random.PCG64(seed))
    if N <= (1 << 26):
        occ = np.repeat(np.arange(K, dtype=np.uint8), counts)
        rng.shuffle(occ)
        return occ
    cum = np.cumsum(counts)
    occ = np.empty(N, dtype=np.uint8)
    chunk = 1 << 24
    for start in range(0, N, chunk):
        stop = min(N, start + chunk)
        if fractions is None:
            occ[start:stop] = rng.integers(0, K, stop - start, dtype=np.uint8)
        else:
            u = rng.integers(0, N, stop - start, dtype=np.int64)
            occ[start:stop] = np.searchsorted(cum, u, side="right").astype(np.uint8)
    have = np.bincount(occ, minlength=K).astype(np.int64)
    surplus = {s: int(have[s] - counts[s]) for s in range(K) if have[s] > counts[s]}
    deficit = [(s, int(counts[s] - have[s])) for s in range(K) if have[s] < counts[s]]
    pool = []
    for s, e in surplus.items():
        idx = np.flatnonzero(occ == s)
        pool.append(idx[rng.choice(len(idx), size=e, replace=False)])
    if pool:
        pool = np.concatenate(pool)
        rng.shuffle(pool)
        pos = 0
        for s, e in deficit:
            occ[pool[pos:pos + e]] = s
            pos += e
    return occ


# ---------------------------------------------------------------------------
# named workloads (the paper's alloy is FCC Fe29Co29Ni28Al7Ti7, Sec. 3; its
# fitted EPIs are missing, so these are synthetic stand-ins of its shapes)
# ---------------------------------------------------------------------------
def workload(name: str) -> dict:
    """Parameters of the named single-lattice workloads."""
    if name == "bcc16_k4":      # BCC 16^3 x2 = 8192 sites, 4 species, shells 1-2
        return dict(kind=BCC, n=(16, 16, 16), K=4, M=2, sigma=0.02, epi_seed=0, seed=0,
                    fractions=None, occ_seed=0, T_first=1000.0, T_last=1000.0, sweeps=100)
    if name == "fcc128_k5":     # FCC 128^3 x4 = 8.4M sites, Dirichlet(5), shells 1-4
        return dict(kind=FCC, n=(128, 128, 128), K=5, M=4, sigma=0.03, epi_seed=0, seed=0,
                    fractions=dirichlet_fractions(5, 5.0, 0), occ_seed=0, T_first=800.0,
                    T_last=800.0, sweeps=1000)
    if name == "bcc812_k5":     # BCC 812^3 x2 = 1.07e9 sites, 5 species, shells 1-3, anneal
        return dict(kind=BCC, n=(812, 812, 812), K=5, M=3, sigma=0.02, epi_seed=0, seed=0,
                    fractions=None, occ_seed=0, T_first=1200.0, T_last=600.0, sweeps=10000)
    if name == "fcc672_k5":     # the paper's production lattice: FCC 672x630x630 x4 = 1.07e9 sites,
        # Fe29Co29Ni28Al7Ti7 composition, 2000 -> 1000 K anneal (Sec. 3.2); synthetic EPIs, shells 1-4
        return dict(kind=FCC, n=(672, 630, 630), K=5, M=4, sigma=0.03, epi_seed=0, seed=0,
                    fractions=[0.29, 0.29, 0.28, 0.07, 0.07], occ_seed=0, T_first=2000.0,
                    T_last=1000.0, sweeps=3000000)
    if name == "bcc448_k5":     # the same recipe on 448^3 x2 = 1.8e8 sites (> L2): profiling case
        return dict(kind=BCC, n=(448, 448, 448), K=5, M=3, sigma=0.02, epi_seed=0, seed=0,
                    fractions=None, occ_seed=0, T_first=1200.0, T_last=600.0, sweeps=10000)
    raise KeyError(name)


def batch_jobs(n_jobs: int = 256, seed: int = 7, n_min: int = 8, n_max: int = 64,
               sweeps: int = 200) -> list:
    """Heterogeneous independent simulations: cubic n ~ round(exp(U(ln n_min,
    ln n_max))), BCC/FCC with p = 1/2, K ~ U{3..6} equiatomic, shells 1-3,
    sigma = 0.02 eV, EPI seed 1000 + job, T ~ U(300, 1500) K."""
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for j in range(n_jobs):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        kind = int(rng.integers(0, 2))
        K = int(rng.integers(3, 7))
        T = float(rng.uniform(300.0, 1500.0))
        jobs.append(dict(job=j, kind=kind, n=(n, n, n), K=K, M=3, sigma=0.02,
                         epi_seed=1000 + j, seed=1000 + j, occ_seed=1000 + j,
                         fractions=None, T_first=T, T_last=T, sweeps=sweeps))
    return jobs


def served_jobs(rate_per_s: float, window_s: float, seed: int, n_sites_min: float = 1e4,
                n_sites_max: float = 1e8, sweeps_min: int = 100, sweeps_max: int = 5000,
                max_jobs: int = 2000) -> list:
    """Poisson arrivals over a window; sites ~ log-U via a cubic n, BCC/FCC,
    K ~ U{3..6}, composition scans (Dirichlet(5) per job) or temperature
    scans, sweeps ~ log-U."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    jobs = []
    while len(jobs) < max_jobs:
        t += rng.exponential(1.0 / rate_per_s)
        if t > window_s:
            break
        kind = int(rng.integers(0, 2))
        nb = nb_of(kind)
        target = math.exp(rng.uniform(math.log(n_sites_min), math.log(n_sites_max)))
        n = max(4, int(round((target / nb) ** (1.0 / 3.0))))
        K = int(rng.integers(3, 7))
        sweeps = int(round(math.exp(rng.uniform(math.log(sweeps_min), math.log(sweeps_max)))))
        j = len(jobs)
        if rng.uniform() < 0.5:
            fractions = list(rng.dirichlet(np.full(K, 5.0)))
        else:
            fractions = None
        T = float(rng.uniform(300.0, 1500.0))
        jobs.append(dict(job=j, arrival_s=t, kind=kind, n=(n, n, n), K=K, M=3, sigma=0.02,
                         epi_seed=5000 + j, seed=5000 + j, occ_seed=5000 + j,
                         fractions=fractions, T=T, T_first=T, T_last=T, sweeps=sweeps))
    return jobs
