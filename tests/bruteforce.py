"""Independent brute-force references used to pin the oracle.

Nothing here reuses the oracle's displacement tables or neighbour routine:
lattice sites are generated from the conventional cell and its basis, bonds
are found by measuring Euclidean distances between a site and every periodic
image of every other site, and shells are identified by the textbook squared
distances in tests/golden/shells.json.
"""
import itertools
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

BASIS = {
    0: np.array([[0, 0, 0], [1, 1, 1]]),
    1: np.array([[0, 0, 0], [0, 1, 1], [1, 0, 1], [1, 1, 0]]),
}


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def shell_d2(kind, M):
    g = golden("shells.json")["bcc" if kind == 0 else "fcc"]
    return g["d2"][:M]


def positions(kind, n):
    """Site positions in half units, canonical order ((z*ny+y)*nx+x)*nb+b."""
    nx, ny, nz = n
    out = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for bv in BASIS[kind]:
                    out.append((2 * x + bv[0], 2 * y + bv[1], 2 * z + bv[2]))
    return np.array(out, dtype=np.int64)


def multiplicity(kind, n, M):
    """mult[m, i, j] = number of periodic images of site j at squared
    distance d2_m from site i (ordered pairs; i == j allowed)."""
    P = positions(kind, n)
    box = 2 * np.array(n, dtype=np.int64)
    d2s = shell_d2(kind, M)
    reach = int(np.ceil(np.sqrt(max(d2s))))
    rng = [range(-(reach // int(b)) - 1, (reach // int(b)) + 2) for b in box]
    diff = P[None, :, :] - P[:, None, :]  # [i, j, 3]
    N = len(P)
    mult = np.zeros((M, N, N), dtype=np.int64)
    for w in itertools.product(*rng):
        v = diff + (box * np.array(w))[None, None, :]
        d2 = (v * v).sum(-1)
        for m, target in enumerate(d2s):
            mult[m] += (d2 == target)
    return mult


def energy(kind, n, V, occ):
    """H = 1/2 sum_m sum_{i,j} mult_m(i,j) V_m(s_i, s_j) (exact integer)."""
    M = V.shape[0]
    mult = multiplicity(kind, n, M)
    occ = np.asarray(occ, dtype=np.int64)
    tot = 0
    for m in range(M):
        Vm = V[m][occ[:, None], occ[None, :]]
        tot += int((mult[m].astype(object) * Vm.astype(object)).sum())
    assert tot % 2 == 0
    return tot // 2


def pair_counts(kind, n, M, K, occ):
    mult = multiplicity(kind, n, M)
    occ = np.asarray(occ, dtype=np.int64)
    out = np.zeros((M, K, K), dtype=np.int64)
    for m in range(M):
        for pc in range(K):
            for p in range(K):
                out[m, pc, p] = mult[m][np.ix_(occ == pc, occ == p)].sum()
    return out


def binary_energies(kind, n, V, states):
    """Energies of many binary configurations at once.  states: [C, N] in
    {0,1}.  Uses the brute-force multiplicity matrices."""
    M = V.shape[0]
    mult = multiplicity(kind, n, M).astype(np.float64)
    x = states.astype(np.float64)
    y = 1.0 - x
    E = np.zeros(len(states), dtype=np.float64)
    exact = np.zeros(len(states), dtype=object)
    for m in range(M):
        A = mult[m]
        xx = np.einsum("ci,ij,cj->c", x, A, x)
        yy = np.einsum("ci,ij,cj->c", y, A, y)
        xy = np.einsum("ci,ij,cj->c", y, A, x)
        yx = np.einsum("ci,ij,cj->c", x, A, y)
        # counts are exact small integers in float64
        for c in range(len(states)):
            exact[c] += (int(round(yy[c])) * int(V[m, 0, 0]) + int(round(xx[c])) * int(V[m, 1, 1])
                         + (int(round(xy[c])) + int(round(yx[c]))) * int(V[m, 0, 1]))
    for c in range(len(states)):
        assert exact[c] % 2 == 0
        exact[c] //= 2
    return exact


def local_energies(kind, n, T, states):
    """Local-energy model E = sum_i sum_m sum_s T[m][s_i][s][c_{i,m,s}] of
    many configurations (states: [C, N] species ids), with the shell counts
    c_{i,m,s} = sum_j mult_m(i, j) [s_j = s] taken from the brute-force
    multiplicity matrices (every periodic image counted).  Exact integers."""
    M, K = T.shape[0], T.shape[1]
    states = np.atleast_2d(np.asarray(states, dtype=np.int64))
    mult = multiplicity(kind, n, M)
    onehot = (states[:, :, None] == np.arange(K)[None, None, :]).astype(np.int64)  # [C, N, K]
    out = np.zeros(len(states), dtype=object)
    for m in range(M):
        cnt = np.einsum("ij,cjk->cik", mult[m], onehot)  # [C, N, K]
        for s in range(K):
            vals = T[m][states, s, cnt[:, :, s]]  # [C, N]
            out += np.array([int(v) for v in vals.astype(object).sum(1)], dtype=object)
    return out
