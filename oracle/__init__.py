"""Sequential CPU oracle of the SMC-X EPI swap sweep (arXiv 2509.20949).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library: the arithmetic lives in
``smcx_oracle.c`` (plain C, compiled with gcc, no fast-math, no FMA
contraction) and this module only marshals numpy arrays through ctypes.

Functions and the passages they follow:
  philox            Philox4x32-10, Salmon et al. SC11 (the RNG the method keys
                    by seed, sweep, cell and trial)
  shells            neighbour shells by brute-force distance classification
  layout            link-cell edge and counts (Sec. 2.2, Eq. 5)
  thresholds        Metropolis acceptance tables (Sec. 2.1, Eq. 3)
  energy            EPI Hamiltonian, pairwise only (Sec. 3, EPI model)
  delta_e           energy change of one swap from its local interaction zone
                    (Sec. 2.2)
  pair_counts /     directed shell pair counts and the Warren-Cowley SRO
  sro_alpha         (Sec. 3.2, Eq. 9)
  sweeps            full MC steps: one trial per site (Sec. 2.1) over the
                    checkerboard of link cells (Sec. 2.2)
  phase_cells       the trials of chosen cells of one colour phase
  sweeps_par /      the same with the cells of one colour shared out over
  phase_cells_par   OpenMP threads (cells of one colour never interact, so the
                    results are the sequential ones bit for bit)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smcx_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle_smcx.so")
_lock = threading.Lock()
_lib = None

FLAG_NO_SHIFT = 1
FLAG_SINGLE_CELL = 2
MODE_NORMAL, MODE_ACCEPT_ALL, MODE_ZERO_T = 0, 1, 2
BCC, FCC = 0, 1


class OracleError(RuntimeError):
    pass


class _Desc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("n", ctypes.c_int32 * 3),
        ("K", ctypes.c_int32),
        ("M", ctypes.c_int32),
        ("min_cell", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [
        ("attempts", ctypes.c_uint64),
        ("unlike", ctypes.c_uint64),
        ("accepted", ctypes.c_uint64),
        ("sum_dE", ctypes.c_int64),
    ]


class _Opts(ctypes.Structure):
    _fields_ = [
        ("L_override", ctypes.c_int32),
        ("shuffle_cells", ctypes.c_int32),
        ("shuffle_seed", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (idempotent)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    # the *_par functions share the cells of one colour out over OpenMP
    # threads; without OpenMP they run on one thread (same results)
    r = subprocess.run(cmd[:-4] + ["-fopenmp"] + cmd[-4:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.orc_philox.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            lib.orc_shells.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int),
                                       P(ctypes.c_int), ctypes.c_int]
            lib.orc_layout.argtypes = [P(_Desc), P(ctypes.c_int32), P(ctypes.c_int32)]
            lib.orc_thresholds.argtypes = [ctypes.c_double, P(ctypes.c_uint32), P(ctypes.c_int32),
                                           P(ctypes.c_int32)]
            lib.orc_energy.argtypes = [P(_Desc), P(ctypes.c_int64), P(ctypes.c_uint8),
                                       P(ctypes.c_int64)]
            lib.orc_pair_counts.argtypes = [P(_Desc), P(ctypes.c_uint8), P(ctypes.c_uint64)]
            lib.orc_sro_alpha.argtypes = [P(_Desc), P(ctypes.c_uint64), P(ctypes.c_uint64),
                                          P(ctypes.c_double)]
            lib.orc_delta_e.argtypes = [P(_Desc), P(ctypes.c_int64), P(ctypes.c_uint8),
                                        ctypes.c_int64, ctypes.c_int64, P(ctypes.c_int64)]
            lib.orc_sweeps.argtypes = [P(_Desc), P(ctypes.c_int64), P(ctypes.c_uint8),
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                       ctypes.c_double, P(_Stats), P(_Opts)]
            lib.orc_phase_cells.argtypes = [P(_Desc), P(ctypes.c_int64), P(ctypes.c_uint8),
                                            ctypes.c_uint32, ctypes.c_double, ctypes.c_int,
                                            P(ctypes.c_uint32), ctypes.c_uint32, P(_Stats)]
            lib.orc_sweep_shift.argtypes = [P(_Desc), ctypes.c_uint32, P(ctypes.c_int32)]
            lib.orc_phase_cells_par.argtypes = [P(_Desc), P(ctypes.c_int64), P(ctypes.c_uint8),
                                                ctypes.c_uint32, ctypes.c_double, ctypes.c_int,
                                                P(ctypes.c_uint32), ctypes.c_uint32, ctypes.c_int,
                                                P(_Stats)]
            lib.orc_sweeps_par.argtypes = [P(_Desc), P(ctypes.c_int64), P(ctypes.c_uint8),
                                           ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                           ctypes.c_double, P(_Stats), ctypes.c_int]
            lib.orc_max_threads.argtypes = []
            for name in ("orc_phase_cells_par", "orc_sweeps_par", "orc_max_threads"):
                getattr(lib, name).restype = ctypes.c_int
            lib.orc_exchange.argtypes = [ctypes.c_uint32, P(ctypes.c_int64), P(ctypes.c_double),
                                         ctypes.c_uint64, ctypes.c_uint32, P(ctypes.c_uint32),
                                         P(ctypes.c_uint8)]
            lib.orc_exchange.restype = ctypes.c_int
            lib.orc_profile.argtypes = [P(_Desc), P(ctypes.c_uint8), ctypes.c_int, P(ctypes.c_int32),
                                        ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        P(ctypes.c_uint64)]
            lib.orc_profile.restype = ctypes.c_int
            lib.orc_clusters.argtypes = [P(_Desc), P(ctypes.c_uint8), ctypes.c_uint32,
                                         P(ctypes.c_uint64), P(ctypes.c_uint64)]
            lib.orc_clusters.restype = ctypes.c_int
            lib.orc_local_width.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.orc_local_energy.argtypes = [P(_Desc), P(ctypes.c_int64), P(ctypes.c_uint8),
                                             P(ctypes.c_int64)]
            lib.orc_local_delta_e.argtypes = [P(_Desc), P(ctypes.c_int64), P(ctypes.c_uint8),
                                              ctypes.c_int64, ctypes.c_int64, P(ctypes.c_int64)]
            lib.orc_local_layout.argtypes = [P(_Desc), P(ctypes.c_int32), P(ctypes.c_int32)]
            lib.orc_local_sweeps.argtypes = [P(_Desc), P(ctypes.c_int64), P(ctypes.c_uint8),
                                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                             ctypes.c_double, P(_Stats), P(_Opts)]
            for name in ("orc_local_width", "orc_local_energy", "orc_local_delta_e",
                         "orc_local_layout", "orc_local_sweeps"):
                getattr(lib, name).restype = ctypes.c_int
            for name in ("orc_shells", "orc_layout", "orc_thresholds", "orc_energy",
                         "orc_pair_counts", "orc_sro_alpha", "orc_delta_e", "orc_sweeps",
                         "orc_phase_cells"):
                getattr(lib, name).restype = ctypes.c_int
            lib.orc_philox.restype = None
            lib.orc_sweep_shift.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(code: int, what: str):
    if code != 0:
        raise OracleError(f"oracle {what} failed with status {code}")


def nb_of(kind: int) -> int:
    return 2 if kind == BCC else 4


class Desc:
    """Lattice description: kind (0 BCC, 1 FCC), n = conventional cells per
    dimension (periodic), K species, M EPI shells, seed, flags, min_cell."""

    def __init__(self, kind, n, K, M, seed=0, flags=0, min_cell=0):
        self.kind, self.n, self.K, self.M = int(kind), tuple(int(v) for v in n), int(K), int(M)
        self.seed, self.flags, self.min_cell = int(seed), int(flags), int(min_cell)

    @property
    def n_sites(self) -> int:
        return nb_of(self.kind) * self.n[0] * self.n[1] * self.n[2]

    def c(self) -> _Desc:
        d = _Desc()
        d.kind = self.kind
        d.n[0], d.n[1], d.n[2] = self.n
        d.K, d.M, d.min_cell, d.flags, d.seed = self.K, self.M, self.min_cell, self.flags, self.seed
        return d


def philox(counter, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter and 2-word key -> 4 uint32."""
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def shells(kind: int, M: int):
    """Returns (disp [Z,3] int, z [M], d2 [M]) with shells in ascending
    distance and vectors sorted lexicographically inside a shell."""
    lib = _load()
    disp = np.zeros((128, 3), dtype=np.int32)
    z = np.zeros(M, dtype=np.int32)
    d2 = np.zeros(M, dtype=np.int32)
    tot = lib.orc_shells(kind, M, _ptr(disp, ctypes.c_int), _ptr(z, ctypes.c_int),
                         _ptr(d2, ctypes.c_int), 128)
    if tot < 0:
        raise OracleError("bad shell request")
    return disp[:tot].copy(), z, d2


def layout(desc: Desc):
    lib = _load()
    L = ctypes.c_int32()
    m = np.zeros(3, dtype=np.int32)
    _check(lib.orc_layout(ctypes.byref(desc.c()), ctypes.byref(L), _ptr(m, ctypes.c_int32)),
           "layout")
    return int(L.value), tuple(int(v) for v in m)


def thresholds(T: float):
    """-> (tables [3,512] uint32, s, mode)."""
    lib = _load()
    tab = np.zeros(3 * 512, dtype=np.uint32)
    s = ctypes.c_int32()
    mode = ctypes.c_int32()
    _check(lib.orc_thresholds(float(T), _ptr(tab, ctypes.c_uint32), ctypes.byref(s),
                              ctypes.byref(mode)), "thresholds")
    return tab.reshape(3, 512), int(s.value), int(mode.value)


def _occ(occ):
    a = np.ascontiguousarray(occ, dtype=np.uint8)
    return a


def _V(V):
    return np.ascontiguousarray(V, dtype=np.int64)


def energy(desc: Desc, V, occ) -> int:
    lib = _load()
    e = ctypes.c_int64()
    o, v = _occ(occ), _V(V)
    _check(lib.orc_energy(ctypes.byref(desc.c()), _ptr(v, ctypes.c_int64), _ptr(o, ctypes.c_uint8),
                          ctypes.byref(e)), "energy")
    return int(e.value)


def pair_counts(desc: Desc, occ) -> np.ndarray:
    lib = _load()
    o = _occ(occ)
    out = np.zeros((desc.M, desc.K, desc.K), dtype=np.uint64)
    _check(lib.orc_pair_counts(ctypes.byref(desc.c()), _ptr(o, ctypes.c_uint8),
                               _ptr(out, ctypes.c_uint64)), "pair_counts")
    return out


def sro_alpha(desc: Desc, counts, species_count) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    sc = np.ascontiguousarray(species_count, dtype=np.uint64)
    out = np.zeros((desc.M, desc.K, desc.K), dtype=np.float64)
    _check(lib.orc_sro_alpha(ctypes.byref(desc.c()), _ptr(c, ctypes.c_uint64),
                             _ptr(sc, ctypes.c_uint64), _ptr(out, ctypes.c_double)), "sro_alpha")
    return out


def delta_e(desc: Desc, V, occ, i: int, j: int) -> int:
    lib = _load()
    o, v = _occ(occ), _V(V)
    out = ctypes.c_int64()
    _check(lib.orc_delta_e(ctypes.byref(desc.c()), _ptr(v, ctypes.c_int64), _ptr(o, ctypes.c_uint8),
                           int(i), int(j), ctypes.byref(out)), "delta_e")
    return int(out.value)


STATS_DTYPE = np.dtype([("attempts", np.uint64), ("unlike", np.uint64), ("accepted", np.uint64),
                        ("sum_dE", np.int64)])


def sweeps(desc: Desc, V, occ, t0: int, n_sweeps: int, T_first: float, T_last=None,
           L_override: int = 0, shuffle_cells: bool = False, shuffle_seed: int = 0):
    """Runs n_sweeps MC steps in place on a copy of occ.
    Returns (occ_after, per_sweep_stats structured array)."""
    lib = _load()
    o = np.array(occ, dtype=np.uint8, copy=True, order="C")
    v = _V(V)
    stats = np.zeros(n_sweeps, dtype=STATS_DTYPE)
    opts = _Opts()
    opts.L_override, opts.shuffle_cells, opts.shuffle_seed = int(L_override), int(bool(shuffle_cells)), int(shuffle_seed)
    T_last = T_first if T_last is None else T_last
    code = lib.orc_sweeps(ctypes.byref(desc.c()), _ptr(v, ctypes.c_int64), _ptr(o, ctypes.c_uint8),
                          int(t0), int(n_sweeps), float(T_first), float(T_last),
                          stats.ctypes.data_as(ctypes.POINTER(_Stats)), ctypes.byref(opts))
    _check(code, "sweeps")
    return o, stats


def phase_cells(desc: Desc, V, occ, t: int, T: float, colour: int, cids, inplace=False):
    """Replays the trials of the listed cells (all of one colour) of sweep t.
    Returns (occ_after, stats dict)."""
    lib = _load()
    o = occ if inplace else np.array(occ, dtype=np.uint8, copy=True, order="C")
    if inplace and (o.dtype != np.uint8 or not o.flags.c_contiguous):
        raise OracleError("in-place replay needs a contiguous uint8 array")
    v = _V(V)
    c = np.ascontiguousarray(cids, dtype=np.uint32)
    st = _Stats()
    _check(lib.orc_phase_cells(ctypes.byref(desc.c()), _ptr(v, ctypes.c_int64),
                               _ptr(o, ctypes.c_uint8), int(t), float(T), int(colour),
                               _ptr(c, ctypes.c_uint32), len(c), ctypes.byref(st)), "phase_cells")
    return o, dict(attempts=st.attempts, unlike=st.unlike, accepted=st.accepted, sum_dE=st.sum_dE)


def max_threads() -> int:
    """Threads the *_par functions use by default (1 without OpenMP)."""
    return int(_load().orc_max_threads())


def phase_cells_par(desc: Desc, V, occ, t: int, T: float, colour: int, cids, n_threads=None,
                    inplace=False):
    """phase_cells with the cells shared out over n_threads OpenMP threads
    (cells of one colour never interact: same occupancy and statistics)."""
    lib = _load()
    o = occ if inplace else np.array(occ, dtype=np.uint8, copy=True, order="C")
    if inplace and (o.dtype != np.uint8 or not o.flags.c_contiguous):
        raise OracleError("in-place replay needs a contiguous uint8 array")
    v = _V(V)
    c = np.ascontiguousarray(cids, dtype=np.uint32)
    st = _Stats()
    nt = max_threads() if n_threads is None else int(n_threads)
    _check(lib.orc_phase_cells_par(ctypes.byref(desc.c()), _ptr(v, ctypes.c_int64),
                                   _ptr(o, ctypes.c_uint8), int(t), float(T), int(colour),
                                   _ptr(c, ctypes.c_uint32), len(c), nt, ctypes.byref(st)),
           "phase_cells_par")
    return o, dict(attempts=st.attempts, unlike=st.unlike, accepted=st.accepted, sum_dE=st.sum_dE)


def sweeps_par(desc: Desc, V, occ, t0: int, n_sweeps: int, T_first: float, T_last=None,
               n_threads=None):
    """sweeps with the cells of each colour shared out over n_threads OpenMP
    threads (same occupancy and per-sweep statistics)."""
    lib = _load()
    o = np.array(occ, dtype=np.uint8, copy=True, order="C")
    v = _V(V)
    stats = np.zeros(n_sweeps, dtype=STATS_DTYPE)
    T_last = T_first if T_last is None else T_last
    nt = max_threads() if n_threads is None else int(n_threads)
    code = lib.orc_sweeps_par(ctypes.byref(desc.c()), _ptr(v, ctypes.c_int64),
                              _ptr(o, ctypes.c_uint8), int(t0), int(n_sweeps), float(T_first),
                              float(T_last), stats.ctypes.data_as(ctypes.POINTER(_Stats)), nt)
    _check(code, "sweeps_par")
    return o, stats


def sweep_shift(desc: Desc, t: int):
    lib = _load()
    s = np.zeros(3, dtype=np.int32)
    lib.orc_sweep_shift(ctypes.byref(desc.c()), int(t), _ptr(s, ctypes.c_int32))
    return tuple(int(v) for v in s)


def species_counts(occ, K: int) -> np.ndarray:
    return np.bincount(np.asarray(occ, dtype=np.uint8).ravel(), minlength=K).astype(np.uint64)


def exchange(E, T, seed: int, rnd: int, perm):
    """Replica exchange round (Sec. 2.2, Eqs. 6-7): E[r] = energy of replica
    r (q units), T[k] = k-th temperature, perm[k] = replica at T[k].
    Returns (new perm, accepted flags per pair (k, k+1))."""
    lib = _load()
    n = len(T)
    e = np.ascontiguousarray(E, dtype=np.int64)
    t = np.ascontiguousarray(T, dtype=np.float64)
    p = np.ascontiguousarray(perm, dtype=np.uint32).copy()
    acc = np.zeros(n, dtype=np.uint8)
    _check(lib.orc_exchange(n, _ptr(e, ctypes.c_int64), _ptr(t, ctypes.c_double), int(seed),
                            int(rnd), _ptr(p, ctypes.c_uint32), _ptr(acc, ctypes.c_uint8)),
           "exchange")
    return p, acc[: n - 1].astype(bool)


def composition_profile(desc: Desc, occ, axis: int, origin_h, radius2_h: int, length_h: int,
                        n_bins: int) -> np.ndarray:
    """Species counts [n_bins][K] along a cylinder (atom-probe-like
    analysis, Sec. 3.2); positions in half lattice-constant units."""
    lib = _load()
    o = _occ(occ)
    org = np.ascontiguousarray(origin_h, dtype=np.int32)
    out = np.zeros((n_bins, desc.K), dtype=np.uint64)
    _check(lib.orc_profile(ctypes.byref(desc.c()), _ptr(o, ctypes.c_uint8), int(axis),
                           _ptr(org, ctypes.c_int32), int(radius2_h), int(length_h), int(n_bins),
                           _ptr(out, ctypes.c_uint64)), "profile")
    return out


def clusters(desc: Desc, occ, species) -> np.ndarray:
    """Sizes (descending) of the first-shell-connected clusters of the sites
    whose species is in `species` (precipitates, Sec. 3.2)."""
    lib = _load()
    o = _occ(occ)
    mask = 0
    for sp in species:
        mask |= 1 << int(sp)
    sizes = np.zeros(max(1, o.size), dtype=np.uint64)
    n = ctypes.c_uint64()
    _check(lib.orc_clusters(ctypes.byref(desc.c()), _ptr(o, ctypes.c_uint8), mask,
                            _ptr(sizes, ctypes.c_uint64), ctypes.byref(n)), "clusters")
    return sizes[: int(n.value)]


# ---- local-energy model (the nonlinear short-range model of Sec. 3) ---------

def local_width(kind: int, M: int) -> int:
    """Length zt of the count axis of a local-energy table: 1 + max z_m."""
    w = _load().orc_local_width(int(kind), int(M))
    if w < 0:
        raise OracleError("local_width: bad kind or M")
    return w


def _T(T):
    return np.ascontiguousarray(T, dtype=np.int64)


def local_energy(desc: Desc, T, occ) -> int:
    """E = sum_i sum_m sum_s T[m][s_i][s][c_{i,m,s}]."""
    lib = _load()
    t, o = _T(T), _occ(occ)
    e = ctypes.c_int64()
    _check(lib.orc_local_energy(ctypes.byref(desc.c()), _ptr(t, ctypes.c_int64),
                                _ptr(o, ctypes.c_uint8), ctypes.byref(e)), "local_energy")
    return int(e.value)


def local_delta_e(desc: Desc, T, occ, i: int, j: int) -> int:
    lib = _load()
    t, o = _T(T), _occ(occ)
    e = ctypes.c_int64()
    _check(lib.orc_local_delta_e(ctypes.byref(desc.c()), _ptr(t, ctypes.c_int64),
                                 _ptr(o, ctypes.c_uint8), int(i), int(j), ctypes.byref(e)),
           "local_delta_e")
    return int(e.value)


def local_layout(desc: Desc):
    lib = _load()
    L = ctypes.c_int32()
    m = np.zeros(3, dtype=np.int32)
    _check(lib.orc_local_layout(ctypes.byref(desc.c()), ctypes.byref(L), _ptr(m, ctypes.c_int32)),
           "local_layout")
    return int(L.value), tuple(int(v) for v in m)


def local_sweeps(desc: Desc, T, occ, t0: int, n_sweeps: int, T_first: float, T_last=None,
                 L_override: int = 0, shuffle_cells: bool = False, shuffle_seed: int = 0):
    """n_sweeps MC steps of the local-energy model on a copy of occ.
    Returns (occ_after, per_sweep_stats structured array)."""
    lib = _load()
    o = np.array(occ, dtype=np.uint8, copy=True, order="C")
    t = _T(T)
    stats = np.zeros(n_sweeps, dtype=STATS_DTYPE)
    opts = _Opts()
    opts.L_override, opts.shuffle_cells, opts.shuffle_seed = int(L_override), int(bool(shuffle_cells)), int(shuffle_seed)
    T_last = T_first if T_last is None else T_last
    code = lib.orc_local_sweeps(ctypes.byref(desc.c()), _ptr(t, ctypes.c_int64), _ptr(o, ctypes.c_uint8),
                                int(t0), int(n_sweeps), float(T_first), float(T_last),
                                stats.ctypes.data_as(ctypes.POINTER(_Stats)), ctypes.byref(opts))
    _check(code, "local_sweeps")
    return o, stats
