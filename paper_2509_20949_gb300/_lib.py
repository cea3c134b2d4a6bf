"""Build and ctypes binding of libsmcx.so (the C ABI in include/smcx.h).

Argument marshalling only: every step of the sweep, the pair counts and the
energies run in the library's CUDA kernels and C++ host code.  There is no
fallback: if the shared library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG_DIR)
CSRC = os.path.join(PKG_DIR, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG_DIR, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libsmcx.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "--expt-relaxed-constexpr"]

SMCX_OK, SMCX_EINVAL, SMCX_ENOMEM, SMCX_ECUDA, SMCX_EOVERFLOW, SMCX_ETIMEOUT, SMCX_ESTATE, \
    SMCX_EBUDGET = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EOVERFLOW", "ETIMEOUT", "ESTATE", "EBUDGET"]


class SmcxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"SMCX_{name}: {msg}")
        self.status = status


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    files = _sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC)
                          if f.endswith((".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "smcx.h"))
    return files


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles every .cu under csrc/ for sm_103a (in parallel) and links
    libsmcx.so into the package's _build directory."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        newest = max(os.path.getmtime(f) for f in _deps())
        if os.path.getmtime(LIB_PATH) >= newest:
            return LIB_PATH
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH_FLAGS, *NVCC_FLAGS, "-I", INCLUDE, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH_FLAGS, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class LatticeDesc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_uint32),
        ("n", ctypes.c_uint32 * 3),
        ("n_species", ctypes.c_uint32),
        ("pack_bits", ctypes.c_uint32),
        ("min_cell", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
    ]


class SweepStats(ctypes.Structure):
    _fields_ = [
        ("attempts", ctypes.c_uint64),
        ("unlike", ctypes.c_uint64),
        ("accepted", ctypes.c_uint64),
        ("sum_dE_q", ctypes.c_int64),
    ]

    def as_dict(self):
        return dict(attempts=self.attempts, unlike=self.unlike, accepted=self.accepted,
                    sum_dE=self.sum_dE_q)


class Slab(ctypes.Structure):
    """smcx_slab: one rank's part of a lattice decomposed along z in one sweep."""
    _fields_ = [
        ("c_lo", ctypes.c_int32),
        ("c_hi", ctypes.c_int32),
        ("z_lo", ctypes.c_int32),
        ("n_own", ctypes.c_int32),
        ("halo", ctypes.c_int32),
        ("m_z", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_P = ctypes.POINTER
_vp = ctypes.c_void_p
_st = ctypes.c_int

# name -> (restype, argtypes); the declarations of include/smcx.h
SIGNATURES = {
    "smcx_occupancy_bytes": (ctypes.c_size_t, [_P(LatticeDesc)]),
    "smcx_workspace_bytes": (ctypes.c_size_t, [_P(LatticeDesc)]),
    "smcx_create_lattice": (_st, [_P(LatticeDesc), _vp, _vp, _vp, _vp, _P(_vp)]),
    "smcx_set_epi": (_st, [_vp, ctypes.c_uint32, _vp]),
    "smcx_sweep": (_st, [_vp, ctypes.c_uint32, ctypes.c_double, ctypes.c_double, _P(SweepStats)]),
    "smcx_run_colour": (_st, [_vp, ctypes.c_uint32, ctypes.c_double, _P(SweepStats)]),
    "smcx_run_colour_planes": (_st, [_vp, ctypes.c_uint32, ctypes.c_double, ctypes.c_int32,
                                     ctypes.c_int32, _P(SweepStats)]),
    "smcx_slab_plan": (_st, [_P(LatticeDesc), ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                             ctypes.c_uint32, _P(Slab)]),
    "smcx_slab_transfer": (_st, [_P(LatticeDesc), ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                 _P(ctypes.c_int32), _P(ctypes.c_uint32)]),
    "smcx_local_model_width": (ctypes.c_uint32, [ctypes.c_uint32, ctypes.c_uint32]),
    "smcx_set_local_model": (_st, [_vp, ctypes.c_uint32, _vp]),
    "smcx_planes_bytes": (ctypes.c_size_t, [_vp, ctypes.c_uint32]),
    "smcx_get_planes": (_st, [_vp, ctypes.c_int32, ctypes.c_uint32, _vp]),
    "smcx_put_planes": (_st, [_vp, ctypes.c_int32, ctypes.c_uint32, _vp]),
    "smcx_merge_planes": (_st, [_vp, ctypes.c_int32, ctypes.c_uint32, _vp, _vp]),
    "smcx_energy": (_st, [_vp, _P(ctypes.c_int64)]),
    "smcx_running_energy": (_st, [_vp, _P(ctypes.c_int64)]),
    "smcx_warren_cowley_sro": (_st, [_vp, ctypes.c_uint32, _vp, _vp]),
    "smcx_get_occupancy": (_st, [_vp, _vp]),
    "smcx_get_occupancy_async": (_st, [_vp, _vp]),
    "smcx_wait_occupancy": (_st, [_vp]),
    "smcx_set_occupancy": (_st, [_vp, _vp]),
    "smcx_get_sweep_counter": (_st, [_vp, _P(ctypes.c_uint32)]),
    "smcx_set_sweep_counter": (_st, [_vp, ctypes.c_uint32]),
    "smcx_get_layout": (_st, [_vp, _P(ctypes.c_uint32), _P(ctypes.c_uint32)]),
    "smcx_checkpoint": (_st, [_vp, _vp, _P(ctypes.c_size_t)]),
    "smcx_restore": (_st, [_vp, _vp, ctypes.c_size_t]),
    "smcx_set_option": (_st, [_vp, ctypes.c_uint32, ctypes.c_int64]),
    "smcx_tile_shape_count": (ctypes.c_uint32, [ctypes.c_uint32]),
    "smcx_tile_shape": (_st, [ctypes.c_uint32, ctypes.c_uint32, _P(ctypes.c_uint32)]),
    "smcx_kernel_tuning": (_st, [_vp, _P(ctypes.c_uint32), _P(ctypes.c_uint32), _P(ctypes.c_uint32),
                                 _P(ctypes.c_int32), _P(ctypes.c_float)]),
    "smcx_composition_profile": (_st, [_vp, ctypes.c_uint32, _P(ctypes.c_int32), ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_uint32, _vp]),
    "smcx_clusters": (_st, [_vp, ctypes.c_uint32, _vp, ctypes.c_size_t, _P(ctypes.c_uint64), _vp,
                            ctypes.c_uint64]),
    "smcx_kernel_in_use": (_st, [_vp, _P(ctypes.c_uint32), _P(ctypes.c_int32)]),
    "smcx_destroy": (_st, [_vp]),
    "smcx_last_error": (ctypes.c_char_p, []),
    "smcx_shell_table": (ctypes.c_uint32, [ctypes.c_uint32, ctypes.c_uint32, _P(ctypes.c_int32),
                                           ctypes.c_uint32, _P(ctypes.c_uint32)]),
    "smcx_batch_control_bytes": (ctypes.c_size_t, [ctypes.c_uint32, ctypes.c_size_t]),
    "smcx_batch_job_bytes": (ctypes.c_size_t, [_P(LatticeDesc)]),
    "smcx_batch_create": (_st, [ctypes.c_uint32, _vp, ctypes.c_size_t, ctypes.c_size_t, _vp, _P(_vp)]),
    "smcx_batch_add": (_st, [_vp, _P(LatticeDesc), _vp, ctypes.c_uint32, _vp, ctypes.c_double,
                             ctypes.c_uint32, _P(ctypes.c_uint32)]),
    "smcx_batch_run": (_st, [_vp, ctypes.c_uint32, _P(ctypes.c_uint32)]),
    "smcx_batch_launch": (_st, [_vp, ctypes.c_uint32]),
    "smcx_batch_wait": (_st, [_vp, _P(ctypes.c_uint32)]),
    "smcx_batch_poll": (_st, [_vp, _P(ctypes.c_uint32), ctypes.c_uint32, _P(ctypes.c_uint32)]),
    "smcx_batch_result": (_st, [_vp, ctypes.c_uint32, _vp, _P(SweepStats), _P(ctypes.c_int64),
                                _P(ctypes.c_uint32)]),
    "smcx_batch_remove": (_st, [_vp, ctypes.c_uint32]),
    "smcx_batch_info": (_st, [_vp, _P(ctypes.c_uint32), _P(ctypes.c_uint32), _P(ctypes.c_size_t),
                              _P(ctypes.c_size_t)]),
    "smcx_batch_destroy": (_st, [_vp]),
    "smcx_batch_set_option": (_st, [_vp, ctypes.c_uint32, ctypes.c_int64]),
    "smcx_batch_tuning": (_st, [_vp, _P(ctypes.c_int32), _P(ctypes.c_int32), _P(ctypes.c_int32),
                                _P(ctypes.c_uint32)]),
    "smcx_batch_tile_shape": (_st, [ctypes.c_uint32, _P(ctypes.c_uint32)]),
    "smcx_batch_queue_stats": (_st, [_vp, _P(ctypes.c_uint64)]),
    "smcx_batch_exchange": (_st, [_vp, _P(ctypes.c_uint32), ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_uint32, _P(ctypes.c_uint32)]),
    "smcx_batch_temperature": (_st, [_vp, ctypes.c_uint32, _P(ctypes.c_double)]),
    "smcx_pair_counts_noalloc": (_st, [ctypes.c_uint32, _P(ctypes.c_uint32), ctypes.c_uint32,
                                       ctypes.c_uint32, _vp, _vp, _vp]),
    "smcx_philox4x32_10": (None, [_P(ctypes.c_uint32), _P(ctypes.c_uint32), _P(ctypes.c_uint32)]),
    "smcx_philox_device": (_st, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_uint64, ctypes.c_uint32, _vp, _vp]),
}

_lock = threading.Lock()
_lib = None


def lib(build_if_missing: bool = True):
    """The loaded libsmcx.so with typed entry points (raises if unavailable)."""
    global _lib
    with _lock:
        if _lib is None:
            path = build() if build_if_missing else LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(f"libsmcx.so not found at {path}")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int):
    if status != SMCX_OK:
        raise SmcxError(status, lib().smcx_last_error().decode())
