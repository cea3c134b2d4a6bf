"""The C-ABI library builds, loads and exports every entry point declared in
include/smcx.h; host-only entry points agree with the oracle (not gpu: no
kernel is launched)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2509_20949_gb300 import _lib
from paper_2509_20949_gb300.lattice import make_desc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(smcx_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def L():
    return _lib.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names <= set(_lib.SIGNATURES) | names  # all bound names are declared
    for n in _lib.SIGNATURES:
        assert n in names, f"binding for undeclared {n}"


def test_shell_tables_agree_with_oracle(L, orc):
    for kind in (0, 1):
        for M in (1, 2, 3, 4):
            disp = (ctypes.c_int32 * 192)()
            z = (ctypes.c_uint32 * 4)()
            tot = L.smcx_shell_table(kind, M, disp, 64, z)
            mine = np.frombuffer(disp, dtype=np.int32)[: 3 * tot].reshape(-1, 3)
            od, oz, _ = orc.shells(kind, M)
            assert np.array_equal(mine, od)
            assert list(z)[:M] == list(oz)


def test_host_philox_agrees_with_oracle(L, orc):
    rng = np.random.default_rng(3)
    for _ in range(200):
        c = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        k = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        out = (ctypes.c_uint32 * 4)()
        L.smcx_philox4x32_10((ctypes.c_uint32 * 4)(*c), (ctypes.c_uint32 * 2)(*k), out)
        assert list(out) == list(orc.philox(c, k))


def test_buffer_sizes_and_validation(L):
    d = make_desc(0, (16, 16, 16), 4)
    ob = L.smcx_occupancy_bytes(ctypes.byref(d))
    assert ob >= 8192 and ob % 16 == 0
    assert L.smcx_workspace_bytes(ctypes.byref(d)) >= 256 + 8192
    d4 = make_desc(0, (3, 3, 3), 4, pack_bits=4)
    assert 27 <= L.smcx_occupancy_bytes(ctypes.byref(d4)) and \
        L.smcx_occupancy_bytes(ctypes.byref(d4)) % 16 == 0
    for bad in (make_desc(2, (4, 4, 4), 4), make_desc(0, (0, 4, 4), 4), make_desc(0, (4, 4, 4), 0),
                make_desc(0, (4, 4, 4), 17, pack_bits=4), make_desc(0, (4, 4, 4), 4, pack_bits=2),
                make_desc(0, (2048, 2048, 1024), 4), make_desc(0, (4, 4, 4), 4, flags=64)):
        assert L.smcx_occupancy_bytes(ctypes.byref(bad)) == 0
        assert L.smcx_workspace_bytes(ctypes.byref(bad)) == 0
    # create with null buffers fails cleanly, without touching a device
    h = ctypes.c_void_p()
    occ = np.zeros(8192, dtype=np.uint8)
    st = L.smcx_create_lattice(ctypes.byref(d), None, None, occ.ctypes.data, None, ctypes.byref(h))
    assert st == _lib.SMCX_EINVAL and not h.value
    assert b"null" in L.smcx_last_error()


def test_batch_tile_shapes(L):
    """The batched kernel's work-item boxes hold one warp of cells each."""
    shapes = []
    for i in range(4):
        c = (ctypes.c_uint32 * 3)()
        assert L.smcx_batch_tile_shape(i, c) == _lib.SMCX_OK
        shapes.append(tuple(c))
        assert np.prod(shapes[-1]) == 32 and all(v & (v - 1) == 0 for v in shapes[-1])
    assert len(set(shapes)) == 4
    c = (ctypes.c_uint32 * 3)()
    assert L.smcx_batch_tile_shape(4, c) == _lib.SMCX_EINVAL
    # options of a null batch are refused without a device
    assert L.smcx_batch_set_option(None, 1, 0) == _lib.SMCX_EINVAL
    assert L.smcx_batch_tuning(None, None, None, None, None) == _lib.SMCX_EINVAL


def test_local_model_width_agrees_with_oracle(L, orc):
    for kind in (0, 1):
        for M in (1, 2, 3):
            assert L.smcx_local_model_width(kind, M) == orc.local_width(kind, M)
    assert L.smcx_local_model_width(0, 4) == 0 and L.smcx_local_model_width(2, 1) == 0
