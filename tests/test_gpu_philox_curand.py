"""Philox4x32-10 pinned to an implementation that is not ours: curand's
device generator (called, not copied), compared with the oracle's and the
library's device Philox on counters spanning all four words and keys."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe():
    require_cuda()
    d = tempfile.mkdtemp()
    so = os.path.join(d, "curand_probe.so")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", "-o", so, os.path.join(HERE, "curand_probe.cu")],
                   check=True)
    lib = ctypes.CDLL(so)
    lib.curand_philox_probe.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong,
                                        ctypes.c_ulonglong, ctypes.c_uint, ctypes.c_void_p]
    lib.curand_philox_probe.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("seed,subseq,offset4", [(0, 0, 0), (0x1234567890ABCDEF, 7 | (13 << 32), 3),
                                                 (2 ** 64 - 1, 2 ** 64 - 2, 2 ** 40 + 5)])
def test_oracle_and_library_philox_equal_curand(orc, probe, seed, subseq, offset4):
    torch = require_cuda()
    from paper_2509_20949_gb300 import _lib
    n = 512
    out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    assert probe.curand_philox_probe(seed, subseq, offset4, n, out.data_ptr()) == 0
    cur = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(0, n, 37):
        off = offset4 + i
        ctr = (off & 0xFFFFFFFF, (off >> 32) & 0xFFFFFFFF, subseq & 0xFFFFFFFF, subseq >> 32)
        assert list(orc.philox(ctr, key)) == list(cur[i]), i
    # the library's device generator on the same counters (word 0 advances)
    if (offset4 & 0xFFFFFFFF) + n < 2 ** 32:
        lib_out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
        _lib.check(_lib.lib().smcx_philox_device(offset4 & 0xFFFFFFFF, (offset4 >> 32) & 0xFFFFFFFF,
                                                 subseq & 0xFFFFFFFF, subseq >> 32, seed, n,
                                                 lib_out.data_ptr(), None))
        assert np.array_equal(lib_out.cpu().numpy().view(np.uint32).reshape(n, 4), cur)
