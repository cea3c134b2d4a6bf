"""smcx_pair_counts_noalloc: pair counts for callers that cannot allocate
device memory (it keeps its counters in a static device array of the
library instead of a workspace).  Its counts must equal those of the
handle-based smcx_warren_cowley_sro exactly (integer counts: tolerance 0),
on two calls in a row that share the static array."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import gpu_lattice, make_case, require_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,n,K,M", [(0, (12, 10, 14), 5, 3), (1, (9, 8, 7), 4, 4)])
def test_noalloc_pair_counts_match_sro(kind, n, K, M):
    torch = require_cuda()
    from paper_2509_20949_gb300 import _lib
    L = _lib.lib()
    case = make_case(kind, n, K, M, seed=3, sigma=0.03)
    lat = gpu_lattice(case)
    stream = torch.cuda.current_stream()
    dims = (ctypes.c_uint32 * 3)(*n)
    for call in range(2):
        lat.sweep(2, 900.0)
        want, _ = lat.sro(M)                       # existing entry point
        occ = torch.from_numpy(lat.occupancy()).to("cuda")
        out = torch.full((M, K, K), -1, dtype=torch.int64, device="cuda")
        _lib.check(L.smcx_pair_counts_noalloc(kind, dims, K, M, ctypes.c_void_p(occ.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()),
                                              ctypes.c_void_p(stream.cuda_stream)))
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, want), f"call {call}"


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    require_cuda()
    from paper_2509_20949_gb300 import _lib
    L = _lib.lib()
    dims = (ctypes.c_uint32 * 3)(4, 4, 4)
    bogus = ctypes.c_void_p(16)  # never dereferenced: rejected before any launch
    assert L.smcx_pair_counts_noalloc(0, dims, 17, 2, bogus, bogus, None) == _lib.SMCX_EINVAL
    assert L.smcx_pair_counts_noalloc(0, dims, 4, 5, bogus, bogus, None) == _lib.SMCX_EINVAL
