"""smcx_pair_counts_noalloc: pair counts for callers that cannot allocate
device memory where they need them -- code running inside another
framework's memory-pool callbacks or allocator hooks (a nested allocation
would recurse or deadlock), processes whose device memory is wholly reserved
by their host framework, deployments that forbid allocation after start-up.
It keeps its counters in a static device array of the library instead of a
workspace.  Its counts must equal the oracle's and those of the handle-based
smcx_warren_cowley_sro exactly (integer counts: tolerance 0), on two calls in
a row that share the static array; ids >= n_species in the buffer are left
out of the counts."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import gpu_lattice, make_case, oracle_desc, require_cuda

pytestmark = pytest.mark.gpu


def _noalloc(L, torch, kind, n, K, M, occ_host, stream):
    from paper_2509_20949_gb300 import _lib
    occ = torch.from_numpy(np.ascontiguousarray(occ_host)).to("cuda")
    out = torch.full((M, K, K), -1, dtype=torch.int64, device="cuda")
    dims = (ctypes.c_uint32 * 3)(*n)
    _lib.check(L.smcx_pair_counts_noalloc(kind, dims, K, M, ctypes.c_void_p(occ.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream)))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.uint64)


@pytest.mark.parametrize("kind,n,K,M", [(0, (12, 10, 14), 5, 3), (1, (9, 8, 7), 4, 4)])
def test_noalloc_pair_counts_match_oracle_and_sro(orc, kind, n, K, M):
    torch = require_cuda()
    from paper_2509_20949_gb300 import _lib
    L = _lib.lib()
    case = make_case(kind, n, K, M, seed=3, sigma=0.03)
    lat = gpu_lattice(case)
    d = oracle_desc(orc, case)
    stream = torch.cuda.current_stream()
    for call in range(2):
        lat.sweep(2, 900.0)
        occ = lat.occupancy()
        want = orc.pair_counts(d, occ)             # the oracle
        sro, _ = lat.sro(M)                         # the existing entry point
        got = _noalloc(L, torch, kind, n, K, M, occ, stream)
        assert np.array_equal(got, want), f"call {call}"
        assert np.array_equal(got, sro), f"call {call}"


def test_noalloc_leaves_out_ids_beyond_n_species(orc):
    """A buffer holding ids 0..K+1 counted as K species: the counts are the
    oracle's counts of the same buffer read as K + 2 species, restricted to
    the first K (pairs with a larger id on either side drop out)."""
    torch = require_cuda()
    from paper_2509_20949_gb300 import _lib
    from paper_2509_20949_gb300 import inputs
    L = _lib.lib()
    kind, n, K, M = 0, (10, 9, 11), 3, 3
    occ = inputs.initial_occupancy(kind, n, K + 2, 5)
    full = orc.pair_counts(orc.Desc(kind, n, K + 2, M), occ)
    stream = torch.cuda.current_stream()
    for call in range(2):
        got = _noalloc(L, torch, kind, n, K, M, occ, stream)
        assert np.array_equal(got, full[:, :K, :K]), f"call {call}"


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    require_cuda()
    from paper_2509_20949_gb300 import _lib
    L = _lib.lib()
    dims = (ctypes.c_uint32 * 3)(4, 4, 4)
    bogus = ctypes.c_void_p(16)  # never dereferenced: rejected before any launch
    assert L.smcx_pair_counts_noalloc(0, dims, 17, 2, bogus, bogus, None) == _lib.SMCX_EINVAL
    assert L.smcx_pair_counts_noalloc(0, dims, 4, 5, bogus, bogus, None) == _lib.SMCX_EINVAL
