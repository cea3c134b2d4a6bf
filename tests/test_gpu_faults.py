"""Failure detection without a GPU fault: a device-side wait of the
persistent batch schedule is made to run out (the testing aid reports one more
work item for a job than it has, so the counter its next phase waits for is
never reached); the wait gives up after its limit, the run returns
SMCX_ETIMEOUT, the batch refuses further work, and the CUDA context stays
usable."""
import time

import numpy as np
import pytest

from tests.gpu_util import gpu_lattice, make_case, oracle_desc, require_cuda

pytestmark = pytest.mark.gpu


def test_device_wait_timeout_is_reported_and_context_survives(orc):
    require_cuda()
    from paper_2509_20949_gb300 import SmcxError, _lib
    from paper_2509_20949_gb300.batch import Batch
    case = make_case(0, (8, 8, 8), 3, 2, seed=3)
    b = Batch(4, 1 << 22, 1 << 14)
    for k in range(2):
        b.add(0, (8, 8, 8), 3, case["occ"], case["V"], 500.0 + 100 * k, 20, seed=k)
    b.set_option(Batch.OPT_SCHEDULE, 0)  # the persistent schedule (the one with device waits)
    b.set_option(Batch.OPT_TEST_WAIT_TIMEOUT, 1)
    t0 = time.perf_counter()
    with pytest.raises(SmcxError) as err:
        b.run(2)
    elapsed = time.perf_counter() - t0
    assert err.value.status == _lib.SMCX_ETIMEOUT
    assert 1.0 < elapsed < 60.0  # the ~2 s limit, not a hang
    with pytest.raises(SmcxError) as err:
        b.run(1)
    assert err.value.status == _lib.SMCX_ESTATE
    b.close()
    # the context is still usable: a lattice runs and matches the oracle
    lat = gpu_lattice(case)
    lat.sweep(3, 700.0)
    d = oracle_desc(orc, case)
    o_occ, _ = orc.sweeps(d, case["V"], case["occ"], 0, 3, 700.0)
    assert np.array_equal(lat.occupancy(), o_occ)
