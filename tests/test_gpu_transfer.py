"""Occupancy transfers through the C ABI (gpu): the canonical -> device
layout conversion is checked byte for byte against the device layout
written out in numpy (codes sigma * W in rows [basis][z][y] of pitch px, or
two 4-bit ids per byte, zero padding), for rows whose length is a multiple
of 4 (the vector conversion) and for rows that are not (the scalar one);
the read-back returns the upload; and the asynchronous read-back holds the
occupancy of its point of the stream while a sweep and a pair count run
after it."""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs
from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu


def _width(K):
    return 8 if K <= 5 else (5 if K == 6 else 1)


def _expected_device(kind, n, K, occ, pack_bits, px):
    nb = 2 if kind == 0 else 4
    nx, ny, nz = n
    c = occ.reshape(nz, ny, nx, nb)  # canonical: basis fastest, then x, y, z
    if pack_bits == 8:
        dev = np.zeros((nb, nz, ny, px), np.uint8)
        dev[:, :, :, :nx] = np.moveaxis(c, 3, 0) * _width(K)
    else:
        dev = np.zeros((nb // 2, nz, ny, px), np.uint8)
        lo = np.moveaxis(c[..., 0::2], 3, 0)
        hi = np.moveaxis(c[..., 1::2], 3, 0)
        dev[:, :, :, :nx] = lo | (hi << 4)
    return dev.ravel()


@pytest.mark.parametrize("kind,n,K,pack_bits", [
    (0, (16, 12, 10), 5, 8),    # n_x % 4 == 0: vector conversion
    (0, (20, 9, 7), 6, 8),      # K = 6: codes sigma * 5
    (1, (12, 8, 9), 3, 8),
    (1, (8, 6, 5), 16, 4),      # packed, FCC
    (0, (24, 7, 6), 4, 4),      # packed, BCC
    (0, (13, 9, 8), 5, 8),      # n_x odd: scalar conversion
    (1, (10, 7, 6), 6, 8),
    (0, (7, 5, 9), 12, 4),
    (0, (16, 16, 16), 40, 8),   # K > 6: codes = ids
])
def test_upload_layout_and_round_trip(kind, n, K, pack_bits):
    torch = require_cuda()
    from paper_2509_20949_gb300.lattice import Lattice
    occ = inputs.initial_occupancy(kind, n, K, 11)
    lat = Lattice(kind, n, K, occ, seed=1, pack_bits=pack_bits)
    G = (2 if kind == 0 else 4) // (2 if pack_bits == 4 else 1)
    px = lat.d_occ.numel() // (G * n[1] * n[2])
    rng = np.random.default_rng(5)
    new = rng.integers(0, K, size=occ.size).astype(np.uint8)
    lat.set_occupancy(new)
    torch.cuda.synchronize()
    raw = lat.d_occ.cpu().numpy()[:G * n[1] * n[2] * px]
    want = _expected_device(kind, n, K, new, pack_bits, px)
    diff = np.flatnonzero(raw != want)
    assert diff.size == 0, f"{diff.size} device bytes differ, first at {diff[:4]}"
    assert np.array_equal(lat.occupancy(), new)
    lat.close()


def test_async_read_back_holds_its_point_of_the_stream():
    torch = require_cuda()
    from paper_2509_20949_gb300.lattice import Lattice
    kind, n, K, M = 0, (64, 60, 56), 5, 3
    occ = inputs.initial_occupancy(kind, n, K, 4)
    V = inputs.epi_table(M, K, 0.03, 2)
    lat = Lattice(kind, n, K, occ, seed=9)
    lat.set_epi(V)
    lat.sweep(2, 900.0)
    before = lat.occupancy()
    out = torch.empty(lat.N, dtype=torch.uint8, pin_memory=True).numpy()
    lat.occupancy_async(out)
    lat.sweep(3, 900.0)          # changes the lattice after the copy's point
    cnt, _ = lat.sro(M)          # reads it while the copy may still run
    lat.wait_occupancy()
    assert np.array_equal(out, before)
    after = lat.occupancy()
    assert not np.array_equal(after, before)
    # a second asynchronous copy, then an upload that reuses the transfer buffer
    out2 = torch.empty(lat.N, dtype=torch.uint8, pin_memory=True).numpy()
    lat.occupancy_async(out2)
    lat.set_occupancy(before)
    lat.wait_occupancy()
    assert np.array_equal(out2, after)
    assert np.array_equal(lat.occupancy(), before)
    assert lat.running_energy() == lat.energy()
    lat.wait_occupancy()  # nothing pending: returns at once
    lat.close()


def test_async_read_back_packed_and_invalid_upload_while_in_flight():
    """4-bit FCC storage; an upload with an id >= K, issued while a read-back
    is in flight, fails with EINVAL, leaves the lattice as it was and does
    not disturb the copy."""
    torch = require_cuda()
    from paper_2509_20949_gb300 import SmcxError, _lib
    from paper_2509_20949_gb300.lattice import Lattice
    kind, n, K, M = 1, (40, 36, 30), 4, 3
    occ = inputs.initial_occupancy(kind, n, K, 8)
    V = inputs.epi_table(M, K, 0.03, 6)
    lat = Lattice(kind, n, K, occ, seed=3, pack_bits=4)
    lat.set_epi(V)
    lat.sweep(2, 800.0)
    now = lat.occupancy()
    out = torch.empty(lat.N, dtype=torch.uint8, pin_memory=True).numpy()
    lat.occupancy_async(out)
    bad = now.copy()
    bad[123] = K
    with pytest.raises(SmcxError) as err:
        lat.set_occupancy(bad)
    assert err.value.status == _lib.SMCX_EINVAL
    lat.wait_occupancy()
    assert np.array_equal(out, now)
    assert np.array_equal(lat.occupancy(), now)
    assert lat.running_energy() == lat.energy()
    lat.close()
