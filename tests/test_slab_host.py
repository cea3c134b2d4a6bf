"""Plan of the z decomposition (smcx_slab_plan / smcx_slab_transfer, pure host
code of libsmcx.so): each sweep's cell planes and owned planes partition the
lattice, the owned planes follow the oracle's moving link-cell grid (Sec. 2.2),
and the planes moved between sweeps are exactly owned(src, t) intersected
with window(dst, t + 1), checked by brute-force set arithmetic."""
import pytest

from paper_2509_20949_gb300 import SmcxError, slab
from paper_2509_20949_gb300.lattice import make_desc

CASES = [(0, (8, 8, 16), 3), (0, (6, 10, 13), 2), (1, (6, 6, 12), 3), (1, (5, 7, 23), 4),
         (0, (4, 4, 40), 1)]


def _owned(p, nz):
    return {(p["z_lo"] + k) % nz for k in range(p["n_own"])}


def _window(p, nz):
    return {(p["z_lo"] - p["halo"] + k) % nz for k in range(p["n_own"] + 2 * p["halo"])}


@pytest.mark.parametrize("kind,n,M", CASES)
def test_plans_partition_and_follow_the_moving_grid(orc, kind, n, M):
    d = make_desc(kind, n, 3, seed=11)
    od = orc.Desc(kind, n, 3, M, seed=11)
    L, m = orc.layout(od)
    mz = m[2]
    for world in range(1, mz // 2 + 1):
        for t in range(5):
            ps = [slab.plan(d, M, world, r, t) for r in range(world)]
            assert ps[0]["c_lo"] == 0 and ps[-1]["c_hi"] == mz
            for a, b in zip(ps, ps[1:]):
                assert a["c_hi"] == b["c_lo"]
            seen = []
            sz = orc.sweep_shift(od, t)[2]
            for p in ps:
                assert p["halo"] == L and p["m_z"] == mz
                assert p["c_hi"] - p["c_lo"] >= (2 if world > 1 else 1)
                assert p["z_lo"] == (sz + p["c_lo"] * n[2] // mz) % n[2]
                assert p["n_own"] == p["c_hi"] * n[2] // mz - p["c_lo"] * n[2] // mz
                seen += sorted(_owned(p, n[2]))
            assert sorted(seen) == list(range(n[2]))


@pytest.mark.parametrize("kind,n,M", CASES)
def test_transfers_are_owned_intersect_window(kind, n, M):
    d = make_desc(kind, n, 3, seed=5)
    mz = slab.plan(d, M, 1, 0, 0)["m_z"]
    nz = n[2]
    for world in range(2, mz // 2 + 1):
        for t in range(4):
            for dst in range(world):
                win = _window(slab.plan(d, M, world, dst, t + 1), nz)
                covered = set(_owned(slab.plan(d, M, world, dst, t), nz))
                for src in range(world):
                    runs = slab.transfer(d, M, world, src, dst, t)
                    got = []
                    for z0, k in runs:
                        assert 0 <= z0 < nz and 1 <= k <= nz
                        got += [(z0 + i) % nz for i in range(k)]
                    assert len(got) == len(set(got))
                    want = set() if src == dst else _owned(slab.plan(d, M, world, src, t), nz) & win
                    assert set(got) == want, (world, t, src, dst)
                    covered |= set(got)
                assert win <= covered  # every plane a rank reads next has a source


def test_plan_errors():
    d = make_desc(0, (8, 8, 16), 3)
    mz = slab.plan(d, 3, 1, 0, 0)["m_z"]
    for args in [(0, 0), (2, 2), (mz // 2 + 1, 0)]:
        with pytest.raises(SmcxError):
            slab.plan(d, 3, *args, 0)
    with pytest.raises(SmcxError):
        slab.plan(d, 5, 2, 0, 0)
    with pytest.raises(SmcxError):
        slab.transfer(d, 3, 2, 0, 2, 0)
