"""Failure detection on the GPU without a fault: every device-side wait of the
library is bounded.  A wait on a flag that nothing sets gives up after its
limit, records ZD_ERR_TIMEOUT in the status word, and the context stays
usable for the next call.  Host-side failures (bad arguments, unknown or
repeated delete ids, capacity) return clean status codes."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2111_04182_gb300 import zd as z

    assert z.zd_check() == 0
    return z


def test_bounded_wait_times_out_and_context_survives(zd):
    t0 = time.time()
    zd.zd_selftest_wait_timeout(50)
    assert zd.zd_check() == zd.ZD_ERR_TIMEOUT
    assert time.time() - t0 < 10.0
    assert zd.zd_check() == zd.ZD_OK  # cleared
    keys = torch.from_numpy(np.random.default_rng(0).integers(0, 2 ** 40, 100_000, dtype=np.int64)).cuda()
    sk, perm = zd.zd_morton_sort(keys, 40)
    assert zd.zd_check() == zd.ZD_OK
    assert torch.equal(sk, torch.sort(keys).values)


def test_host_checked_errors(zd):
    pts = torch.zeros((10, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(zd.ZdError) as e:
        zd.zd_build(pts, 0, 21)  # leaf size 0
    assert e.value.code == zd.ZD_ERR_INVALID_ARG
    with pytest.raises(zd.ZdError) as e:
        zd.zd_build(pts, 16, 22)  # 3D keys need B <= 21
    assert e.value.code == zd.ZD_ERR_INVALID_ARG
    t = zd.zd_build(pts, 16, 21)
    with pytest.raises(zd.ZdError) as e:
        t.knn(zd.ZD_MAX_K + 1)
    assert e.value.code == zd.ZD_ERR_UNIMPLEMENTED
    with pytest.raises(zd.ZdError):
        zd.zd_selftest_wait_timeout(0)
    t.free()
    assert zd.zd_check() == zd.ZD_OK


def test_non_finite_float_coordinates_are_range_errors(zd):
    pts = np.random.default_rng(3).standard_normal((1000, 3)).astype(np.float32)
    for bad in (np.nan, np.inf, -np.inf, 3e18):
        p = pts.copy()
        p[17, 1] = bad
        t = zd.zd_build(torch.from_numpy(p).cuda(), 16, 21)
        assert zd.zd_check() == zd.ZD_ERR_RANGE, bad
        t.free()
    t = zd.zd_build(torch.from_numpy(pts).cuda(), 16, 21)
    q = pts[:10].copy()
    q[3, 0] = np.nan
    t.knn(4, queries=torch.from_numpy(q).cuda())
    assert zd.zd_check() == zd.ZD_ERR_RANGE
    t.free()
    assert zd.zd_check() == zd.ZD_OK
