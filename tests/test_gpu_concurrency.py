"""Searches of one tree from several streams at once.

Every k-NN search is a persistent launch whose warps take their work from
per-SM queues the call allocates for itself, and no warp waits for another,
so searches that run at the same time on different streams share the SMs
and still return exactly what they return alone.  Four searches that use the
four kernels (warp groups, one thread per query, one warp per query, warp
groups on external queries) run concurrently and are compared with the same
searches run one after another, and one of them with the oracle.
"""
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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_concurrent_searches_match_sequential_ones(zd, oracle):
    from paper_2111_04182_gb300 import datagen
    rng = np.random.default_rng(90)
    n = 200_000
    pts = datagen.clustered(rng, n, 3, n_clusters=40, bits=21, log2_sigma=(8, 12))
    t = zd.zd_build(_t(pts), 16, 21)
    q_sparse = _t(rng.integers(0, 2 ** 21, size=(30_000, 3)).astype(np.int32))  # 4m < n: one thread per query
    q_dense = _t(rng.integers(0, 2 ** 21, size=(100_000, 3)).astype(np.int32))  # 4m >= n: warp groups
    jobs = [dict(k=10, queries=None), dict(k=5, queries=q_sparse), dict(k=50, queries=None),
            dict(k=8, queries=q_dense)]

    def outs(j):
        rows = n if j["queries"] is None else j["queries"].shape[0]
        return (torch.empty((rows, j["k"]), dtype=torch.int32, device="cuda:0"),
                torch.empty((rows, j["k"]), dtype=torch.int64, device="cuda:0"))

    alone = []
    for j in jobs:  # one after another on the default stream
        o = outs(j)
        t.knn(j["k"], queries=j["queries"], out=o)
        alone.append(o)
    assert zd.zd_check() == zd.ZD_OK

    streams = [torch.cuda.Stream() for _ in jobs]
    together = [outs(j) for j in jobs]
    for s in streams:
        s.wait_stream(torch.cuda.current_stream())  # inputs and outputs are ready
    for _ in range(3):  # several rounds, all four in flight each time
        for j, s, o in zip(jobs, streams, together):
            with torch.cuda.stream(s):
                t.knn(j["k"], queries=j["queries"], out=o, stream=s)
    torch.cuda.synchronize()
    assert zd.zd_check() == zd.ZD_OK
    for j, a, b in zip(jobs, alone, together):
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), j["k"]
    oi, od = oracle.OracleTree(pts, 16, 21).knn(10)
    assert np.array_equal(together[0][0].cpu().numpy(), oi) and np.array_equal(together[0][1].cpu().numpy(), od)
    t.free()
