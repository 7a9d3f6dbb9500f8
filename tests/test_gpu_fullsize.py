"""Full-size parity: the 3D clustered workload (n = 10,000,000, L = 16,
k = 10) in the launch configuration the benchmark times.  The oracle cannot
redo all 10^7 queries in seconds, so sampled rows are checked one by one
against brute force, and properties that hold at any size are checked on
every row."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def zd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2111_04182_gb300 import zd as z

    return z


def test_clustered_10m_sampled(zd, oracle):
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_3d_clustered()
    pts = w["pts"]
    n = len(pts)
    t = zd.zd_build(torch.from_numpy(pts).to(DEV), w["leaf_size"], w["coord_bits"])
    idx, d2 = t.knn(w["k"])
    assert zd.zd_check() == 0
    e = t.export()
    keys = e["keys"].cpu().numpy().view(np.uint64)
    ids = e["ids"].cpu().numpy()
    # sorted Morton order by (key, id); a permutation of all ids
    assert np.all(keys[1:] >= keys[:-1])
    tie = keys[1:] == keys[:-1]
    assert np.all(ids[1:][tie] > ids[:-1][tie])
    assert np.array_equal(np.sort(ids), np.arange(n))
    # keys equal the oracle's encoding of the points in that order (sampled)
    samp = np.random.default_rng(0).choice(n, 200_000, replace=False)
    assert np.array_equal(keys[samp], oracle.morton_keys(pts[ids[samp]], w["coord_bits"]))
    # leaves: at most L points unless all keys equal
    lo = e["leaf_lo"].cpu().numpy().astype(np.int64)
    sz = np.diff(lo)
    big = np.nonzero(sz > w["leaf_size"])[0]
    assert np.all(keys[lo[big]] == keys[lo[big + 1] - 1])
    # every row: ids distinct, not self, distances non-decreasing and exact
    I, D = idx.cpu().numpy(), d2.cpu().numpy()
    assert np.all(I != np.arange(n)[:, None])
    assert np.all(D[:, 1:] >= D[:, :-1])
    rows = np.random.default_rng(1).choice(n, 20_000, replace=False)
    diff = pts[I[rows]].astype(np.int64) - pts[rows][:, None, :].astype(np.int64)
    assert np.array_equal((diff * diff).sum(-1), D[rows])
    # sampled rows: exact against brute force over all 10^7 points
    q = np.random.default_rng(2).choice(n, 300, replace=False)
    bi, bd = oracle.knn_brute(pts, w["k"], queries=pts[q], query_ids=q.astype(np.int32))
    assert np.array_equal(I[q], bi) and np.array_equal(D[q], bd)
    t.free()
