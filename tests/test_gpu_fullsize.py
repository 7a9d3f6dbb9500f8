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


def test_uniform_10m_large_k_sampled(zd, oracle):
    """The large-k workload (3D uniform, n = 10^7, L = 16, k = 100) as the
    benchmark runs it: sampled rows exact against brute force over all
    points, properties on more rows."""
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_3d_uniform()
    pts, k = w["pts"], w["k"]
    n = len(pts)
    t = zd.zd_build(torch.from_numpy(pts).to(DEV), w["leaf_size"], w["coord_bits"])
    idx, d2 = t.knn(k)
    assert zd.zd_check() == 0
    rows = np.random.default_rng(3).choice(n, 20_000, replace=False)
    r_d = torch.from_numpy(rows).to(DEV)
    I, D = idx[r_d].cpu().numpy(), d2[r_d].cpu().numpy()
    assert np.all(I != rows[:, None]) and np.all(D[:, 1:] >= D[:, :-1])
    diff = pts[I].astype(np.int64) - pts[rows][:, None, :].astype(np.int64)
    assert np.array_equal((diff * diff).sum(-1), D)
    q = rows[:64]
    bi, bd = oracle.knn_brute(pts, k, queries=pts[q], query_ids=q.astype(np.int32))
    assert np.array_equal(I[:64], bi) and np.array_equal(D[:64], bd)
    t.free()


def test_dynamic_full_size_rounds(zd, oracle):
    """The dynamic workload at full size (5 * 10^7 points, batches of 10^6,
    k = 5, bit-based queries) for its first rounds: sampled queries of every
    round exact against brute force over the live set."""
    from paper_2111_04182_gb300 import datagen
    w = datagen.DynamicWorkload(rounds=3)
    all_pts = np.empty((w.n0 + 3 * w.batch, 3), np.int32)
    all_pts[: w.n0] = w.initial
    t = zd.zd_build(torch.from_numpy(w.initial).to(DEV), w.leaf_size, w.coord_bits, capacity=w.n0 + w.batch)
    rng = np.random.default_rng(7)
    for r in range(3):
        ins, dele, q = w.round()
        new = t.insert(torch.from_numpy(ins).to(DEV))
        t.delete(torch.from_numpy(dele).to(DEV))
        idx, d2 = t.knn(w.k, queries=torch.from_numpy(q).to(DEV), mode=zd.ZD_SEARCH_BIT)
        assert zd.zd_check() == 0
        all_pts[new.cpu().numpy()] = ins
        assert t.info()["n"] == len(w.live)
        sel = rng.choice(len(q), size=16, replace=False)
        live = w.live.astype(np.int64)
        bi, bd = oracle.knn_brute(all_pts[live], w.k, queries=q[sel], ref_ids=live.astype(np.int32))
        s_d = torch.from_numpy(sel).to(DEV)
        assert np.array_equal(idx[s_d].cpu().numpy(), bi), r
        assert np.array_equal(d2[s_d].cpu().numpy(), bd), r
    t.free()


@pytest.mark.parametrize("mapping", [0x100, 0x200])
def test_batched_full_size_sampled_clouds(zd, oracle, mapping):
    """The batched workload at full size (4096 clouds, 1.34 * 10^8 points,
    k = 16) with the leaf size the autotuner picks there (32): sampled clouds
    exact against the oracle's per-cloud trees."""
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_batched()
    off, pts, k = w["offsets"], w["pts"], w["k"]
    t = zd.zd_build_batched(torch.from_numpy(pts).to(DEV), off, 32, w["coord_bits"])
    idx, d2 = zd.zd_knn_batched(t, k, mapping=mapping)
    assert zd.zd_check() == 0
    for c in np.random.default_rng(4).choice(len(off) - 1, 6, replace=False).tolist() + [0, len(off) - 2]:
        a, z = int(off[c]), int(off[c + 1])
        oi, od = oracle.OracleTree(pts[a:z], 32, w["coord_bits"]).knn(k)
        assert np.array_equal(idx[a:z].cpu().numpy(), oi), c
        assert np.array_equal(d2[a:z].cpu().numpy(), od), c
    t.free()


def test_differentiable_full_size(zd, oracle):
    """The differentiable workload at full size (64 pairs, A 16384, B 32768,
    k = 8): sampled pairs' ids equal fp64 brute force and both gradients are
    within 1e-4 (relative to the largest component) of the fp64 oracle."""
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_differentiable()
    A = torch.from_numpy(w["A"]).to(DEV).requires_grad_(True)
    B = torch.from_numpy(w["B"]).to(DEV).requires_grad_(True)
    dist, idx = zd.KnnDist.apply(A, B, w["k"], w["leaf_size"], w["coord_bits"])
    dist.sum().backward()
    assert zd.zd_check() == 0
    rel = lambda g, g64: float(np.max(np.abs(g - g64)) / max(np.max(np.abs(g64)), 1e-3))
    for p in (0, 37, 63):
        bi, _ = oracle.knn_brute(w["B"][p], w["k"], queries=w["A"][p])
        assert np.array_equal(idx[p].cpu().numpy(), bi), p
        _, ga, gb = oracle.knn_dist_grad(w["A"][p], w["B"][p], bi)
        assert rel(A.grad[p].cpu().numpy(), ga) <= 1e-4, p
        assert rel(B.grad[p].cpu().numpy(), gb) <= 1e-4, p
