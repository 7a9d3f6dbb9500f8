"""Full-size parity: every workload at the size the benchmark runs it, in
the launch configuration it times, compared with the oracle on every row:
ids and distances element by element against the oracle's tree search
(Algorithms 2 and 3, whose answer the oracle's own pins tie to the plain
brute-force definition).  The oracle runs on the host cores; the dynamic
workload's rounds run in a spawn process pool."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CORES = len(os.sched_getaffinity(0))


@pytest.fixture(scope="module")
def zd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2111_04182_gb300 import zd as z

    return z


def test_clustered_10m_every_row(zd, oracle):
    """The headline workload (3D clustered, n = 10^7, L = 16, k = 10): the
    tree's sorted order and keys, and all 10^7 rows of ids and int64 squared
    distances equal the oracle's."""
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
    lo = e["leaf_lo"].cpu().numpy().astype(np.int64)
    t.free()
    ot = oracle.OracleTree(pts, w["leaf_size"], w["coord_bits"])
    oe = ot.export()
    assert np.array_equal(keys, oe["keys"]) and np.array_equal(ids, oe["ids"])
    # leaves: at most L points unless all keys equal
    big = np.nonzero(np.diff(lo) > w["leaf_size"])[0]
    assert np.all(keys[lo[big]] == keys[lo[big + 1] - 1])
    oi, od = ot.knn(w["k"], nthreads=CORES)
    I, D = idx.cpu().numpy(), d2.cpu().numpy()
    assert np.array_equal(I, oi)
    assert np.array_equal(D, od)


def test_uniform_10m_large_k_every_row(zd, oracle):
    """The large-k workload (3D uniform, n = 10^7, L = 16, k = 100) as the
    benchmark runs it: all rows equal the oracle's."""
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_3d_uniform()
    pts, k = w["pts"], w["k"]
    t = zd.zd_build(torch.from_numpy(pts).to(DEV), w["leaf_size"], w["coord_bits"])
    idx, d2 = t.knn(k)
    assert zd.zd_check() == 0
    t.free()
    oi, od = oracle.OracleTree(pts, w["leaf_size"], w["coord_bits"]).knn(k, nthreads=CORES)
    assert np.array_equal(idx.cpu().numpy(), oi)
    assert np.array_equal(d2.cpu().numpy(), od)


def test_dynamic_full_size_all_rounds(zd, oracle):
    """The dynamic workload at full size (5 * 10^7 points; 20 rounds of
    +10^6 inserted, -10^6 deleted, 10^6 bit-based queries with k = 5): after
    every round the live set matches, and all 10^6 query rows equal the
    oracle's search of the live set."""
    from paper_2111_04182_gb300 import datagen
    from tests import _oracle_pool
    w = datagen.DynamicWorkload()
    all_pts = np.empty((w.n0 + w.rounds * w.batch, 3), np.int32)
    all_pts[: w.n0] = w.initial
    t = zd.zd_build(torch.from_numpy(w.initial).to(DEV), w.leaf_size, w.coord_bits, capacity=w.n0 + w.batch)
    rounds, got, deleted = [], [], []
    for r in range(w.rounds):
        ins, dele, q = w.round()
        new = t.insert(torch.from_numpy(ins).to(DEV))
        t.delete(torch.from_numpy(dele).to(DEV))
        idx, d2 = t.knn(w.k, queries=torch.from_numpy(q).to(DEV), mode=zd.ZD_SEARCH_BIT)
        assert zd.zd_check() == 0
        new = new.cpu().numpy()
        assert np.array_equal(new, np.arange(w.n0 + r * w.batch, w.n0 + (r + 1) * w.batch))
        all_pts[new] = ins
        assert t.info()["n"] == len(w.live)
        deleted.append(dele)
        rounds.append((w.n0 + (r + 1) * w.batch, np.concatenate(deleted), q))
        got.append((idx.cpu().numpy(), d2.cpu().numpy()))
    t.free()
    want = _oracle_pool.dynamic_rounds(all_pts, rounds, w.leaf_size, w.coord_bits, w.k)
    for r, ((gi, gd), (oi, od)) in enumerate(zip(got, want)):
        assert np.array_equal(gi, oi), r
        assert np.array_equal(gd, od), r


def test_batched_full_size_every_cloud(zd, oracle):
    """The batched workload at full size (4096 clouds, 1.34 * 10^8 points,
    k = 16) with the leaf size the autotuner picks there (32), under both
    thread mappings: every cloud's rows equal the oracle's tree of that
    cloud."""
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_batched()
    off, pts, k = w["offsets"], w["pts"], w["k"]
    t = zd.zd_build_batched(torch.from_numpy(pts).to(DEV), off, 32, w["coord_bits"])
    res = [zd.zd_knn_batched(t, k, mapping=mp) for mp in (zd.ZD_KNN_THREAD_PER_QUERY, zd.ZD_KNN_WARP_GROUP)]
    assert zd.zd_check() == 0
    t.free()
    C = 256  # clouds per host copy
    for c0 in range(0, len(off) - 1, C):
        c1 = min(c0 + C, len(off) - 1)
        a, z = int(off[c0]), int(off[c1])
        host = [(i[a:z].cpu().numpy(), d[a:z].cpu().numpy()) for i, d in res]
        for c in range(c0, c1):
            ca, cz = int(off[c]) - a, int(off[c + 1]) - a
            oi, od = oracle.OracleTree(pts[a + ca:a + cz], 32, w["coord_bits"]).knn(k, nthreads=CORES)
            for m, (I, D) in enumerate(host):
                assert np.array_equal(I[ca:cz], oi), (c, m)
                assert np.array_equal(D[ca:cz], od), (c, m)


def test_differentiable_full_size(zd, oracle):
    """The differentiable workload at full size (64 pairs, A 16384, B 32768,
    k = 8), every pair: ids equal the oracle's root-based search (fp64
    ranking), the fp32 distances are within 1e-6 of the fp64 ones, and both
    gradients are within 1e-4 of the fp64 oracle per element,
    |g_i - g64_i| / max(|g64_i|, 1e-3)."""
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_differentiable()
    A = torch.from_numpy(w["A"]).to(DEV).requires_grad_(True)
    B = torch.from_numpy(w["B"]).to(DEV).requires_grad_(True)
    k = w["k"]
    dist, idx = zd.KnnDist.apply(A, B, k, w["leaf_size"], w["coord_bits"])
    dist.sum().backward()
    assert zd.zd_check() == 0
    I, Dg = idx.cpu().numpy(), dist.detach().cpu().numpy()
    GA, GB = A.grad.cpu().numpy().astype(np.float64), B.grad.cpu().numpy().astype(np.float64)
    worst = dict(dist=0.0, ga=0.0, gb=0.0)
    for p in range(len(w["A"])):
        lo, scale = oracle.quantization_of(w["B"][p], w["coord_bits"])
        ot = oracle.OracleTree(w["B"][p], w["leaf_size"], w["coord_bits"], qlo=lo, qscale=scale)
        oi, od = ot.knn(k, queries=w["A"][p], mode=oracle.MODE_ROOT, nthreads=len(os.sched_getaffinity(0)))
        assert np.array_equal(I[p], oi), p
        d64 = np.sqrt(od)
        worst["dist"] = max(worst["dist"], float(np.max(np.abs(Dg[p] - d64) / d64)))
        _, ga, gb = oracle.knn_dist_grad(w["A"][p], w["B"][p], oi)
        worst["ga"] = max(worst["ga"], float(np.max(np.abs(GA[p] - ga) / np.maximum(np.abs(ga), 1e-3))))
        worst["gb"] = max(worst["gb"], float(np.max(np.abs(GB[p] - gb) / np.maximum(np.abs(gb), 1e-3))))
    print("differentiable, all 64 pairs: max relative error vs fp64:", worst)
    assert worst["dist"] <= 1e-6 and worst["ga"] <= 1e-4 and worst["gb"] <= 1e-4, worst
