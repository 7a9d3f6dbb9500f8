"""GPU parity of the large-k search (32 < k <= 128, one warp per query)
against the oracle: all points, bit- and root-based external queries, float
trees and forests, with duplicates, lattice ties and fewer points than k."""
import numpy as np
import pytest

from tests._checks import brute_knn

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

    assert z.zd_check() == 0
    return z


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("k,L", [(33, 16), (40, 16), (41, 8), (64, 16), (65, 4), (80, 16), (96, 8), (97, 16), (100, 16), (128, 33)])
def test_large_k_all_points(zd, oracle, dim, k, L):
    rng = np.random.default_rng(dim * 1000 + k)
    bits = 21 if dim == 3 else 20
    c = rng.integers(0, 2 ** 19, size=(9, dim))
    n = 30_011
    pts = np.clip(c[rng.integers(0, 9, n)] + rng.normal(0, 3000, (n, dim)), 0, 2 ** 19).astype(np.int32)
    pts[:500] = pts[500:1000]  # duplicates: ties at d^2 = 0
    pts[1000:1200] = pts[1000]  # a leaf of equal keys, larger than L
    t = zd.zd_build(_t(pts), L, bits)
    oi, od = oracle.OracleTree(pts, L, bits).knn(k)
    for mapping in (0, 0x100, 0x200):
        idx, d2 = t.knn(k, mapping=mapping)
        assert zd.zd_check() == 0
        assert np.array_equal(d2.cpu().numpy(), od), mapping
        assert np.array_equal(idx.cpu().numpy(), oi), mapping
    t.free()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("dim", [2, 3])
def test_large_k_external_queries(zd, oracle, mode, dim):
    rng = np.random.default_rng(mode * 7 + dim + 500)
    bits = 21 if dim == 3 else 20
    pts = rng.integers(0, 2 ** 20, size=(40_000, dim)).astype(np.int32)
    q = rng.integers(0, 2 ** 20, size=(5_003, dim)).astype(np.int32)
    q[:50] = pts[:50]
    t = zd.zd_build(_t(pts), 16, bits, shift=[3, 0, 17][:dim])
    for k, mapping in ((100, 0), (90, 0), (47, 0x100), (47, 0x200), (38, 0x100), (38, 0x200)):
        idx, d2 = t.knn(k, queries=_t(q), mode=mode, mapping=mapping)
        assert zd.zd_check() == 0
        oi, od = oracle.knn_brute(pts, k, queries=q)
        assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
    t.free()


def test_large_k_fewer_points_than_k(zd):
    for n, k, L in ((1, 33, 16), (2, 64, 1), (50, 100, 4), (129, 128, 16), (130, 128, 2), (97, 96, 200)):
        pts = np.random.default_rng(n).integers(0, 1000, size=(n, 3)).astype(np.int32)
        t = zd.zd_build(_t(pts), L, 21)
        idx, d2 = t.knn(k)
        bi, bd = brute_knn(pts, k)
        assert np.array_equal(idx.cpu().numpy(), bi) and np.array_equal(d2.cpu().numpy(), bd), (n, k)
        q = np.random.default_rng(n + 1).integers(0, 1000, size=(37, 3)).astype(np.int32)
        for mode in (1, 2):
            idx, d2 = t.knn(k, queries=_t(q), mode=mode)
            bi, bd = brute_knn(pts, k, queries=q)
            assert np.array_equal(idx.cpu().numpy(), bi) and np.array_equal(d2.cpu().numpy(), bd), (n, k, mode)
        t.free()
    assert zd.zd_check() == 0


def test_large_k_lattice_ties(zd, oracle):
    g = (np.stack(np.meshgrid(*[np.arange(16)] * 3, indexing="ij"), -1).reshape(-1, 3) * 5).astype(np.int32)
    oi, od = oracle.OracleTree(g, 16, 21).knn(90)
    for shift in (None, [5, 77, 1 << 19]):
        t = zd.zd_build(_t(g), 16, 21, shift=shift)
        idx, d2 = t.knn(90)
        assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
        t.free()


def test_large_k_float(zd, oracle):
    from paper_2111_04182_gb300 import datagen
    rng = np.random.default_rng(78)
    a, b = datagen.warped_pair(rng, 3000, 9000)
    t = zd.zd_build(_t(b), 16, 21)
    for mode in (1, 2):
        idx, dist = t.knn(96, queries=_t(a), mode=mode)
        bi, bd = oracle.knn_brute(b, 96, queries=a)
        assert np.array_equal(idx.cpu().numpy(), bi)
        assert np.allclose(dist.cpu().numpy(), np.sqrt(bd), rtol=1e-6, atol=0)
    idx, dist = t.knn(40)
    bi, bd = oracle.knn_brute(b, 40)
    assert np.array_equal(idx.cpu().numpy(), bi)
    assert np.allclose(dist.cpu().numpy(), np.sqrt(bd), rtol=1e-6, atol=0)
    t.free()
    assert zd.zd_check() == 0


def test_large_k_forest(zd, oracle):
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_batched(n_clouds=24, seed=9, size_range=(1, 5000))
    off = w["offsets"]
    pts = w["pts"]
    t = zd.zd_build_batched(_t(pts), off, 16, 16)
    idx, d2 = zd.zd_knn_batched(t, 70)
    assert zd.zd_check() == 0
    idx, d2 = idx.cpu().numpy(), d2.cpu().numpy()
    rng = np.random.default_rng(10)
    qs = [rng.integers(0, 2 ** 16, size=(int(rng.integers(0, 300)), 3)).astype(np.int32) for _ in range(24)]
    qoff = np.concatenate([[0], np.cumsum([len(q) for q in qs])]).astype(np.int64)
    qi, qd = zd.zd_knn_batched(t, 70, queries=_t(np.concatenate(qs)), query_offsets=qoff)
    assert zd.zd_check() == 0
    qi, qd = qi.cpu().numpy(), qd.cpu().numpy()
    for c in range(24):
        a, z = off[c], off[c + 1]
        if z == a:
            continue
        cloud = pts[a:z]
        oi, od = oracle.OracleTree(cloud, 16, 16).knn(70)
        assert np.array_equal(idx[a:z], oi) and np.array_equal(d2[a:z], od), c
        bi, bd = oracle.knn_brute(cloud, 70, queries=qs[c])
        assert np.array_equal(qi[qoff[c]:qoff[c + 1]], bi) and np.array_equal(qd[qoff[c]:qoff[c + 1]], bd), c
    t.free()


def test_k_above_limit_is_refused(zd):
    pts = np.random.default_rng(0).integers(0, 1000, size=(500, 3)).astype(np.int32)
    t = zd.zd_build(_t(pts), 16, 21)
    with pytest.raises(zd.ZdError) as e:
        t.knn(zd.ZD_MAX_K + 1)
    assert e.value.code == zd.ZD_ERR_UNIMPLEMENTED
    t.knn(zd.ZD_MAX_K)
    t.free()
    assert zd.zd_check() == 0
