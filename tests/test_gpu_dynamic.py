"""GPU batch insert / delete against the oracle: after every update the tree
equals the canonical tree of the current point set (sorted order, shape,
boxes) and k-NN answers match; insert-then-delete restores the tree."""
import numpy as np
import pytest

from tests._checks import check_tree
from tests._gpu import canonical, nodes_of

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


def _same_tree(t, oset):
    g = nodes_of(t.export())
    o = oset.tree().canonical_dump()
    assert np.array_equal(g["ids"], o["ids"])
    assert np.array_equal(g["keys"], o["keys"])
    c = canonical(g)
    for f in ("lo", "hi", "bit", "box_lo", "box_hi"):
        assert np.array_equal(c[f], o[f]), f
    coords = oset.pts[np.searchsorted(oset.ids, g["ids"])]
    check_tree(g["keys"], g["lo"], g["hi"], g["bit"], oset.leaf_size, coords=coords, box_lo=g["box_lo"],
               box_hi=g["box_hi"], left=g["left"], right=g["right"], parent=g["parent"], root=g["root"])
    return g


def test_insert_delete_rounds(zd, oracle):
    rng = np.random.default_rng(2)
    n0, b = 40_000, 3_000
    pts = rng.integers(0, 2 ** 20, size=(n0, 3)).astype(np.int32)
    t = zd.zd_build(_t(pts), 16, 21, capacity=n0 + 2 * b)
    oset = oracle.OracleSet(pts, 16, 21)
    d0 = canonical(nodes_of(t.export()))
    for rnd in range(4):
        ins = rng.integers(0, 2 ** 20, size=(b, 3)).astype(np.int32)
        ins[:10] = oset.pts[:10]  # duplicates of live points
        new = t.insert(_t(ins)).cpu().numpy()
        want = oset.insert(ins)
        assert np.array_equal(new, want)
        _same_tree(t, oset)
        dele = rng.choice(oset.ids, size=b, replace=False).astype(np.int32)
        t.delete(_t(dele))
        oset.delete(dele)
        _same_tree(t, oset)
        q = rng.integers(0, 2 ** 20, size=(5000, 3)).astype(np.int32)
        idx, d2 = t.knn(5, queries=_t(q))
        oi, od = oracle.knn_brute(oset.pts, 5, queries=q, ref_ids=oset.ids)
        assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
        # all-points rows are indexed by id
        ai, ad = t.knn(4)
        live = oset.ids
        bi, bd = oracle.knn_brute(oset.pts, 4, ref_ids=oset.ids)
        assert np.array_equal(ai.cpu().numpy()[live], bi) and np.array_equal(ad.cpu().numpy()[live], bd)
    assert zd.zd_check() == 0
    t.free()

    # insert then delete the same batch restores the original tree exactly
    t = zd.zd_build(_t(pts), 16, 21, capacity=n0 + b)
    new = t.insert(_t(rng.integers(0, 2 ** 20, size=(b, 3)).astype(np.int32)))
    t.delete(new)
    d1 = canonical(nodes_of(t.export()))
    for f in d0:
        assert np.array_equal(d0[f], d1[f]), f
    t.free()


def test_update_errors_leave_tree_unchanged(zd, oracle):
    """Invalid batches change nothing.  Batches of at most ZD_SMALL_BATCH
    points record their error for zd_check (they do not sync); larger ones
    validate on the host's side of a sync and return it."""
    rng = np.random.default_rng(5)
    pts = rng.integers(0, 2 ** 20, size=(5000, 3)).astype(np.int32)
    t = zd.zd_build(_t(pts), 8, 21, capacity=6000)
    for bad, code in (([1, 2, 99999], zd.ZD_ERR_NOT_FOUND), ([3, 4, 3], zd.ZD_ERR_DUPLICATE_ID),
                      ([-1], zd.ZD_ERR_NOT_FOUND)):
        t.delete(_t(np.array(bad, np.int32)))
        assert zd.zd_check() == code
        big = np.concatenate([np.array(bad, np.int32), np.arange(100, 120, dtype=np.int32)])
        with pytest.raises(zd.ZdError) as e:
            t.delete(_t(big))
        assert e.value.code == code
    t.delete(_t(np.array([10, 11], np.int32)))
    t.delete(_t(np.array([10], np.int32)))  # already deleted
    assert zd.zd_check() == zd.ZD_ERR_NOT_FOUND
    t.insert(_t(np.array([[2 ** 21, 0, 0]], np.int32)))  # out of range
    assert zd.zd_check() == zd.ZD_ERR_RANGE
    with pytest.raises(zd.ZdError) as e:
        t.insert(_t(np.concatenate([np.zeros((20, 3), np.int32), np.array([[2 ** 21, 0, 0]], np.int32)])))
    assert e.value.code == zd.ZD_ERR_RANGE
    with pytest.raises(zd.ZdError) as e:
        t.insert(_t(rng.integers(0, 100, size=(2000, 3)).astype(np.int32)))
    assert e.value.code == zd.ZD_ERR_CAPACITY
    oset = oracle.OracleSet(pts, 8, 21)
    oset.delete([10, 11])
    _same_tree(t, oset)
    assert t.info()["n"] == 4998
    # the all-points search reads the float copy of the points, which a
    # rejected large insert has to leave (or put back) as it was
    idx, d2 = t.knn(4)
    oi, od, oids = oset.tree().knn(4)  # rows in sorted order, with their ids
    rows = oids.astype(np.int64)
    assert np.array_equal(idx.cpu().numpy()[rows], oi) and np.array_equal(d2.cpu().numpy()[rows], od)
    assert zd.zd_check() == zd.ZD_OK
    t.free()
    assert zd.zd_check() == 0
