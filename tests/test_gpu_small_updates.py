"""Small update batches (at most ZD_SMALL_BATCH points: applied point by point
on the tree's pointer form by one device thread, no sync) against the
oracle: after every batch the tree -- re-derived into the flat layout by the
export -- equals the canonical tree of the current point set, k-NN answers
match, invalid batches change nothing, and mixing small and large batches
keeps both forms in step.  A leaf of equal keys that outgrows the slab room
sends later updates through the fallback log, which the re-derivation
replays."""
import numpy as np
import pytest

from tests.test_gpu_dynamic import _same_tree, _t

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


@pytest.mark.parametrize("dim,L,B", [(3, 16, 21), (2, 4, 12), (3, 1, 9)])
def test_small_batches_keep_the_canonical_tree(zd, oracle, dim, L, B):
    rng = np.random.default_rng(31 * dim + L)
    n0 = 6000
    pts = rng.integers(0, 2 ** (B - 1), size=(n0, dim)).astype(np.int32)
    t = zd.zd_build(_t(pts), L, B, capacity=n0 + 4000)
    oset = oracle.OracleSet(pts, L, B)
    q = rng.integers(0, 2 ** (B - 1), size=(300, dim)).astype(np.int32)
    for step in range(60):
        r = rng.random()
        if r < 0.45:
            b = int(rng.integers(1, zd.ZD_SMALL_BATCH + 1))
            ins = rng.integers(0, 2 ** (B - 1), size=(b, dim)).astype(np.int32)
            if step % 3 == 0:
                ins[: b // 2] = oset.pts[rng.integers(0, len(oset.pts), size=b // 2)]  # duplicates
            new = t.insert(_t(ins)).cpu().numpy()
            assert np.array_equal(new, oset.insert(ins))
        elif r < 0.9:
            b = int(rng.integers(1, zd.ZD_SMALL_BATCH + 1))
            dele = rng.choice(oset.ids, size=b, replace=False).astype(np.int32)
            t.delete(_t(dele))
            oset.delete(dele)
        else:  # a large batch in between: both forms must stay in step
            b = 200
            if rng.random() < 0.5:
                ins = rng.integers(0, 2 ** (B - 1), size=(b, dim)).astype(np.int32)
                assert np.array_equal(t.insert(_t(ins)).cpu().numpy(), oset.insert(ins))
            else:
                dele = rng.choice(oset.ids, size=b, replace=False).astype(np.int32)
                t.delete(_t(dele))
                oset.delete(dele)
        if step % 4 == 3 or step == 59:
            # queries first: after small batches, sparse queries (300 here)
            # search the pointer form; the export then re-derives the flat tree
            kk = (1, 5, 12, 32)[(step // 4) % 4]
            ot = oset.tree()
            for mode, omode in ((zd.ZD_SEARCH_BIT, oracle.MODE_BIT), (zd.ZD_SEARCH_ROOT, oracle.MODE_ROOT)):
                idx, d2 = t.knn(kk, queries=_t(q), mode=mode)
                oi, od = ot.knn(kk, queries=q, mode=omode)
                assert np.array_equal(idx.cpu().numpy(), oi), (step, mode)
                assert np.array_equal(d2.cpu().numpy(), od), (step, mode)
            assert zd.zd_check() == zd.ZD_OK
            _same_tree(t, oset)
            assert t.info()["n"] == len(oset.ids)
            idx, d2 = t.knn(5, queries=_t(q), mode=zd.ZD_SEARCH_BIT)  # the flat searches
            oi, od = ot.knn(5, queries=q, mode=oracle.MODE_BIT)
            assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
    # all points, each excluding itself, rows by id
    idx, d2 = t.knn(4)
    oi, od, oids = oset.tree().knn(4)  # rows in sorted order, with their ids
    rows = oids.astype(np.int64)
    assert np.array_equal(idx.cpu().numpy()[rows], oi) and np.array_equal(d2.cpu().numpy()[rows], od)
    t.free()


def test_small_batch_errors_change_nothing(zd, oracle):
    rng = np.random.default_rng(5)
    pts = rng.integers(0, 2 ** 16, size=(3000, 3)).astype(np.int32)
    t = zd.zd_build(_t(pts), 8, 21, capacity=4000)
    oset = oracle.OracleSet(pts, 8, 21)
    t.insert(_t(pts[:5] + 1))
    oset.insert(pts[:5] + 1)
    # a coordinate out of range: recorded, the batch does nothing (its ids are used up)
    bad = np.array([[1, 2, 3], [1 << 22, 0, 0]], np.int32)
    t.insert(_t(bad))
    assert zd.zd_check() == zd.ZD_ERR_RANGE
    oset.next_id += 2
    # unknown, dead and repeated ids: recorded, nothing deleted
    for ids in ([2, 999_999], [3, 3], [3000 + 5]):
        t.delete(_t(np.array(ids, np.int32)))
        assert zd.zd_check() in (zd.ZD_ERR_NOT_FOUND, zd.ZD_ERR_DUPLICATE_ID)
    _same_tree(t, oset)
    new = t.insert(_t(pts[10:12] * 0 + 7)).cpu().numpy()
    assert np.array_equal(new, oset.insert(pts[10:12] * 0 + 7))
    _same_tree(t, oset)
    assert zd.zd_check() == zd.ZD_OK
    t.free()


def test_equal_keys_past_the_slab_room_replay_exactly(zd, oracle):
    """A leaf of 2.5 million equal points: growing it past its slab needs more
    entries than the pointer form reserves, so the updater falls back and
    logs; the re-derivation replays the log through the flat update path and
    the tree is still the canonical one."""
    rng = np.random.default_rng(9)
    n_eq = 2_500_000
    pts = np.concatenate([np.full((n_eq, 3), 777, np.int32),
                          rng.integers(0, 2 ** 20, size=(5000, 3)).astype(np.int32)])
    t = zd.zd_build(_t(pts), 16, 21, capacity=len(pts) + 200)
    oset = oracle.OracleSet(pts, 16, 21)
    for i in range(5):
        ins = np.full((zd.ZD_SMALL_BATCH, 3), 777, np.int32)
        ins[-1] = rng.integers(0, 2 ** 20, size=3)
        assert np.array_equal(t.insert(_t(ins)).cpu().numpy(), oset.insert(ins))
        dele = rng.choice(oset.ids[n_eq:], size=3, replace=False).astype(np.int32)
        t.delete(_t(dele))
        oset.delete(dele)
    assert zd.zd_check() == zd.ZD_OK
    g = t.export()
    o = oset.tree().canonical_dump()
    assert np.array_equal(g["ids"].cpu().numpy(), o["ids"])
    assert np.array_equal(g["keys"].cpu().numpy().view(np.uint64), o["keys"])
    assert t.info()["n"] == len(oset.ids)
    # and small batches work again afterwards (a fresh pointer form)
    t.delete(_t(oset.ids[-2:].astype(np.int32)))
    oset.delete(oset.ids[-2:])
    assert t.info()["n"] == len(oset.ids)
    t.free()


def test_small_batches_on_an_empty_tree_with_a_shift(zd, oracle):
    """A 2D tree with a coordinate shift, started empty, grown and emptied by
    small batches only, up to exactly its capacity."""
    rng = np.random.default_rng(17)
    shift = [5, 1000]
    t = zd.zd_build(_t(np.zeros((0, 2), np.int32)), 4, 12, shift=shift, capacity=40)
    oset = oracle.OracleSet(np.zeros((0, 2), np.int32), 4, 12, shift=shift)
    for _ in range(5):
        ins = rng.integers(0, 2 ** 11, size=(8, 2)).astype(np.int32)
        assert np.array_equal(t.insert(_t(ins)).cpu().numpy(), oset.insert(ins))
        _same_tree(t, oset)
    with pytest.raises(zd.ZdError) as e:  # 40 points: the capacity is full
        t.insert(_t(np.zeros((1, 2), np.int32)))
    assert e.value.code == zd.ZD_ERR_CAPACITY
    while len(oset.ids):
        dele = oset.ids[: zd.ZD_SMALL_BATCH].astype(np.int32)
        t.delete(_t(dele))
        oset.delete(dele)
        assert zd.zd_check() == zd.ZD_OK
        assert t.info()["n"] == len(oset.ids)
        if len(oset.ids):
            _same_tree(t, oset)
    t.insert(_t(np.array([[1, 2]], np.int32)))
    oset.insert(np.array([[1, 2]], np.int32))
    _same_tree(t, oset)
    t.free()
