"""The point-by-point updater of small batches (csrc/local.cuh), built for the
host, against the oracle: after every insert or delete the tree in pointer
form has exactly the oracle's canonical dump of the current point set (the
reading of Sec. 2 "Batch-dynamic updates": the tree after an update equals
the canonical tree of the new set), with correct sizes, parents, tight boxes
and point locations.  No GPU needed."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("shim") / "liblocal_shim.so")
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", os.path.join(ROOT, "tests", "local_shim.cpp"),
                        "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    lib = C.CDLL(out)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    lib.lt_new.restype = vp
    lib.lt_new.argtypes = [i32, i32, i32, i64, i32, i32, i64]
    lib.lt_free.argtypes = [vp]
    lib.lt_insert.argtypes = [vp, vp, i64, i32]
    lib.lt_delete.argtypes = [vp, vp, i64]
    lib.lt_count.argtypes = [vp]
    lib.lt_export.restype = i64
    lib.lt_export.argtypes = [vp] + [vp] * 7
    return lib


class Tree:
    def __init__(self, lib, dim, L, B, cap=20000):
        self.lib, self.dim = lib, dim
        self.h = lib.lt_new(dim, L, B, cap, 4 * cap, 4 * cap, 64 * cap)

    def __del__(self):
        self.lib.lt_free(self.h)

    def insert(self, pts, first_id):
        pts = np.ascontiguousarray(pts, np.int32)
        return self.lib.lt_insert(self.h, pts.ctypes.data, len(pts), first_id)

    def delete(self, ids):
        ids = np.ascontiguousarray(ids, np.int32)
        return self.lib.lt_delete(self.h, ids.ctypes.data, len(ids))

    def dump(self, n):
        m = 2 * max(n, 1) + 2
        lo, hi = np.zeros(m, np.int64), np.zeros(m, np.int64)
        bit = np.zeros(m, np.int32)
        blo, bhi = np.zeros((m, 3), np.int32), np.zeros((m, 3), np.int32)
        ids, keys = np.zeros(max(n, 1), np.int32), np.zeros(max(n, 1), np.uint64)
        k = self.lib.lt_export(self.h, *[a.ctypes.data for a in (lo, hi, bit, blo, bhi, ids, keys)])
        assert k >= 0, "stored sizes, parents or point locations are inconsistent"
        order = np.lexsort((hi[:k], lo[:k]))
        return dict(lo=lo[:k][order], hi=hi[:k][order], bit=bit[:k][order], box_lo=blo[:k][order],
                    box_hi=bhi[:k][order], ids=ids[:n], keys=keys[:n])


def _same(t, oracle, pts, ids, L, B, dim):
    n = len(ids)
    got = t.dump(n)
    if n == 0:
        assert len(got["lo"]) == 0
        return
    want = oracle.OracleTree(pts, L, B, ids=ids).canonical_dump()
    for f in ("lo", "hi", "bit"):
        assert np.array_equal(got[f], want[f]), f
    assert np.array_equal(got["ids"], want["ids"])
    assert np.array_equal(got["keys"], want["keys"])
    assert np.array_equal(got["box_lo"][:, :dim], want["box_lo"])
    assert np.array_equal(got["box_hi"][:, :dim], want["box_hi"])


@pytest.mark.parametrize("dim,L,B", [(2, 1, 6), (2, 4, 8), (3, 3, 5), (3, 16, 10), (2, 16, 20)])
def test_small_updates_keep_the_canonical_tree(shim, oracle, dim, L, B):
    rng = np.random.default_rng(100 * dim + L)
    t = Tree(shim, dim, L, B)
    live_pts = np.zeros((0, dim), np.int32)
    live_ids = np.zeros(0, np.int32)
    next_id = 0
    pool = rng.integers(0, 2 ** B, size=(40, dim)).astype(np.int32)  # a source of duplicates
    for step in range(260):
        if len(live_ids) == 0 or rng.random() < 0.6:
            b = int(rng.integers(1, 6))
            if rng.random() < 0.3:
                new = pool[rng.integers(0, len(pool), size=b)]
            else:
                new = rng.integers(0, 2 ** B, size=(b, dim)).astype(np.int32)
            assert t.insert(new, next_id) == 0
            live_pts = np.concatenate([live_pts, new])
            live_ids = np.concatenate([live_ids, np.arange(next_id, next_id + b, dtype=np.int32)])
            next_id += b
        else:
            b = int(rng.integers(1, min(6, len(live_ids)) + 1))
            pick = rng.choice(len(live_ids), size=b, replace=False)
            assert t.delete(live_ids[pick]) == 0
            keep = np.ones(len(live_ids), bool)
            keep[pick] = False
            live_pts, live_ids = live_pts[keep], live_ids[keep]
        assert shim.lt_count(t.h) == len(live_ids)
        _same(t, oracle, live_pts, live_ids, L, B, dim)


def test_insert_then_delete_restores_and_empties(shim, oracle):
    rng = np.random.default_rng(7)
    t = Tree(shim, 3, 4, 12)
    base = rng.integers(0, 2 ** 12, size=(300, 3)).astype(np.int32)
    assert t.insert(base, 0) == 0
    d0 = t.dump(300)
    extra = rng.integers(0, 2 ** 12, size=(40, 3)).astype(np.int32)
    assert t.insert(extra, 300) == 0
    assert t.delete(np.arange(300, 340, dtype=np.int32)) == 0
    d1 = t.dump(300)
    for f in d0:
        assert np.array_equal(d0[f], d1[f]), f
    _same(t, oracle, base, np.arange(300, dtype=np.int32), 4, 12, 3)
    assert t.delete(rng.permutation(300).astype(np.int32)) == 0
    assert shim.lt_count(t.h) == 0 and len(t.dump(0)["lo"]) == 0
    # and the emptied tree grows again
    assert t.insert(base[:5], 400) == 0
    _same(t, oracle, base[:5], np.arange(400, 405, dtype=np.int32), 4, 12, 3)


def test_out_of_room_leaves_the_tree_unchanged(shim, oracle):
    """An insert or delete that could need more pool entries than are left
    reports it and changes nothing."""
    rng = np.random.default_rng(3)
    h = shim.lt_new(2, 2, 8, 100, 8, 8, 4000)
    try:
        pts = rng.integers(0, 256, size=(60, 2)).astype(np.int32)
        applied = 0
        for i in range(60):
            r = shim.lt_insert(h, pts[i:i + 1].ctypes.data, 1, i)
            if r != 0:
                break
            applied += 1
        assert r == 1 and 0 < applied < 60
        assert shim.lt_count(h) == applied
    finally:
        shim.lt_free(h)
