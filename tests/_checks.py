"""Independent checkers used by the tests (no code shared with the oracle or
the CUDA library).

* ``check_tree``   -- the invariants that characterise the canonical pruned
  zd-tree of Algorithm 1 (with the empty-cut pruning of Sec. 2.1) uniquely,
  given the sorted keys: any tree that passes them IS the canonical tree.
* ``brute_knn``    -- numpy brute-force k-NN ranked by (d^2, id).
* ``decode``       -- inverse of the Morton interleave of Sec. 1.1.
"""
from __future__ import annotations

import numpy as np


def hibit(x: int) -> int:
    return int(x).bit_length() - 1


def decode(key: int, dim: int, bits: int):
    """Inverse of the interleave: key bit d*b + (d-1-j) is bit b of coordinate j."""
    c = [0] * dim
    for b in range(bits):
        for j in range(dim):
            c[j] |= ((int(key) >> (dim * b + (dim - 1 - j))) & 1) << b
    return c


def check_tree(keys, lo, hi, bit, leaf_size, coords=None, box_lo=None, box_hi=None,
               left=None, right=None, parent=None, root=None):
    """Assert the canonical-tree invariants.  Nodes are given as parallel arrays
    (lo, hi, bit; bit < 0 marks a leaf), in any order.  With children/parent
    arrays the links are checked too; with coords/boxes the tight boxes are.
    Returns the tree depth."""
    keys = np.asarray(keys, np.uint64)
    n = len(keys)
    lo = np.asarray(lo, np.int64)
    hi = np.asarray(hi, np.int64)
    bit = np.asarray(bit, np.int64)
    assert np.all(keys[1:] >= keys[:-1]) if n > 1 else True, "keys not sorted"
    by_range = {}
    for v in range(len(lo)):
        key = (int(lo[v]), int(hi[v]))
        assert key not in by_range, "two nodes with the same range %s" % (key,)
        by_range[key] = v
    assert (0, n) in by_range, "no root covering [0, n)"
    # Walk from the root, reconstructing children from the split rule.
    depth = 0
    stack = [(0, n, 0)]
    seen = 0
    leaves = []
    while stack:
        a, z, dpt = stack.pop()
        v = by_range.get((a, z))
        assert v is not None, "missing node [%d,%d)" % (a, z)
        seen += 1
        depth = max(depth, dpt)
        all_equal = z - a == 0 or keys[a] == keys[z - 1]
        if bit[v] < 0:
            assert z - a <= leaf_size or all_equal, "leaf [%d,%d) too big" % (a, z)
            leaves.append((a, z))
            continue
        assert z - a > leaf_size and not all_equal, "internal node [%d,%d) should be a leaf" % (a, z)
        b = hibit(int(keys[a]) ^ int(keys[z - 1]))
        assert bit[v] == b, "node [%d,%d): bit %d, expected %d" % (a, z, bit[v], b)
        seg = keys[a:z]
        hb = (seg >> np.uint64(b)) & np.uint64(1)
        s = a + int(np.argmax(hb == 1))
        assert np.all(hb[: s - a] == 0) and np.all(hb[s - a:] == 1)
        above = seg >> np.uint64(b + 1) if b < 63 else np.zeros_like(seg)
        assert np.all(above == above[0]), "keys of a node differ above its split bit"
        if left is not None:
            lv, rv = by_range.get((a, s)), by_range.get((s, z))
            assert lv is not None and rv is not None
            assert int(left[v]) == lv and int(right[v]) == rv, "child links"
            assert int(parent[lv]) == v and int(parent[rv]) == v, "parent links"
            for c in (lv, rv):
                if bit[c] >= 0:
                    assert bit[c] < bit[v], "child bit must be below parent bit"
        stack.append((a, s, dpt + 1))
        stack.append((s, z, dpt + 1))
    assert seen == len(lo), "extra nodes not reachable from the root"
    leaves.sort()
    pos = 0
    for a, z in leaves:
        assert a == pos
        pos = z
    assert pos == n
    if root is not None:
        assert int(root) == by_range[(0, n)]
        if parent is not None:
            assert int(parent[int(root)]) < 0
    if coords is not None:
        coords = np.asarray(coords)
        for v in range(len(lo)):
            a, z = int(lo[v]), int(hi[v])
            if z > a:
                np.testing.assert_array_equal(np.asarray(box_lo[v]), coords[a:z].min(axis=0))
                np.testing.assert_array_equal(np.asarray(box_hi[v]), coords[a:z].max(axis=0))
    return depth


def brute_knn(ref, k, queries=None, ref_ids=None, query_ids=None):
    """numpy brute force: rank candidates by (d^2, id).  Integer inputs use
    int64 d^2; float inputs use float64 ((dx*dx + dy*dy) + dz*dz)."""
    ref = np.asarray(ref)
    n, dim = ref.shape
    is_float = ref.dtype.kind == "f"
    rid = np.arange(n) if ref_ids is None else np.asarray(ref_ids, np.int64)
    if queries is None:
        q = ref
        qid = rid
    else:
        q = np.asarray(queries)
        qid = None if query_ids is None else np.asarray(query_ids, np.int64)
    m = len(q)
    idx = np.full((m, k), -1, np.int32)
    d2 = np.full((m, k), np.inf if is_float else np.iinfo(np.int64).max,
                 np.float64 if is_float else np.int64)
    R = ref.astype(np.float64 if is_float else np.int64)
    for i in range(m):
        qi = q[i].astype(np.float64 if is_float else np.int64)
        diff = R - qi[None, :]
        sq = diff * diff
        dist = sq[:, 0].copy()
        for j in range(1, dim):
            dist = dist + sq[:, j]
        cand = np.ones(n, bool)
        if qid is not None:
            cand &= rid != qid[i]
        ci = np.nonzero(cand)[0]
        order = np.lexsort((rid[ci], dist[ci]))[:k]
        idx[i, : len(order)] = rid[ci][order]
        d2[i, : len(order)] = dist[ci][order]
    return idx, d2
