"""Pins of the CPU oracle against what the paper and mathematics fix.

Every check here is independent of the oracle's own code: hand-derived
fixtures (tests/golden), closed forms, invariants that characterise the
canonical tree, brute force in numpy, library routines (numpy.lexsort) and
finite differences.  None needs a GPU.
"""
import json
import os

import numpy as np
import pytest

from tests._checks import brute_knn, check_tree, decode

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))
I64MAX = np.iinfo(np.int64).max


# ---------------------------------------------------------------- Morton keys
@pytest.mark.parametrize("case", GOLD["morton"]["cases"], ids=lambda c: "%dd-%s" % (c["dim"], c["pt"]))
def test_morton_hand_values(oracle, case):
    pts = np.array([case["pt"]], np.int64)
    if case["pt"] and max(case["pt"]) >= 2 ** 31:
        pytest.skip("not an int32 point")
    keys = oracle.morton_keys(pts.astype(np.int32), case["bits"], case["shift"])
    assert int(keys[0]) == int(case["key"])


def test_morton_roundtrip_and_monotone(oracle):
    rng = np.random.default_rng(11)
    for dim, bits in ((2, 20), (3, 21), (2, 31), (3, 5)):
        pts = rng.integers(0, 2 ** bits, size=(2000, dim)).astype(np.int32)
        keys = oracle.morton_keys(pts, bits)
        for i in range(0, 2000, 7):
            assert decode(int(keys[i]), dim, bits) == list(map(int, pts[i]))
        # box property (Sec. 1.1): every point of the box spanned by lo and hi
        # lies between them in Morton order.
        a = rng.integers(0, 2 ** bits, size=(3000, dim))
        b = rng.integers(0, 2 ** bits, size=(3000, dim))
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        r = lo + (rng.random((3000, dim)) * (hi - lo + 1)).astype(np.int64)
        r = np.minimum(r, hi)
        kl = oracle.morton_keys(lo.astype(np.int32), bits)
        kh = oracle.morton_keys(hi.astype(np.int32), bits)
        kr = oracle.morton_keys(r.astype(np.int32), bits)
        assert np.all(kl <= kr) and np.all(kr <= kh)


def test_morton_z_order_of_unit_square(oracle):
    # Level-1 Z pattern: (0,0) (0,1) (1,0) (1,1) with x most significant.
    pts = np.array([[0, 0], [0, 1], [1, 0], [1, 1]], np.int32)
    assert list(oracle.morton_keys(pts, 1)) == [0, 1, 2, 3]


def test_morton_range_errors(oracle):
    with pytest.raises(oracle.OracleError) as e:
        oracle.morton_keys(np.array([[4, 0]], np.int32), 2)
    assert e.value.code == oracle.ERR_RANGE
    with pytest.raises(oracle.OracleError):
        oracle.morton_keys(np.array([[-1, 0, 0]], np.int32), 21)
    with pytest.raises(oracle.OracleError):
        oracle.morton_keys(np.array([[3, 0]], np.int32), 2, shift=[1, 0])


# ----------------------------------------------------------------------- sort
def test_sort_matches_lexsort_and_is_stable(oracle):
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 50, size=5000).astype(np.uint64)  # many ties
    perm = oracle.sort_perm(keys)
    assert np.array_equal(perm, np.lexsort((np.arange(5000), keys)))
    assert sorted(perm.tolist()) == list(range(5000))
    ids = rng.permutation(5000).astype(np.int32)
    perm2 = oracle.sort_perm(keys, ids)
    assert np.array_equal(perm2, np.lexsort((ids, keys)))


# ----------------------------------------------------------------------- tree
@pytest.mark.parametrize("case", GOLD["trees"]["cases"], ids=lambda c: c["name"])
def test_tree_hand_cases(oracle, case):
    pts = np.array(case["pts"], np.int32)
    t = oracle.OracleTree(pts, case["L"], case["bits"])
    d = t.canonical_dump()
    assert d["ids"].tolist() == case["sorted_ids"]
    assert [int(x) for x in d["keys"]] == [int(x) for x in case["sorted_keys"]]
    want = sorted(case["nodes"])
    got = sorted(zip(d["lo"].tolist(), d["hi"].tolist(), d["bit"].tolist()))
    assert [list(g) for g in got] == want
    want_boxes = {(a, z): bx for (a, z, _), bx in zip(case["nodes"], case["boxes"])}
    for a, z, blo, bhi in zip(d["lo"], d["hi"], d["box_lo"], d["box_hi"]):
        assert [blo.tolist(), bhi.tolist()] == want_boxes[(int(a), int(z))]
    if "knn" in case:
        for kk, ref in case["knn"].items():
            if not kk.startswith("k"):
                continue
            k = int(kk[1:])
            for mode_all in (True,):
                idx, d2 = t.knn(k)
                assert idx.tolist() == ref["idx"]
                want_d2 = [[I64MAX if v == "max" else v for v in row] for row in ref["d2"]]
                assert d2.tolist() == want_d2


def _tree_checked(oracle, pts, L, bits, shift=None):
    t = oracle.OracleTree(pts, L, bits, shift)
    e = t.export()
    coords = pts[np.asarray(e["ids"], np.int64)] if len(pts) else np.zeros((0, pts.shape[1]), np.int32)
    depth = check_tree(e["keys"], e["lo"], e["hi"], e["bit"], L, coords=coords,
                       box_lo=e["box_lo"], box_hi=e["box_hi"], left=e["left"], right=e["right"],
                       parent=e["parent"], root=e["root"])
    return t, e, depth


@pytest.mark.parametrize("seed", range(6))
def test_tree_invariants_random(oracle, seed):
    rng = np.random.default_rng(seed)
    dim = 2 + seed % 2
    bits = 10 if seed < 3 else 20
    n = int(rng.integers(1, 3000))
    if seed % 3 == 0:
        pts = rng.integers(0, 2 ** bits, size=(n, dim)).astype(np.int32)
    elif seed % 3 == 1:  # clustered with duplicates
        c = rng.integers(0, 2 ** bits, size=(5, dim))
        pts = np.clip(c[rng.integers(0, 5, n)] + rng.integers(-3, 4, size=(n, dim)), 0, 2 ** bits - 1).astype(np.int32)
    else:  # collinear
        x = rng.integers(0, 2 ** bits, size=n)
        pts = np.stack([x] + [np.full(n, 7)] * (dim - 1), axis=1).astype(np.int32)
    for L in (1, 4, 16):
        _, e, depth = _tree_checked(oracle, pts, L, bits)
        assert depth <= dim * bits + 1
        ids = e["ids"]
        assert sorted(ids.tolist()) == list(range(n))


def test_tree_full_lattice_is_perfect(oracle):
    # [0, 2^m)^d with L = 2^j: every split halves the points, so the tree is a
    # perfect binary tree of depth d*m - j with 2^(d*m-j) leaves of 2^j points.
    for dim, m, j in ((2, 4, 0), (2, 4, 2), (3, 3, 1), (3, 3, 3)):
        g = np.stack(np.meshgrid(*[np.arange(2 ** m)] * dim, indexing="ij"), -1).reshape(-1, dim)
        t, e, depth = _tree_checked(oracle, g.astype(np.int32), 2 ** j, m)
        leaves = e["bit"] < 0
        assert depth == dim * m - j
        assert leaves.sum() == 2 ** (dim * m - j)
        assert np.all((e["hi"] - e["lo"])[leaves] == 2 ** j)


def test_tree_degenerate_cases(oracle):
    pts = np.random.default_rng(1).integers(0, 1000, size=(50, 3)).astype(np.int32)
    _, e, _ = _tree_checked(oracle, pts, 64, 10)  # L >= n: one leaf
    assert len(e["lo"]) == 1 and e["bit"][0] == -1
    same = np.full((40, 2), 9, np.int32)  # all equal: one oversize leaf
    _, e, _ = _tree_checked(oracle, same, 4, 8)
    assert len(e["lo"]) == 1 and e["hi"][0] == 40
    _, e, _ = _tree_checked(oracle, np.zeros((0, 3), np.int32), 16, 21)  # empty
    assert len(e["lo"]) == 1 and e["hi"][0] == 0
    _, e, _ = _tree_checked(oracle, np.array([[1, 2, 3]], np.int32), 1, 21)
    assert len(e["lo"]) == 1


def test_shift_changes_tree_not_answer(oracle):
    rng = np.random.default_rng(3)
    pts = rng.integers(0, 2 ** 18, size=(1500, 3)).astype(np.int32)
    t0 = oracle.OracleTree(pts, 8, 21)
    t1 = oracle.OracleTree(pts, 8, 21, shift=[12345, 999, 77777])
    i0, d0 = t0.knn(6)
    i1, d1 = t1.knn(6)
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)
    _tree_checked(oracle, pts, 8, 21, shift=[12345, 999, 77777])


# ------------------------------------------------------------------------ kNN
def _shapes(rng, kind, n, dim, bits):
    if kind == "uniform":
        return rng.integers(0, 2 ** bits, size=(n, dim)).astype(np.int32)
    if kind == "clustered":
        c = rng.integers(0, 2 ** bits, size=(4, dim))
        return np.clip(c[rng.integers(0, 4, n)] + rng.normal(0, 30, (n, dim)), 0, 2 ** bits - 1).astype(np.int32)
    if kind == "dups":
        base = rng.integers(0, 64, size=(max(1, n // 4), dim))
        return base[rng.integers(0, len(base), n)].astype(np.int32)
    if kind == "collinear":
        x = rng.integers(0, 2 ** bits, size=n)
        return np.stack([x] + [np.full(n, 3)] * (dim - 1), 1).astype(np.int32)
    if kind == "lattice":
        s = int(round(n ** (1.0 / dim))) + 1
        g = np.stack(np.meshgrid(*[np.arange(s)] * dim, indexing="ij"), -1).reshape(-1, dim)
        return g[:n].astype(np.int32) * 5
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["uniform", "clustered", "dups", "collinear", "lattice"])
@pytest.mark.parametrize("dim", [2, 3])
def test_knn_all_points_vs_numpy_brute(oracle, kind, dim):
    rng = np.random.default_rng(hash((kind, dim)) % 2 ** 32)
    bits = 12
    for n, L, k in ((600, 4, 5), (300, 16, 10), (40, 1, 40), (5, 2, 8)):
        pts = _shapes(rng, kind, n, dim, bits)
        t = oracle.OracleTree(pts, L, bits)
        idx, d2 = t.knn(k)
        bi, bd = brute_knn(pts, k)
        assert np.array_equal(d2, bd)
        assert np.array_equal(idx, bi)
        ci, cd = oracle.knn_brute(pts, k)
        assert np.array_equal(ci, bi) and np.array_equal(cd, bd)


@pytest.mark.parametrize("mode", [1, 2])
def test_knn_external_queries_bit_and_root(oracle, mode):
    rng = np.random.default_rng(40 + mode)
    for dim in (2, 3):
        pts = _shapes(rng, "clustered", 1200, dim, 14)
        q = rng.integers(0, 2 ** 14, size=(300, dim)).astype(np.int32)
        q[:20] = pts[:20]  # queries that coincide with points: d^2 = 0 is legal
        t = oracle.OracleTree(pts, 8, 14)
        idx, d2 = t.knn(7, queries=q, mode=mode)
        bi, bd = brute_knn(pts, 7, queries=q)
        assert np.array_equal(idx, bi) and np.array_equal(d2, bd)


@pytest.mark.parametrize("name", ["2DinCube", "2Dkuzmin", "3DonSphere", "3DinCube", "3Dplummer"])
def test_knn_skewed_sets_vs_numpy_brute(oracle, name):
    """The five point sets of the search-start comparison, small: the
    oracle's tree search (all points, and external queries from both starts)
    equals numpy brute force, at k = 1 and 12."""
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_skewed(name, n=2500)
    pts, bits = w["pts"], w["coord_bits"]
    t = oracle.OracleTree(pts, 16, bits)
    rng = np.random.default_rng(9)
    q = pts[rng.choice(len(pts), 200, replace=False)] + rng.integers(-3, 4, size=(200, w["dim"])).astype(np.int32)
    q = np.clip(q, 0, 2 ** (bits - (1 if w["dim"] == 3 else 0)) - 1).astype(np.int32)
    for k in (1, 12):
        idx, d2 = t.knn(k)
        bi, bd = brute_knn(pts, k)
        assert np.array_equal(idx, bi) and np.array_equal(d2, bd), k
        for mode in (1, 2):
            idx, d2 = t.knn(k, queries=q, mode=mode)
            bi, bd = brute_knn(pts, k, queries=q)
            assert np.array_equal(idx, bi) and np.array_equal(d2, bd), (k, mode)


def test_knn_lattice_closed_form(oracle):
    # Interior points of the unit lattice have exactly 2d neighbours at d^2 = 1.
    for dim in (2, 3):
        s = 7
        g = np.stack(np.meshgrid(*[np.arange(s)] * dim, indexing="ij"), -1).reshape(-1, dim).astype(np.int32)
        t = oracle.OracleTree(g, 4, 4)
        idx, d2 = t.knn(2 * dim + 1)
        for i, p in enumerate(g):
            if np.all((p > 0) & (p < s - 1)):
                assert np.all(d2[i, : 2 * dim] == 1) and d2[i, 2 * dim] == 2
                nb = np.nonzero(np.abs(g - p).sum(1) == 1)[0]
                assert idx[i, : 2 * dim].tolist() == sorted(nb.tolist())


def _floats(rows):
    return np.array([[float(v) for v in r] for r in rows], np.float32)


@pytest.mark.parametrize("case", GOLD["quantize"]["frames"], ids=lambda c: c["name"])
def test_quantize_frame_hand_values(oracle, case):
    # Sec. 3.1 "Numerical details": the frame (per-axis minimum, one common
    # scale from the largest extent), the floored grid and the Morton keys
    # of the tree built on it, all worked out by hand.
    pts = _floats(case["pts"])
    lo, scale = oracle.quantization_of(pts, case["bits"])
    assert lo.tolist() == case["lo"] and scale == case["scale"]
    q = oracle.quantize(pts, lo, scale, case["bits"])
    assert q.tolist() == case["q"]
    t = oracle.OracleTree(pts, 1, case["bits"], qlo=lo, qscale=scale)
    e = t.export()
    assert sorted(int(k) for k in e["keys"]) == sorted(int(k) for k in case["keys"])
    assert [int(e["keys"][i]) for i in np.argsort(e["ids"])] == [int(k) for k in case["keys"]]


@pytest.mark.parametrize("case", GOLD["quantize"]["explicit"], ids=lambda c: c["name"])
def test_quantize_explicit_hand_values(oracle, case):
    # Floor, clamp to [0, 2^B - 1], NaN -> 0, and the product taken in fp64.
    q = oracle.quantize(_floats(case["pts"]), np.array(case["lo"]), case["scale"], case["bits"])
    assert q.tolist() == case["q"]


def test_knn_float_fp64_ranking(oracle):
    rng = np.random.default_rng(8)
    a = rng.standard_normal((400, 3)).astype(np.float32)
    b = rng.standard_normal((900, 3)).astype(np.float32)
    lo, scale = oracle.quantization_of(b, 21)
    t = oracle.OracleTree(b, 16, 21, qlo=lo, qscale=scale)
    bi, bd = brute_knn(b, 8, queries=a)
    for mode in (1, 2):
        idx, d2 = t.knn(8, queries=a, mode=mode)
        assert np.array_equal(idx, bi) and np.array_equal(d2, bd)
    idx, d2 = t.knn(5)  # all points, self excluded
    bi, bd = brute_knn(b, 5)
    assert np.array_equal(idx, bi) and np.array_equal(d2, bd)
    ci, cd = oracle.knn_brute(b, 8, queries=a)
    bi, bd = brute_knn(b, 8, queries=a)
    assert np.array_equal(ci, bi) and np.array_equal(cd, bd)


# ------------------------------------------------------------------- dynamic
def test_dynamic_insert_delete_restores_tree(oracle):
    rng = np.random.default_rng(21)
    pts = rng.integers(0, 2 ** 16, size=(2000, 3)).astype(np.int32)
    s = oracle.OracleSet(pts, 8, 21)
    d0 = s.tree().canonical_dump()
    new = s.insert(rng.integers(0, 2 ** 16, size=(500, 3)).astype(np.int32))
    assert new.tolist() == list(range(2000, 2500))
    t1 = s.tree()
    e = t1.export()
    coords = s.pts[np.searchsorted(s.ids, e["ids"])]
    check_tree(e["keys"], e["lo"], e["hi"], e["bit"], 8, coords=coords, box_lo=e["box_lo"],
               box_hi=e["box_hi"], left=e["left"], right=e["right"], parent=e["parent"], root=e["root"])
    q = rng.integers(0, 2 ** 16, size=(100, 3)).astype(np.int32)
    idx, d2 = t1.knn(5, queries=q, mode=1)
    bi, bd = brute_knn(s.pts, 5, queries=q, ref_ids=s.ids)
    assert np.array_equal(idx, bi) and np.array_equal(d2, bd)
    s.delete(new)
    d1 = s.tree().canonical_dump()
    for key in d0:
        assert np.array_equal(d0[key], d1[key])
    with pytest.raises(oracle.OracleError):
        s.delete([99999])
    with pytest.raises(oracle.OracleError):
        s.delete([3, 3])


# ------------------------------------------------------------------- gradient
def _loss64(a, b, idx):
    d = a[:, None, :] - b[idx]
    return np.sqrt((d * d).sum(-1)).sum()


def test_gradient_finite_differences(oracle):
    rng = np.random.default_rng(17)
    a = rng.standard_normal((60, 3)).astype(np.float32)
    b = rng.standard_normal((150, 3)).astype(np.float32)
    idx, _ = brute_knn(b, 4, queries=a)
    loss, ga, gb = oracle.knn_dist_grad(a, b, idx)
    A, B = a.astype(np.float64), b.astype(np.float64)
    assert abs(loss - _loss64(A, B, idx)) <= 1e-9 * abs(loss)
    h = 1e-6
    for i in range(0, 60, 7):
        for c in range(3):
            Ap, Am = A.copy(), A.copy()
            Ap[i, c] += h
            Am[i, c] -= h
            fd = (_loss64(Ap, B, idx) - _loss64(Am, B, idx)) / (2 * h)
            assert abs(fd - ga[i, c]) <= 1e-6 * max(1.0, abs(fd))
    for m in np.unique(idx)[:20]:
        for c in range(3):
            Bp, Bm = B.copy(), B.copy()
            Bp[m, c] += h
            Bm[m, c] -= h
            fd = (_loss64(A, Bp, idx) - _loss64(A, Bm, idx)) / (2 * h)
            assert abs(fd - gb[m, c]) <= 1e-6 * max(1.0, abs(fd))
    # points never chosen as neighbours get no gradient
    unused = np.setdiff1d(np.arange(150), idx.ravel())
    assert np.all(gb[unused] == 0)


def test_gradient_zero_distance_is_zero(oracle):
    a = np.array([[0.5, 0.5, 0.5]], np.float32)
    b = np.array([[0.5, 0.5, 0.5], [1.5, 0.5, 0.5]], np.float32)
    loss, ga, gb = oracle.knn_dist_grad(a, b, np.array([[0, 1]], np.int32))
    assert loss == pytest.approx(1.0)
    assert np.allclose(ga, [[-1.0, 0, 0]]) and np.allclose(gb[0], 0) and np.allclose(gb[1], [1.0, 0, 0])
