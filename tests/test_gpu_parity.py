"""GPU parity: every step of the path through the C ABI against the oracle.

Integer work is compared bit-exactly (keys, sorted order, tree shape and
boxes, neighbour ids and squared distances).  Sizes span several tiles of
every kernel (4096-key sort tiles, 1024-boundary split tiles, 128-query k-NN
blocks) plus a ragged tail.
"""
import numpy as np
import pytest

from tests._checks import brute_knn, check_tree
from tests._gpu import canonical, nodes_of

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


DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


# --------------------------------------------------------------- encode
@pytest.mark.parametrize("dim,bits,shift", [(3, 21, None), (2, 20, None), (2, 31, [5, 7]), (3, 18, [3, 1000, 77])])
def test_encode_matches_oracle(zd, oracle, dim, bits, shift):
    rng = np.random.default_rng(dim * 100 + bits)
    hi = 2 ** bits - (max(shift) if shift else 0)
    for n in (0, 1, 31, 4097, 100_003):
        pts = rng.integers(0, hi, size=(n, dim)).astype(np.int32)
        keys = zd.zd_morton_encode(_t(pts), bits, shift).cpu().numpy().view(np.uint64)
        assert np.array_equal(keys, oracle.morton_keys(pts, bits, shift))
    assert zd.zd_check() == 0


def test_encode_range_error(zd):
    pts = np.array([[0, 0, 0], [2 ** 21, 0, 0]], np.int32)
    zd.zd_morton_encode(_t(pts), 21)
    assert zd.zd_check() == zd.ZD_ERR_RANGE
    assert zd.zd_check() == 0  # cleared


# ----------------------------------------------------------------- sort
@pytest.mark.parametrize("n", [0, 1, 2, 4095, 4096, 4097, 3 * 4096 + 17, 250_001])
@pytest.mark.parametrize("kind", ["random64", "ties", "equal", "morton"])
def test_sort_matches_lexsort(zd, oracle, n, kind):
    rng = np.random.default_rng(n + len(kind))
    if kind == "random64":
        keys = rng.integers(0, 2 ** 63, size=n, dtype=np.int64).view(np.uint64) ^ (
            rng.integers(0, 2, size=n).astype(np.uint64) << np.uint64(63))
        bits = 64
    elif kind == "ties":
        keys = rng.integers(0, 37, size=n).astype(np.uint64) << np.uint64(20)
        bits = 26
    elif kind == "equal":
        keys = np.full(n, 12345, np.uint64)
        bits = 20
    else:
        keys = oracle.morton_keys(rng.integers(0, 2 ** 21, size=(n, 3)).astype(np.int32), 21)
        bits = 63
    sk, perm = zd.zd_morton_sort(_t(keys.view(np.int64)), bits)
    assert zd.zd_check() == 0
    want = np.lexsort((np.arange(n), keys))
    assert np.array_equal(perm.cpu().numpy(), want)
    assert np.array_equal(sk.cpu().numpy().view(np.uint64), keys[want])


# ----------------------------------------------------------------- tree
def _compare_tree(zd, oracle, pts, L, bits, shift=None):
    t = zd.zd_build(_t(pts), L, bits, shift)
    assert zd.zd_check() == 0
    g = nodes_of(t.export())
    ot = oracle.OracleTree(pts, L, bits, shift)
    o = ot.canonical_dump()
    assert np.array_equal(g["ids"], o["ids"]), "sorted order"
    assert np.array_equal(g["keys"], o["keys"]), "sorted keys"
    c = canonical(g)
    for f in ("lo", "hi", "bit"):
        assert np.array_equal(c[f], o[f]), "tree shape: " + f
    nonempty = c["hi"] > c["lo"]
    assert np.array_equal(c["box_lo"][nonempty], o["box_lo"][nonempty]), "boxes"
    assert np.array_equal(c["box_hi"][nonempty], o["box_hi"][nonempty]), "boxes"
    coords = pts[g["ids"].astype(np.int64)]
    check_tree(g["keys"], g["lo"], g["hi"], g["bit"], L, coords=coords, box_lo=g["box_lo"],
               box_hi=g["box_hi"], left=g["left"], right=g["right"], parent=g["parent"], root=g["root"])
    return t


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("L", [1, 4, 16, 33])
def test_build_matches_oracle(zd, oracle, dim, L):
    rng = np.random.default_rng(dim * 10 + L)
    bits = 21 if dim == 3 else 20
    for n in (1, 2, 17, 5000, 70_001):
        pts = rng.integers(0, 2 ** (bits - 1), size=(n, dim)).astype(np.int32)
        _compare_tree(zd, oracle, pts, L, bits).free()
    c = rng.integers(0, 2 ** 19, size=(8, dim))
    pts = np.clip(c[rng.integers(0, 8, 30000)] + rng.integers(-4, 5, size=(30000, dim)), 0, 2 ** 19).astype(np.int32)
    _compare_tree(zd, oracle, pts, L, bits).free()  # clustered, many duplicates


def test_build_degenerate(zd, oracle):
    _compare_tree(zd, oracle, np.full((5000, 3), 7, np.int32), 16, 21).free()  # one oversize leaf
    _compare_tree(zd, oracle, np.random.default_rng(0).integers(0, 100, (40, 2)).astype(np.int32), 64, 20).free()
    x = np.arange(3000, dtype=np.int32)
    _compare_tree(zd, oracle, np.stack([x, x * 0 + 5, x * 0 + 9], 1), 8, 21).free()  # collinear
    _compare_tree(zd, oracle, np.zeros((0, 3), np.int32), 16, 21).free()  # empty
    g = np.stack(np.meshgrid(*[np.arange(16)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.int32)
    _compare_tree(zd, oracle, g, 8, 4).free()  # full lattice: perfect tree
    _compare_tree(zd, oracle, g, 8, 21, shift=[1000, 2000, 3000]).free()


# ------------------------------------------------------------------ kNN
MAPPINGS = [0x100, 0x200]  # one thread per query; one warp per 32-point group


@pytest.mark.parametrize("mapping", MAPPINGS)
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("k", [1, 3, 5, 10, 12, 16, 20, 24, 27, 32])
def test_knn_all_points(zd, oracle, dim, k, mapping):
    rng = np.random.default_rng(dim * 1000 + k)
    bits = 21 if dim == 3 else 20
    c = rng.integers(0, 2 ** 19, size=(12, dim))
    pts = np.clip(c[rng.integers(0, 12, 40_000)] + rng.normal(0, 2000, (40_000, dim)), 0, 2 ** 19).astype(np.int32)
    pts[:300] = pts[300:600]  # duplicates: ties at d^2 = 0
    t = zd.zd_build(_t(pts), 16, bits)
    idx, d2 = t.knn(k, mapping=mapping)
    assert zd.zd_check() == 0
    oi, od = oracle.OracleTree(pts, 16, bits).knn(k)
    assert np.array_equal(d2.cpu().numpy(), od)
    assert np.array_equal(idx.cpu().numpy(), oi)
    t.free()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("k", [1, 10, 40])
def test_knn_graph_three_starts(zd, oracle, dim, k):
    """The k-NN graph computed leaf-based, bit-based and root-based (the
    paper's three algorithms) is the same exact answer."""
    rng = np.random.default_rng(dim * 10 + k)
    bits = 21 if dim == 3 else 20
    c = rng.integers(0, 2 ** 19, size=(6, dim))
    pts = np.clip(c[rng.integers(0, 6, 20_000)] + rng.normal(0, 1500, (20_000, dim)), 0, 2 ** 19).astype(np.int32)
    pts[:200] = pts[200:400]
    t = zd.zd_build(_t(pts), 16, bits)
    oi, od = oracle.OracleTree(pts, 16, bits).knn(k)
    for mode in (zd.ZD_SEARCH_LEAF, zd.ZD_SEARCH_BIT, zd.ZD_SEARCH_ROOT):
        idx, d2 = t.knn(k, mode=mode)
        assert zd.zd_check() == 0
        assert np.array_equal(idx.cpu().numpy(), oi), mode
        assert np.array_equal(d2.cpu().numpy(), od), mode
    t.free()


@pytest.mark.parametrize("name", ["2DinCube", "2Dkuzmin", "3DonSphere", "3DinCube", "3Dplummer"])
def test_skewed_sets_tree_and_all_starts(zd, oracle, name):
    """The five point sets of the paper's search-start comparison (skewed
    Plummer and Kuzmin sets, a sphere surface, uniform square and cube): the
    canonical tree and the k-NN graph from every start and mapping equal the
    oracle's."""
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_skewed(name, n=30_000)
    pts, bits = w["pts"], w["coord_bits"]
    t = zd.zd_build(_t(pts), 16, bits)
    ot = oracle.OracleTree(pts, 16, bits)
    o, g = ot.canonical_dump(), canonical(nodes_of(t.export()))
    assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["bit"], o["bit"])
    for k in (1, 8):
        oi, od = ot.knn(k)
        for mode, mapping in ((0, 0x100), (0, 0x200), (1, 0), (2, 0)):
            idx, d2 = t.knn(k, mode=mode, mapping=mapping)
            assert zd.zd_check() == 0
            assert np.array_equal(idx.cpu().numpy(), oi), (k, mode, mapping)
            assert np.array_equal(d2.cpu().numpy(), od), (k, mode, mapping)
    t.free()


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_float_knn_ties_and_duplicates(zd, oracle, mapping):
    """Float lattice points (many exactly equal distances) with duplicated
    points: the estimate band overflows the warp-group list and those
    queries take the exact fallback; the answer stays the oracle's."""
    g = np.stack(np.meshgrid(*[np.arange(18)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float32) * 0.25
    pts = np.concatenate([g, g[:700], g[::5] + 0.125]).astype(np.float32)
    t = zd.zd_build(_t(pts), 16, 21)
    for k in (1, 6, 8, 16):
        idx, dist = t.knn(k, mapping=mapping)
        assert zd.zd_check() == 0
        bi, bd = oracle.knn_brute(pts, k)
        assert np.array_equal(idx.cpu().numpy(), bi), k
        assert np.allclose(dist.cpu().numpy(), np.sqrt(bd), rtol=1e-6, atol=0), k
    q = (np.random.default_rng(80).integers(0, 70, size=(3000, 3)) * 0.0625).astype(np.float32)
    for mode in (1, 2):
        idx, dist = t.knn(8, queries=_t(q), mode=mode, mapping=mapping)
        bi, bd = oracle.knn_brute(pts, 8, queries=q)
        assert np.array_equal(idx.cpu().numpy(), bi), mode
    t.free()


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_float_knn_near_ties_at_the_kth_place(zd, oracle, mapping):
    """A float lattice jittered by ~1e-6 of its spacing: distances that differ
    in the 6th or 7th digit, closer than the fp32 estimates can separate, so
    the k-th and (k+1)-th neighbours fall in one estimate band again and
    again.  The exact (fp64, id) ranking of the band must pick the oracle's
    k-th neighbour, whatever order the candidates were found in."""
    rng = np.random.default_rng(81)
    g = np.stack(np.meshgrid(*[np.arange(20)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    pts = (g * 0.5 + rng.normal(0, 5e-7, g.shape)).astype(np.float32)
    t = zd.zd_build(_t(pts), 16, 21)
    for k in (5, 8, 10, 16, 24):
        idx, dist = t.knn(k, mapping=mapping)
        assert zd.zd_check() == 0
        bi, bd = oracle.knn_brute(pts, k)
        assert np.array_equal(idx.cpu().numpy(), bi), k
    q = (g[::3] * 0.5 + 0.25 + rng.normal(0, 5e-7, g[::3].shape)).astype(np.float32)
    for mode in (1, 2):
        idx, dist = t.knn(8, queries=_t(q), mode=mode, mapping=mapping)
        bi, bd = oracle.knn_brute(pts, 8, queries=q)
        assert np.array_equal(idx.cpu().numpy(), bi), mode
    t.free()


def test_float_knn_graph_three_starts(zd, oracle):
    from paper_2111_04182_gb300 import datagen
    _, b = datagen.warped_pair(np.random.default_rng(79), 10, 7000)
    t = zd.zd_build(_t(b), 16, 21)
    bi, bd = oracle.knn_brute(b, 7)
    for mode in (zd.ZD_SEARCH_LEAF, zd.ZD_SEARCH_BIT, zd.ZD_SEARCH_ROOT):
        idx, dist = t.knn(7, mode=mode)
        assert np.array_equal(idx.cpu().numpy(), bi), mode
        assert np.allclose(dist.cpu().numpy(), np.sqrt(bd), rtol=1e-6, atol=0)
    t.free()
    assert zd.zd_check() == 0


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_knn_saturated_keys_fall_back_exactly(zd, oracle, mapping):
    """Far-apart 2D points with 31-bit coordinates: squared distances exceed
    the packed-key field of the warp-group mapping, whose queries must then
    be answered by the exact fallback -- the result stays exact."""
    rng = np.random.default_rng(31)
    pts = rng.integers(0, 2 ** 31 - 1, size=(3000, 2)).astype(np.int32)
    pts[:40] = rng.integers(0, 64, size=(40, 2))  # a tight cluster too
    t = zd.zd_build(_t(pts), 8, 31)
    idx, d2 = t.knn(6, mapping=mapping)
    assert zd.zd_check() == 0
    bi, bd = oracle.knn_brute(pts, 6)
    assert np.array_equal(idx.cpu().numpy(), bi) and np.array_equal(d2.cpu().numpy(), bd)
    t.free()


def test_knn_small_and_padding(zd, oracle):
    for n, k, L in ((1, 4, 16), (2, 4, 1), (7, 10, 2), (33, 32, 4), (300, 5, 1)):
        pts = np.random.default_rng(n).integers(0, 1000, size=(n, 3)).astype(np.int32)
        t = zd.zd_build(_t(pts), L, 21)
        idx, d2 = t.knn(k)
        bi, bd = brute_knn(pts, k)
        assert np.array_equal(idx.cpu().numpy(), bi) and np.array_equal(d2.cpu().numpy(), bd)
        t.free()
    assert zd.zd_check() == 0


def test_knn_lattice_ties(zd, oracle):
    g = (np.stack(np.meshgrid(*[np.arange(20)] * 3, indexing="ij"), -1).reshape(-1, 3) * 3).astype(np.int32)
    oi, od = oracle.OracleTree(g, 16, 21).knn(10)
    for shift in (None, [5, 77, 1 << 19]):
        t = zd.zd_build(_t(g), 16, 21, shift=shift)
        for mapping in MAPPINGS:
            idx, d2 = t.knn(10, mapping=mapping)
            assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
        t.free()


@pytest.mark.parametrize("mapping", MAPPINGS)
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("dim", [2, 3])
def test_knn_external_queries(zd, oracle, mode, dim, mapping):
    rng = np.random.default_rng(mode * 7 + dim)
    bits = 21 if dim == 3 else 20
    pts = rng.integers(0, 2 ** 20, size=(60_000, dim)).astype(np.int32)
    q = rng.integers(0, 2 ** 20, size=(9_001, dim)).astype(np.int32)
    q[:50] = pts[:50]
    t = zd.zd_build(_t(pts), 16, bits, shift=[3, 0, 17][:dim])
    idx, d2 = t.knn(5, queries=_t(q), mode=mode, mapping=mapping)
    assert zd.zd_check() == 0
    oi, od = oracle.knn_brute(pts, 5, queries=q)
    assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
    t.free()


@pytest.mark.parametrize("mapping", MAPPINGS)
@pytest.mark.parametrize("dim", [2, 3])
def test_knn_far_from_the_origin(zd, oracle, dim, mapping):
    """Coordinates near -2^29 and -2^30 brought into [0, 2^20) by a large
    shift: the raw values are not exact in fp32, the shifted ones are.  The
    all-points graph (clustered, with duplicates) and external queries
    (bit- and root-based) must still equal the oracle's."""
    rng = np.random.default_rng(40 + dim)
    shift = [1 << 29, (1 << 30) + 12345, 7][:dim]
    c = rng.integers(0, 2 ** 20, size=(10, dim))
    u = np.clip(c[rng.integers(0, 10, 30_000)] + rng.normal(0, 300, (30_000, dim)), 0, 2 ** 20 - 1)
    pts = (u.astype(np.int64) - np.array(shift, np.int64)).astype(np.int32)
    pts[:200] = pts[200:400]  # duplicates
    qu = rng.integers(0, 2 ** 20, size=(5_000, dim))
    q = (qu - np.array(shift, np.int64)).astype(np.int32)
    q[:40] = pts[:40]
    t = zd.zd_build(_t(pts), 16, 20, shift=shift)
    ot = oracle.OracleTree(pts, 16, 20, shift)
    for k in (1, 10):
        idx, d2 = t.knn(k, mapping=mapping)
        oi, od = ot.knn(k)
        assert np.array_equal(d2.cpu().numpy(), od) and np.array_equal(idx.cpu().numpy(), oi), k
    for mode in (1, 2):
        idx, d2 = t.knn(5, queries=_t(q), mode=mode, mapping=mapping)
        oi, od = oracle.knn_brute(pts, 5, queries=q)
        assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od), mode
    assert zd.zd_check() == 0
    t.free()


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_knn_bands_wider_than_the_candidate_buffer(zd, oracle, mapping):
    """Stacks of 50 identical points and lattice shells with many equal
    distances: the band of near-equal estimates holds more candidates than a
    lane buffers, so those queries take the exact fallback; every row must
    still equal the oracle's (ties by id)."""
    rng = np.random.default_rng(77)
    stacks = np.repeat(rng.integers(0, 2 ** 18, size=(40, 3)), 50, axis=0)
    g = np.stack(np.meshgrid(np.arange(14), np.arange(14), np.arange(14), indexing="ij"), -1).reshape(-1, 3)
    lattice = g * 3 + 2 ** 19
    rest = rng.integers(0, 2 ** 20, size=(20_000, 3))
    pts = np.concatenate([stacks, lattice, rest]).astype(np.int32)
    t = zd.zd_build(_t(pts), 16, 21)
    ot = oracle.OracleTree(pts, 16, 21)
    for k in (10, 24, 40):
        idx, d2 = t.knn(k, mapping=mapping)
        oi, od = ot.knn(k)
        assert np.array_equal(d2.cpu().numpy(), od) and np.array_equal(idx.cpu().numpy(), oi), k
    q = np.concatenate([stacks[::50] + 1, lattice[::7] + 1]).astype(np.int32)
    idx, d2 = t.knn(12, queries=_t(q), mode=1, mapping=mapping)
    oi, od = oracle.knn_brute(pts, 12, queries=q)
    assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
    assert zd.zd_check() == 0
    t.free()


@pytest.mark.parametrize("bits", [24, 25])
def test_knn_at_the_float_copy_limit(zd, oracle, bits):
    """2D points spread over [0, 2^bits): B = 24 is the widest grid with exact
    float copies (the warp groups' band lanes, differences and squares at the
    edge of fp32's exact integers), B = 25 the narrowest without them (exact
    int64 lanes).  Clustered, with duplicates; all points and external
    queries against the oracle."""
    rng = np.random.default_rng(60 + bits)
    hi = 2 ** bits - 1
    c = rng.integers(0, hi, size=(8, 2))
    pts = np.clip(c[rng.integers(0, 8, 30_000)] + rng.normal(0, 2 ** (bits - 6), (30_000, 2)), 0, hi)
    pts = pts.astype(np.int64)
    pts[:64] = [[0, 0], [hi, hi], [0, hi], [hi, 0]] * 16  # the grid's corners, repeated
    pts = pts.astype(np.int32)
    t = zd.zd_build(_t(pts), 16, bits)
    ot = oracle.OracleTree(pts, 16, bits)
    for k in (3, 10, 16):
        idx, d2 = t.knn(k)
        oi, od = ot.knn(k)
        assert np.array_equal(d2.cpu().numpy(), od) and np.array_equal(idx.cpu().numpy(), oi), k
    q = rng.integers(0, hi, size=(8_000, 2)).astype(np.int32)
    idx, d2 = t.knn(5, queries=_t(q), mode=1)
    oi, od = oracle.knn_brute(pts, 5, queries=q)
    assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
    assert zd.zd_check() == 0
    t.free()


def test_knn_2d_uniform_workload(zd, oracle):
    """The 2D workload at its full size: n = 100,000, L = 16, k = 10."""
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_2d_uniform()
    t = zd.zd_build(_t(w["pts"]), w["leaf_size"], w["coord_bits"])
    _ = _compare_tree
    g = nodes_of(t.export())
    ot = oracle.OracleTree(w["pts"], w["leaf_size"], w["coord_bits"])
    o = ot.canonical_dump()
    c = canonical(g)
    assert np.array_equal(c["lo"], o["lo"]) and np.array_equal(c["bit"], o["bit"])
    idx, d2 = t.knn(w["k"])
    oi, od = ot.knn(w["k"])
    assert np.array_equal(idx.cpu().numpy(), oi) and np.array_equal(d2.cpu().numpy(), od)
    t.free()
    assert zd.zd_check() == 0


# --------------------------------------------------------------- float
@pytest.mark.parametrize("mapping", MAPPINGS)
def test_float_knn_fp64_ranking(zd, oracle, mapping):
    from paper_2111_04182_gb300 import datagen
    rng = np.random.default_rng(77)
    a, b = datagen.warped_pair(rng, 6000, 12000)
    t = zd.zd_build(_t(b), 16, 21)
    e = nodes_of(t.export())
    lo, scale = oracle.quantization_of(b, 21)
    ot = oracle.OracleTree(b, 16, 21, qlo=lo, qscale=scale)
    o = ot.canonical_dump()
    assert np.array_equal(e["keys"], o["keys"]), "float quantization / keys"
    assert np.array_equal(canonical(e)["bit"], o["bit"])
    for mode in (1, 2):
        idx, dist = t.knn(8, queries=_t(a), mode=mode, mapping=mapping)
        bi, bd = oracle.knn_brute(b, 8, queries=a)
        assert np.array_equal(idx.cpu().numpy(), bi)
        assert np.allclose(dist.cpu().numpy(), np.sqrt(bd), rtol=1e-6, atol=0)
    idx, dist = t.knn(6, mapping=mapping)
    bi, bd = oracle.knn_brute(b, 6)
    assert np.array_equal(idx.cpu().numpy(), bi)
    t.free()
    assert zd.zd_check() == 0
