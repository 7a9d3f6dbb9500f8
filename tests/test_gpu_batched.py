"""GPU batched forest: every cloud's subtree is that cloud's own canonical
tree, and all-points k-NN never leaves a cloud (ids are cloud-local)."""
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


@pytest.mark.parametrize("mapping", [0x100, 0x200])
def test_batched_tiny_clouds_have_their_own_trees(zd, oracle, mapping):
    """Clouds smaller than L next to each other: every cloud boundary is a
    leaf boundary, and each cloud's subtree is that cloud's canonical tree."""
    from tests._gpu import nodes_of
    rng = np.random.default_rng(8)
    sizes = rng.integers(0, 40, size=300)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = rng.integers(0, 2 ** 16, size=(int(off[-1]), 3)).astype(np.int32)
    t = zd.zd_build_batched(torch.from_numpy(pts).to(DEV), off, 16, 16)
    idx, d2 = zd.zd_knn_batched(t, 5, mapping=mapping)
    assert zd.zd_check() == 0
    idx, d2 = idx.cpu().numpy(), d2.cpu().numpy()
    g = nodes_of(t.export())
    cloud_bit = 3 * t.info()["coord_bits"]
    for c in range(300):
        a, z = int(off[c]), int(off[c + 1])
        if z == a:
            continue
        cloud = pts[a:z]
        bi, bd = oracle.knn_brute(cloud, 5)
        assert np.array_equal(idx[a:z], bi) and np.array_equal(d2[a:z], bd), c
        # the nodes inside this cloud are exactly its own canonical tree
        inside = (g["lo"] >= a) & (g["hi"] <= z) & (g["bit"] < cloud_bit)
        got = sorted(zip((g["lo"][inside] - a).tolist(), (g["hi"][inside] - a).tolist(), g["bit"][inside].tolist()))
        o = oracle.OracleTree(cloud, 16, t.info()["coord_bits"]).canonical_dump()
        want = sorted(zip(o["lo"].tolist(), o["hi"].tolist(), o["bit"].tolist()))
        assert got == want, c
    t.free()


@pytest.mark.parametrize("mapping", [0x100, 0x200])
def test_batched_all_points_per_cloud(zd, oracle, mapping):
    from paper_2111_04182_gb300 import datagen
    w = datagen.workload_batched(n_clouds=40, seed=3, size_range=(1, 9000))
    # drop cloud 4's points: an empty cloud in the middle of the forest
    off2 = np.zeros(41, np.int64)
    chunks = []
    for c in range(40):
        sz = 0 if c == 4 else int(w["offsets"][c + 1] - w["offsets"][c])
        chunks.append(w["pts"][w["offsets"][c]:w["offsets"][c] + sz])
        off2[c + 1] = off2[c] + sz
    pts = np.concatenate(chunks)
    t = zd.zd_build_batched(torch.from_numpy(pts).to(DEV), off2, 16, 16)
    idx, d2 = zd.zd_knn_batched(t, 16, mapping=mapping)
    assert zd.zd_check() == 0
    idx, d2 = idx.cpu().numpy(), d2.cpu().numpy()
    for c in range(40):
        a, z = off2[c], off2[c + 1]
        if z == a:
            continue
        cloud = pts[a:z]
        ot = oracle.OracleTree(cloud, 16, 16)
        oi, od = ot.knn(16)
        assert np.array_equal(idx[a:z], oi), c
        assert np.array_equal(d2[a:z], od), c
    t.free()


@pytest.mark.parametrize("mapping", [0x100, 0x200])
def test_batched_external_float_queries(zd, oracle, mapping):
    from paper_2111_04182_gb300 import datagen
    rng = np.random.default_rng(12)
    P = 5
    A, B = zip(*[datagen.warped_pair(rng, 700 + 100 * p, 1500 + 50 * p) for p in range(P)])
    offA = np.concatenate([[0], np.cumsum([len(a) for a in A])])
    offB = np.concatenate([[0], np.cumsum([len(b) for b in B])])
    t = zd.zd_build_batched(torch.from_numpy(np.concatenate(B)).to(DEV), offB, 8, 21)
    idx, dist = zd.zd_knn_batched(t, 8, queries=torch.from_numpy(np.concatenate(A)).to(DEV),
                                  query_offsets=offA, mapping=mapping)
    assert zd.zd_check() == 0
    idx = idx.cpu().numpy()
    for p in range(P):
        bi, bd = oracle.knn_brute(B[p], 8, queries=A[p])
        assert np.array_equal(idx[offA[p]:offA[p + 1]], bi), p
    t.free()


def test_batched_step_in_cuda_graph_matches_eager(zd, oracle):
    """The whole forest step (build + all-points search + free) captured in
    one CUDA graph and replayed gives the eager answer."""
    from paper_2111_04182_gb300 import autotune, datagen
    w = datagen.workload_batched(n_clouds=64, seed=11, size_range=(100, 5000))
    pts = torch.from_numpy(w["pts"]).to(DEV)
    off = w["offsets"]
    off_d = torch.from_numpy(off).to(DEV)
    n = int(off[-1])
    tune = autotune.tune_batched(pts, off, 16, 16, use_cache=False, reps=1)
    assert tune["leaf_size"] in autotune.LEAF_SIZES and len(tune["table"]) == 2 * len(autotune.LEAF_SIZES)
    L, mp = tune["leaf_size"], tune["mapping"]
    idx = torch.full((n, 16), -7, dtype=torch.int32, device=DEV)
    d2 = torch.full((n, 16), -7, dtype=torch.int64, device=DEV)

    def step():
        t = zd.zd_build_batched(pts, off, L, 16, offsets_device=off_d)
        zd.zd_knn_batched(t, 16, out=(idx, d2), mapping=mp)
        t.free()

    step()
    torch.cuda.synchronize()
    ref_i, ref_d = idx.clone(), d2.clone()
    idx.fill_(-7)
    d2.fill_(-7)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        step()
        g.capture_end()
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        idx.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(idx, ref_i) and torch.equal(d2, ref_d)
    assert zd.zd_check() == 0
    c = 3
    a, z = int(off[c]), int(off[c + 1])
    bi, bd = oracle.knn_brute(w["pts"][a:z], 16)
    assert np.array_equal(ref_i[a:z].cpu().numpy(), bi)


@pytest.mark.parametrize("mapping", [0x100, 0x200])
def test_batched_external_int_queries(zd, oracle, mapping):
    """External integer queries per cloud, including an empty cloud and a
    cloud with no queries."""
    rng = np.random.default_rng(21)
    sizes = [500, 0, 1200, 37, 900]
    qsizes = [300, 50, 0, 400, 260]
    B = [rng.integers(0, 2 ** 16, size=(s, 3)).astype(np.int32) for s in sizes]
    A = [rng.integers(0, 2 ** 16, size=(s, 3)).astype(np.int32) for s in qsizes]
    offB = np.concatenate([[0], np.cumsum(sizes)])
    offA = np.concatenate([[0], np.cumsum(qsizes)])
    t = zd.zd_build_batched(torch.from_numpy(np.concatenate(B)).to(DEV), offB, 8, 16)
    idx, d2 = zd.zd_knn_batched(t, 6, queries=torch.from_numpy(np.concatenate(A)).to(DEV),
                                query_offsets=offA, mapping=mapping)
    assert zd.zd_check() == 0
    idx, d2 = idx.cpu().numpy(), d2.cpu().numpy()
    for c in range(5):
        a, z = offA[c], offA[c + 1]
        if z == a:
            continue
        if sizes[c] == 0:
            assert np.all(idx[a:z] == -1)
            continue
        bi, bd = oracle.knn_brute(B[c], 6, queries=A[c])
        assert np.array_equal(idx[a:z], bi) and np.array_equal(d2[a:z], bd), c
    t.free()
