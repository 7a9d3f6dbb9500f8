"""GPU backward of a sum of k-NN distances against the fp64 oracle gradient
and finite differences, and the batched float forward against brute force
with the fp64 ranking.  Gradient tolerance, per element:
max_i |g_i - g64_i| / max(|g64_i|, 1e-3) <= 1e-4."""
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


def _rel(g, g64):
    """Largest per-element error relative to max(|g64_i|, 1e-3)."""
    return float(np.max(np.abs(g.astype(np.float64) - g64) / np.maximum(np.abs(g64), 1e-3)))


def test_backward_matches_fp64(zd, oracle):
    from paper_2111_04182_gb300 import datagen
    rng = np.random.default_rng(4)
    P, m, r, k = 3, 3000, 6000, 8
    A = np.empty((P, m, 3), np.float32)
    B = np.empty((P, r, 3), np.float32)
    for p in range(P):
        A[p], B[p] = datagen.warped_pair(rng, m, r)
    At = torch.from_numpy(A).to(DEV).requires_grad_(True)
    Bt = torch.from_numpy(B).to(DEV).requires_grad_(True)
    dist, idx = zd.KnnDist.apply(At, Bt, k)
    w = torch.from_numpy(rng.standard_normal((P, m, k)).astype(np.float32)).to(DEV)
    (dist * w).sum().backward()
    assert zd.zd_check() == 0
    for p in range(P):
        bi, bd = oracle.knn_brute(B[p], k, queries=A[p])
        assert np.array_equal(idx[p].cpu().numpy(), bi), "fp64 ranking"
        assert np.allclose(dist[p].detach().cpu().numpy(), np.sqrt(bd), rtol=1e-6)
        loss, ga, gb = oracle.knn_dist_grad(A[p], B[p], bi, w[p].cpu().numpy().astype(np.float64))
        assert _rel(At.grad[p].cpu().numpy(), ga) <= 1e-4
        assert _rel(Bt.grad[p].cpu().numpy(), gb) <= 1e-4


def test_backward_finite_differences(zd, oracle):
    rng = np.random.default_rng(9)
    a = rng.standard_normal((200, 3)).astype(np.float32)
    b = rng.standard_normal((500, 3)).astype(np.float32)
    idx, _ = oracle.knn_brute(b, 5, queries=a)
    gq, gr = zd.zd_knn_dist_backward(torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV),
                                     torch.from_numpy(idx).to(DEV), torch.ones(1, device=DEV))
    A, Bd = a.astype(np.float64), b.astype(np.float64)

    def loss(A, Bd):
        d = A[:, None, :] - Bd[idx]
        return np.sqrt((d * d).sum(-1)).sum()

    h = 1e-6
    for i in range(0, 200, 23):
        for c in range(3):
            Ap, Am = A.copy(), A.copy()
            Ap[i, c] += h
            Am[i, c] -= h
            fd = (loss(Ap, Bd) - loss(Am, Bd)) / (2 * h)
            assert abs(gq[i, c].item() - fd) <= 1e-4 * max(1.0, abs(fd))
    for t_ in np.unique(idx)[:25]:
        for c in range(3):
            Bp, Bm = Bd.copy(), Bd.copy()
            Bp[t_, c] += h
            Bm[t_, c] -= h
            fd = (loss(A, Bp) - loss(A, Bm)) / (2 * h)
            assert abs(gr[t_, c].item() - fd) <= 1e-4 * max(1.0, abs(fd))


def test_backward_is_deterministic_and_skips(zd):
    rng = np.random.default_rng(1)
    a = torch.from_numpy(rng.standard_normal((1, 4000, 3)).astype(np.float32)).to(DEV)
    b = torch.from_numpy(rng.standard_normal((1, 100, 3)).astype(np.float32)).to(DEV)
    idx = torch.from_numpy(rng.integers(-1, 100, size=(1, 4000, 8)).astype(np.int32)).to(DEV)
    g1 = zd.zd_knn_dist_backward(a, b, idx, torch.ones(1, device=DEV))
    g2 = zd.zd_knn_dist_backward(a, b, idx, torch.ones(1, device=DEV))
    assert torch.equal(g1[0], g2[0]) and torch.equal(g1[1], g2[1])
    # a zero distance contributes nothing
    q = torch.tensor([[[0.5, 0.5, 0.5]]], device=DEV)
    r = torch.tensor([[[0.5, 0.5, 0.5], [1.5, 0.5, 0.5]]], device=DEV)
    gq, gr = zd.zd_knn_dist_backward(q, r, torch.tensor([[[0, 1]]], dtype=torch.int32, device=DEV),
                                     torch.ones(1, device=DEV))
    assert torch.allclose(gq, torch.tensor([[[-1.0, 0, 0]]], device=DEV))
    assert torch.allclose(gr[0, 0], torch.zeros(3, device=DEV))


@pytest.mark.parametrize("scale", [1e-25, 1.0, 1e12])
def test_backward_per_element_at_extreme_scales(zd, oracle, scale):
    """The same clouds shrunk or blown up: the unit vectors do not depend on
    the scale, so the per-element bound holds whether squared differences
    would underflow or overflow in plain fp32."""
    from paper_2111_04182_gb300 import datagen
    rng = np.random.default_rng(12)
    a, b = datagen.warped_pair(rng, 2000, 5000)
    a, b = (a * scale).astype(np.float32), (b * scale).astype(np.float32)
    idx, _ = oracle.knn_brute(b, 6, queries=a)
    g = rng.standard_normal((2000, 6)).astype(np.float32)
    gq, gr = zd.zd_knn_dist_backward(torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV),
                                     torch.from_numpy(idx).to(DEV), torch.from_numpy(g).to(DEV))
    _, ga, gb = oracle.knn_dist_grad(a, b, idx, g.astype(np.float64))
    assert _rel(gq.cpu().numpy(), ga) <= 1e-4
    assert _rel(gr.cpu().numpy(), gb) <= 1e-4
