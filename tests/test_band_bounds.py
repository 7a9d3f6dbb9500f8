"""The numerical argument behind the band lanes of the integer warp-group
k-NN search, checked on the CPU (no GPU).

The search ranks candidates by an fp32 estimate of d^2 computed from exact
float copies of the (shifted) coordinates,
    est = fma(x, x, fma(y, y, z * z)),   x, y, z exact coordinate differences,
keeps only the K smallest estimates (eK the K-th), accepts candidates and
visits boxes up to thr = eK (1 + 2^-19) rounded up, and at the end ranks the
candidates whose estimate is at most band = eK (1 + 2^-20) rounded up by their
exact int64 d^2 and id.  That answer is exact if (a) the estimate's relative
error is at most (1 + 2^-24)^3 - 1, (b) every true neighbour (the K smallest
by (d^2, id)) has estimate <= band, and (c) a box whose estimate exceeds thr
holds no point with estimate <= band.

The fp32 arithmetic is emulated exactly: for |x| < 2^24, x * x and each
partial sum are exact in fp64 (at most 50 significant bits), so rounding the
fp64 value to fp32 once gives what one fp32 multiply or fma returns.
"""
import numpy as np

U = 2.0 ** -24


def f32(v):
    return np.asarray(v, np.float64).astype(np.float32).astype(np.float64)


def mul_ru(a, c):
    """fp32 product rounded up (both factors fp32, product exact in fp64)."""
    p = np.asarray(a, np.float64) * c
    r = p.astype(np.float32)
    r = np.where(r.astype(np.float64) < p, np.nextafter(r, np.float32(np.inf)), r)
    return r.astype(np.float64)


def est3(x, y, z):
    x, y, z = (np.asarray(v, np.float64) for v in (x, y, z))
    return f32(x * x + f32(y * y + f32(z * z)))


def test_estimate_error_bound():
    rng = np.random.default_rng(0)
    d = rng.integers(-(2 ** 23), 2 ** 23, size=(200_000, 3))
    d[:1000] = rng.integers(-4, 5, size=(1000, 3))          # tiny distances
    d[1000:2000, :2] = 0                                     # one axis only
    D = (d.astype(np.float64) ** 2).sum(1)
    e = est3(d[:, 0], d[:, 1], d[:, 2])
    nz = D > 0
    rel = np.abs(e[nz] - D[nz]) / D[nz]
    assert rel.max() <= (1 + U) ** 3 - 1
    assert np.all(e[~nz] == 0)  # an exact duplicate has estimate 0, nothing else does
    assert np.all(e[nz] > 0)


def _shell(rng, n, r):
    """Integer points rounded onto a sphere of radius r: their d^2 differ by
    about 2^-28 of each other at r = 2^20, below the estimate's rounding."""
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return np.rint(u * r).astype(np.int64)


def test_true_neighbours_lie_in_the_band():
    """Near-tied sets (points rounded onto a sphere, whose estimates may rank
    them in a different order than their exact d^2; lattices with exact
    ties): the K nearest by (d^2, id) all have estimate <= band."""
    rng = np.random.default_rng(1)
    swaps = 0
    for trial in range(300):
        K = int(rng.choice([1, 5, 8, 10, 16, 24]))
        if trial % 2:
            d = _shell(rng, 400, float(rng.choice([2.0 ** 20, 2.0 ** 22, 3.0e6])))
        else:
            scale = int(rng.choice([1, 1000, 2 ** 20]))
            d = rng.integers(-3, 4, size=(400, 3)) * scale + rng.integers(-1, 2, size=(400, 3))
        D = (d.astype(np.int64) ** 2).sum(1)
        e = est3(d[:, 0], d[:, 1], d[:, 2])
        ids = rng.permutation(len(d))
        order = np.lexsort((ids, D))[:K]
        eK = np.sort(e)[K - 1]
        swaps += int(np.any(e[order] > eK))  # the estimates put a true neighbour past eK
        band = mul_ru(eK, 1 + 2.0 ** -20)
        thr = mul_ru(eK, 1 + 2.0 ** -19)
        assert np.all(e[order] <= band), trial
        assert band <= thr
    assert swaps > 20  # the sets do exercise the band beyond eK


def test_box_pruning_margin():
    """A box whose estimate (exact per-axis gaps, fp32 sum) exceeds
    thr = eK (1 + 2^-19) holds no point with estimate <= band = eK (1 + 2^-20)."""
    rng = np.random.default_rng(2)
    for trial in range(2000):
        q = rng.integers(0, 2 ** 21, size=3)
        lo = rng.integers(0, 2 ** 21, size=3)
        hi = lo + rng.integers(0, 2 ** 12, size=3)
        gap = np.maximum(np.maximum(lo - q, q - hi), 0)
        be = est3(gap[0], gap[1], gap[2])
        # the tightest thr the box test could be compared with: just below be
        eK = float(np.float32(be / (1 + 2.0 ** -19)))
        while mul_ru(eK, 1 + 2.0 ** -19) >= be and eK > 0:
            eK = float(np.nextafter(np.float32(eK), np.float32(0)))
        if eK <= 0:
            continue
        band = mul_ru(eK, 1 + 2.0 ** -20)
        # points of the box, the nearest corner first
        near = np.clip(q, lo, hi)
        p = np.concatenate([near[None], rng.integers(lo, hi + 1, size=(200, 3))])
        d = p - q
        e = est3(d[:, 0], d[:, 1], d[:, 2])
        assert np.all(e > band), trial
