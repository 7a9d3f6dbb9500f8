"""Seeded synthetic workloads (numpy ``default_rng``).

This module only draws random inputs: it holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle can consume its arrays.

The paper benchmarks uniform points in a square / cube and a few skewed
distributions (Sec. 4 "Test data"); its generators are not available, so
these recipes stand in for them with the same shapes:

* ``uniform``      -- int32 points uniform in [0, 2^bits)^dim.
* ``clustered``    -- isotropic Gaussian clusters: centres uniform in the cube,
  sigma log-uniform in [2^lo, 2^hi], points assigned to clusters by a
  multinomial with equal weights, rounded to nearest and clipped to the cube.
* ``mixed_cloud``  -- one cloud of the batched workload: a uniform fraction
  f ~ U[0, 1], the rest in 1..8 Gaussian clusters (sigma log-uniform in
  [2^6, 2^12]), clipped to [0, 2^16)^3.
* ``warped_pair``  -- a pair of float32 clouds, N(0, 1) coordinates pushed
  through one random affine map x -> R diag(s) x + t (R a random rotation,
  s log-uniform in [0.5, 2], t ~ N(0, 1)).
* ``plummer``      -- 3D Plummer sphere (the paper's skewed 3D set, Sec. 5
  "Test data"): radius from the inverted cumulative mass profile, isotropic
  direction, truncated and scaled onto the integer grid.
* ``kuzmin``       -- 2D Kuzmin disc (the paper's skewed 2D set): radius from
  the inverted cumulative surface mass, uniform angle, truncated and scaled.
* ``on_sphere``    -- points on the surface of a sphere (the paper's 3D
  "on sphere" set), rounded to the grid.
"""
from __future__ import annotations

import numpy as np


def uniform(rng: np.random.Generator, n: int, dim: int, bits: int = 20) -> np.ndarray:
    return rng.integers(0, 1 << bits, size=(n, dim), dtype=np.int32)


def clustered(rng: np.random.Generator, n: int, dim: int = 3, n_clusters: int = 1000,
              bits: int = 20, log2_sigma=(8.0, 14.0)) -> np.ndarray:
    top = (1 << bits) - 1
    centres = rng.integers(0, 1 << bits, size=(n_clusters, dim)).astype(np.float64)
    sigma = 2.0 ** rng.uniform(log2_sigma[0], log2_sigma[1], size=n_clusters)
    counts = rng.multinomial(n, np.full(n_clusters, 1.0 / n_clusters))
    which = np.repeat(np.arange(n_clusters), counts)
    out = np.empty((n, dim), np.int32)
    chunk = 1 << 22
    for s in range(0, n, chunk):
        w = which[s:s + chunk]
        x = centres[w] + sigma[w, None] * rng.standard_normal((len(w), dim))
        out[s:s + chunk] = np.clip(np.rint(x), 0, top).astype(np.int32)
    return out


def mixed_cloud(rng: np.random.Generator, n: int, bits: int = 16) -> np.ndarray:
    top = (1 << bits) - 1
    f = rng.uniform(0.0, 1.0)
    n_uni = int(round(f * n))
    n_cl = n - n_uni
    parts = [rng.integers(0, 1 << bits, size=(n_uni, 3)).astype(np.float64)]
    if n_cl > 0:
        nc = int(rng.integers(1, 9))
        centres = rng.uniform(0, 1 << bits, size=(nc, 3))
        sigma = 2.0 ** rng.uniform(6.0, 12.0, size=nc)
        w = rng.integers(0, nc, size=n_cl)
        parts.append(centres[w] + sigma[w, None] * rng.standard_normal((n_cl, 3)))
    x = np.concatenate(parts)
    return np.clip(np.rint(x), 0, top).astype(np.int32)


def random_rotation(rng: np.random.Generator, dim: int = 3) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((dim, dim)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def warped_pair(rng: np.random.Generator, na: int, nb: int, dim: int = 3):
    R = random_rotation(rng, dim)
    s = 2.0 ** rng.uniform(-1.0, 1.0, size=dim)
    t = rng.standard_normal(dim)
    M = R @ np.diag(s)
    a = rng.standard_normal((na, dim)) @ M.T + t
    b = rng.standard_normal((nb, dim)) @ M.T + t
    return a.astype(np.float32), b.astype(np.float32)


def _isotropic(rng: np.random.Generator, n: int, dim: int) -> np.ndarray:
    """Unit vectors uniform on the sphere (normalised Gaussian vectors)."""
    v = rng.standard_normal((n, dim))
    nrm = np.linalg.norm(v, axis=1)
    bad = nrm == 0
    while bad.any():
        v[bad] = rng.standard_normal((int(bad.sum()), dim))
        nrm[bad] = np.linalg.norm(v[bad], axis=1)
        bad = nrm == 0
    return v / nrm[:, None]


def _truncated_radii(rng: np.random.Generator, n: int, inv_cdf, r_max: float) -> np.ndarray:
    """Radii drawn by inverting a cumulative mass profile, redrawn above r_max."""
    r = inv_cdf(rng.uniform(0.0, 1.0, n))
    bad = ~(r <= r_max)
    while bad.any():
        r[bad] = inv_cdf(rng.uniform(0.0, 1.0, int(bad.sum())))
        bad = ~(r <= r_max)
    return r


def _to_grid(x: np.ndarray, bits: int) -> np.ndarray:
    top = (1 << bits) - 1
    return np.clip(np.rint(x), 0, top).astype(np.int32)


def plummer(rng: np.random.Generator, n: int, bits: int = 20, r_max: float = 256.0) -> np.ndarray:
    """Plummer sphere of scale radius 1: the mass inside radius r is
    r^3 / (1 + r^2)^(3/2), so r = (u^(-2/3) - 1)^(-1/2) for u ~ U(0, 1)
    (Aarseth, Henon and Wielen 1974).  Radii above r_max scale radii are
    redrawn; the ball of radius r_max fills the grid [0, 2^bits)^3."""
    def inv(u):
        with np.errstate(divide="ignore", invalid="ignore"):
            return 1.0 / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    half = (1 << (bits - 1)) - 1
    r = _truncated_radii(rng, n, inv, r_max)
    x = (1 << (bits - 1)) + _isotropic(rng, n, 3) * (r * (half / r_max))[:, None]
    return _to_grid(x, bits)


def kuzmin(rng: np.random.Generator, n: int, bits: int = 30, r_max: float = 4096.0) -> np.ndarray:
    """Kuzmin disc of scale length 1: the mass inside radius R is
    1 - 1 / sqrt(1 + R^2), so R = sqrt((1 - u)^(-2) - 1) for u ~ U(0, 1).
    Radii above r_max scale lengths are redrawn; the disc of radius r_max
    fills the grid [0, 2^bits)^2."""
    def inv(u):
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.sqrt((1.0 - u) ** -2.0 - 1.0)
    half = (1 << (bits - 1)) - 1
    r = _truncated_radii(rng, n, inv, r_max)
    x = (1 << (bits - 1)) + _isotropic(rng, n, 2) * (r * (half / r_max))[:, None]
    return _to_grid(x, bits)


def on_sphere(rng: np.random.Generator, n: int, bits: int = 20) -> np.ndarray:
    """Points uniform on the sphere inscribed in [0, 2^bits)^3."""
    half = (1 << (bits - 1)) - 1
    return _to_grid((1 << (bits - 1)) + _isotropic(rng, n, 3) * half, bits)


# --------------------------------------------------------------------------
# The five workloads.  Each returns plain numpy arrays plus its parameters.
# --------------------------------------------------------------------------

def workload_2d_uniform(n: int = 100_000, seed: int = 0):
    """2D, int32 uniform in [0, 2^20)^2, L = 16, all-points k = 10."""
    rng = np.random.default_rng(seed)
    return dict(pts=uniform(rng, n, 2, 20), dim=2, coord_bits=20, leaf_size=16, k=10)


def workload_3d_clustered(n: int = 10_000_000, seed: int = 1, n_clusters: int = 1000):
    """3D, int32 in [0, 2^20)^3 from 1000 Gaussian clusters, L = 16, k = 10."""
    rng = np.random.default_rng(seed)
    return dict(pts=clustered(rng, n, 3, n_clusters, 20), dim=3, coord_bits=21, leaf_size=16, k=10)


def workload_3d_uniform(n: int = 10_000_000, k: int = 100, seed: int = 5):
    """3D, int32 uniform in [0, 2^20)^3, L = 16: the uniform cube of the
    paper's k sweep (Sec. 5, k up to 100), at a large k."""
    rng = np.random.default_rng(seed)
    return dict(pts=uniform(rng, n, 3, 20), dim=3, coord_bits=21, leaf_size=16, k=k)


# The five point sets of the paper's search-start comparison (Sec. 5, k = 1):
# name -> (generator, dim, coord_bits of the tree, seed).
SKEWED_SETS = {
    "2DinCube": (lambda rng, n: uniform(rng, n, 2, 20), 2, 20, 6),
    "2Dkuzmin": (lambda rng, n: kuzmin(rng, n, 30), 2, 30, 7),
    "3DonSphere": (lambda rng, n: on_sphere(rng, n, 20), 3, 21, 8),
    "3DinCube": (lambda rng, n: uniform(rng, n, 3, 20), 3, 21, 9),
    "3Dplummer": (lambda rng, n: plummer(rng, n, 20), 3, 21, 10),
}


def workload_skewed(name: str, n: int = 10_000_000, k: int = 1):
    """One of the five point sets of the search-start comparison; L = 16."""
    gen, dim, bits, seed = SKEWED_SETS[name]
    rng = np.random.default_rng(seed)
    return dict(pts=gen(rng, n), dim=dim, coord_bits=bits, leaf_size=16, k=k, name=name)


class DynamicWorkload:
    """3D batch-dynamic workload: an initial uniform set, then rounds of
    (insert a uniform batch, delete random live ids, query uniform points).
    Deleted ids are drawn uniformly without replacement from the ids live
    after that round's insert; ids are assigned sequentially from n0."""

    def __init__(self, n0: int = 50_000_000, batch: int = 1_000_000, n_queries: int = 1_000_000,
                 rounds: int = 20, seed: int = 2):
        self.rng = np.random.default_rng(seed)
        self.n0, self.batch, self.n_queries, self.rounds = n0, batch, n_queries, rounds
        self.dim, self.coord_bits, self.leaf_size, self.k = 3, 21, 16, 5
        self.initial = uniform(self.rng, n0, 3, 20)
        self.live = np.arange(n0, dtype=np.int64)
        self.next_id = n0

    def round(self):
        ins = uniform(self.rng, self.batch, 3, 20)
        new_ids = np.arange(self.next_id, self.next_id + self.batch, dtype=np.int64)
        self.next_id += self.batch
        self.live = np.concatenate([self.live, new_ids])
        pick = self.rng.choice(len(self.live), size=min(self.batch, len(self.live)), replace=False)
        dele = self.live[pick].astype(np.int32)
        mask = np.ones(len(self.live), bool)
        mask[pick] = False
        self.live = self.live[mask]
        q = uniform(self.rng, self.n_queries, 3, 20)
        return ins, dele, q


def workload_batched(n_clouds: int = 4096, seed: int = 3, size_range=(1024, 65536)):
    """4096 independent 3D clouds, sizes uniform in [1024, 65536], int32 in
    [0, 2^16)^3, k = 16.  Returns the concatenated points and CSR offsets."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(size_range[0], size_range[1] + 1, size=n_clouds)
    offsets = np.zeros(n_clouds + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    pts = np.empty((int(offsets[-1]), 3), np.int32)
    for c in range(n_clouds):
        pts[offsets[c]:offsets[c + 1]] = mixed_cloud(rng, int(sizes[c]), 16)
    return dict(pts=pts, offsets=offsets, dim=3, coord_bits=16, k=16)


def workload_differentiable(n_pairs: int = 64, na: int = 16384, nb: int = 32768, seed: int = 4):
    """64 pairs of 3D float32 clouds (A: 16384 points, B: 32768), k = 8."""
    rng = np.random.default_rng(seed)
    A = np.empty((n_pairs, na, 3), np.float32)
    B = np.empty((n_pairs, nb, 3), np.float32)
    for p in range(n_pairs):
        A[p], B[p] = warped_pair(rng, na, nb, 3)
    return dict(A=A, B=B, k=8, dim=3, coord_bits=21, leaf_size=16)
