"""The seeded input generators: deterministic, inside the grid, and with the
mass profiles they are drawn from (checked on a sample)."""
import numpy as np
import pytest

from paper_2111_04182_gb300 import datagen


@pytest.mark.parametrize("name", sorted(datagen.SKEWED_SETS))
def test_skewed_sets_deterministic_and_in_range(name):
    a = datagen.workload_skewed(name, n=20_000)
    b = datagen.workload_skewed(name, n=20_000)
    assert np.array_equal(a["pts"], b["pts"])
    p = a["pts"]
    assert p.dtype == np.int32 and p.shape == (20_000, a["dim"])
    assert p.min() >= 0 and p.max() < 2 ** (a["coord_bits"] - (a["dim"] == 3 and a["coord_bits"] == 21))


def test_plummer_mass_profile():
    # mass inside r scale radii: r^3 / (1 + r^2)^(3/2); 1/2^(3/2) inside r = 1
    rng = np.random.default_rng(0)
    p = datagen.plummer(rng, 400_000, 20, r_max=256.0).astype(np.float64)
    scale = ((1 << 19) - 1) / 256.0
    r = np.linalg.norm(p - (1 << 19), axis=1) / scale
    for rr in (0.5, 1.0, 3.0):
        want = rr ** 3 / (1 + rr * rr) ** 1.5
        assert abs(np.mean(r <= rr) - want) < 0.005, rr


def test_kuzmin_mass_profile():
    # mass inside R scale lengths: 1 - 1 / sqrt(1 + R^2)
    rng = np.random.default_rng(1)
    p = datagen.kuzmin(rng, 400_000, 30, r_max=4096.0).astype(np.float64)
    scale = ((1 << 29) - 1) / 4096.0
    r = np.linalg.norm(p - (1 << 29), axis=1) / scale
    for rr in (0.5, 1.0, 10.0):
        want = 1 - 1 / np.sqrt(1 + rr * rr)
        assert abs(np.mean(r <= rr) - want) < 0.005, rr


def test_on_sphere_radius():
    p = datagen.on_sphere(np.random.default_rng(2), 50_000, 20).astype(np.float64)
    r = np.linalg.norm(p - (1 << 19), axis=1)
    assert np.all(np.abs(r - ((1 << 19) - 1)) <= 1.0)
