"""Host-side pieces of bench.py and the committed profile summaries (no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_headline_config_keys(bench):
    c = bench.headline_config(10_000_000, 10, 16, 21, "1 GPU")
    assert c["workload"] == "3d-clustered-1e7"
    for key in ("n", "dim", "k", "leaf_size", "coord_bits", "l2", "parallelism"):
        assert key in c


def test_algorithmic_bytes(bench):
    assert bench.knn_bytes_per_query(10) == 148
    assert bench.knn_bytes_per_query(100) == 1228
    assert bench.build_bytes_per_point() == 276
    assert bench.knn_bytes_per_query(10, dim=2) == 144
    assert bench.knn_bytes_per_query(8, dist_bytes=4, own_id=False) == 24 + 64
    assert bench.sort_passes(63) == 8 and bench.sort_passes(40) == 5 and bench.sort_passes(64) == 8
    assert bench.update_bytes(1, 1) == 276 + 512 + 48
    r = bench.roofline("k", 2e9, 1.0)
    assert abs(r["achieved"] - 2000.0) < 1e-9 and abs(r["frac"] - 2000.0 / r["peak"]) < 1e-12


def test_profiled_traffic_follows_the_sources(bench, tmp_path, monkeypatch):
    """A traffic line counts only while its source digest matches."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    src = tmp_path / "k.cuh"
    src.write_text("kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    dig = bench.source_digest(["k.cuh"])
    (prof / "p.md").write_text("traffic_bytes_per_launch: 123 source: %s kernel: kk workload: ww\n" % dig)
    assert bench.profiled_traffic("kk", "ww", "p.md", ["k.cuh"]) == 123
    assert bench.profiled_traffic("kk", "other", "p.md", ["k.cuh"]) is None
    src.write_text("kernel v2")
    assert bench.profiled_traffic("kk", "ww", "p.md", ["k.cuh"]) is None


def test_profile_commands_run_committed_files():
    """Every command quoted in profiles/ runs a committed file, never a
    scratch one."""
    pdir = os.path.join(ROOT, "profiles")
    for f in os.listdir(pdir):
        text = open(os.path.join(pdir, f)).read()
        assert "_work" not in text, f
        for m in re.finditer(r"python (\S+\.py)", text):
            assert os.path.exists(os.path.join(ROOT, m.group(1))), (f, m.group(1))


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` (the oracle on the host cores) runs
    without a GPU and prints the contract's keys."""
    import json
    import subprocess
    import sys
    import time
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "0", "--n", "20000"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    wall = time.perf_counter() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    # the reported time per step is a measured one: the steps fit in the run
    assert d["ms_per_step"] * d["steps"] / 1e3 <= wall
    assert abs(d["value"] - 20000 / (d["ms_per_step"] / 1e3)) <= 1e-6 * d["value"]
