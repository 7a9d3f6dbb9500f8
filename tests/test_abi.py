"""The C-ABI library builds, loads and exports every entry point that
include/zd.h declares (no compute: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "zd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(zd_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_04182_gb300 import build_lib
    path = build_lib.build()
    import ctypes
    return path, ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared()
    for must in ("zd_build", "zd_knn", "zd_insert_batch", "zd_delete_batch", "zd_knn_dist_backward",
                 "zd_morton_encode", "zd_morton_sort", "zd_build_batched", "zd_knn_batched"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    path, so = lib
    for name in declared():
        assert hasattr(so, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (zd_\w+)", out))
    assert set(declared()) <= exported


def test_binding_names_match_header(lib):
    from paper_2111_04182_gb300 import zd
    assert sorted(zd.EXPORTED) == declared()


def test_status_strings(lib):
    import ctypes
    _, so = lib
    so.zd_status_string.restype = ctypes.c_char_p
    seen = {so.zd_status_string(i) for i in range(11)}
    assert len(seen) == 11 and b"unknown status" not in seen


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2111_04182_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).lower() or f == "datagen.py", f


def test_no_host_fallback_without_library(tmp_path, monkeypatch):
    from paper_2111_04182_gb300 import zd
    monkeypatch.setattr(zd, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(zd, "_LIB", None)
    with pytest.raises(RuntimeError):
        zd._lib()


def test_binding_constants_match_header():
    """Every integer constant of the header (enum members and #defines) has
    the same value in the Python binding."""
    from paper_2111_04182_gb300 import zd
    src = open(os.path.join(ROOT, "include", "zd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\w*\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"\b(ZD_\w+)\s*=\s*([^,\s]+)", body):
            consts[name] = int(val, 0)
    for name, val, sh in re.findall(r"#define\s+(ZD_\w+)[ \t]+\(?([0-9x]+)(?:\s*<<\s*(\d+))?", src):
        consts[name] = int(val, 0) << int(sh or 0)
    assert len(consts) > 15
    for name, val in consts.items():
        assert getattr(zd, name) == val, name


def test_bench_runs_the_oracle_only_for_the_cpu_baseline():
    """bench.py imports the oracle in its CPU-baseline function only."""
    text = open(os.path.join(ROOT, "bench.py")).read()
    funcs = re.split(r"\ndef ", text)
    users = [f.split("(")[0] for f in funcs if "from oracle import" in f or "import oracle" in f]
    assert users == ["cpu_baseline"], users


def test_size_limits_rejected_on_the_host(lib):
    """Sizes beyond ZD_MAX_KEYS (the radix sort's look-back words count a
    digit's running total in 30 bits) return ZD_ERR_CAPACITY before any CUDA
    call, so this runs without a GPU.  The device pointers are never touched."""
    import ctypes as C
    from paper_2111_04182_gb300 import zd
    so = zd._lib()
    fake = C.c_void_p(0x1000)
    big = zd.ZD_MAX_KEYS + 1
    assert so.zd_morton_sort(fake, big, 63, fake, fake, None, None) == zd.ZD_ERR_CAPACITY
    p = zd.ZdParams(dim=3, leaf_size=16, coord_bits=21, coord_type=zd.ZD_COORD_I32)
    h = C.c_void_p()
    assert so.zd_build(C.byref(p), None, fake, big, None, C.byref(h)) == zd.ZD_ERR_CAPACITY
    p.capacity = big
    assert so.zd_build(C.byref(p), None, fake, 10, None, C.byref(h)) == zd.ZD_ERR_CAPACITY
    assert not h.value
    p.capacity = 0
    off = (C.c_int64 * 2)(0, big)
    assert so.zd_build_batched(C.byref(p), None, fake, off, fake, 1, None, C.byref(h)) == zd.ZD_ERR_CAPACITY
    one = C.c_float(1.0)
    # 2^27 * 8 pairs of (query, neighbour) > ZD_MAX_KEYS
    assert so.zd_knn_dist_backward(fake, fake, fake, 1, 1 << 27, 16, 3, 8, C.byref(one), 0, fake, fake,
                                   None) == zd.ZD_ERR_CAPACITY
    assert so.zd_knn_dist_backward(fake, fake, fake, 1 << 40, 1 << 40, 16, 3, 8, C.byref(one), 0, fake,
                                   fake, None) == zd.ZD_ERR_CAPACITY


def test_debug_checks_compile(tmp_path):
    """The -DZD_DEBUG variant of the kernels compiles (the debug library is
    built on the GPU machine by build_lib.build(debug=True))."""
    from paper_2111_04182_gb300 import build_lib
    for src in ("sort.cu", "build.cu"):
        cmd = [build_lib.nvcc()] + build_lib.ARCH + build_lib.FLAGS + ["-DZD_DEBUG", "-c",
                                                                      os.path.join(build_lib.CSRC, src),
                                                                      "-o", str(tmp_path / (src + ".o"))]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-3000:]
