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
    seen = {so.zd_status_string(i) for i in range(10)}
    assert len(seen) == 10 and b"unknown status" not in seen


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
