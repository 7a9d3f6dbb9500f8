"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a swapped
bit order, an off-by-one margin, a reversed tie-break, a dropped term, a wrong
sign ...), builds the copy on the CPU, and runs a quick subset of the pins of
tests/test_oracle.py against it.  The unmodified oracle must pass that subset
and every mutant must fail it.
"""
import importlib.util
import json
import os
import shutil

import numpy as np
import pytest

from tests._checks import brute_knn, check_tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "hand_examples.json")))

MUTATIONS = {
    "z-major bit order": ("for (int j = 0; j < dim; ++j)\n            key = (key << 1)",
                          "for (int j = dim - 1; j >= 0; --j)\n            key = (key << 1)"),
    "climb margin off by one": ("q->ic[j] - v->ibox_lo[j] + 1", "q->ic[j] - v->ibox_lo[j] + 2"),
    "tie-break by larger id": ("return d2 < wd || (d2 == wd && id < wi);\n}\nstatic int kb_accepts_f",
                               "return d2 < wd || (d2 == wd && id > wi);\n}\nstatic int kb_accepts_f"),
    "strict box pruning": ("return s <= N->i2[N->k - 1];", "return s < N->i2[N->k - 1];"),
    "dropped last coordinate": ("for (int j = 0; j < dim; ++j) s += (a[j] - b[j]) * (a[j] - b[j]);",
                                "for (int j = 0; j + 1 < dim; ++j) s += (a[j] - b[j]) * (a[j] - b[j]);"),
    "leaf holds fewer than L": ("if (hi - lo <= t->leaf_size || b == 0)", "if (hi - lo < t->leaf_size || b == 0)"),
    "split on the wrong bit": ("int64_t s = split_using_bit(t->keys, lo, hi, b - 1);",
                               "int64_t s = split_using_bit(t->keys, lo, hi, b > 1 ? b - 2 : 0);"),
    "gradient sign of the reference": ("gb[(int64_t)t * dim + c] -= u;", "gb[(int64_t)t * dim + c] += u;"),
    "self not excluded": ("if (q->self_id >= 0 && id == q->self_id) return;", "if (0) return;"),
    "internal box from one child": ("x->ibox_hi[j] = l->ibox_hi[j] > r->ibox_hi[j] ? l->ibox_hi[j] : r->ibox_hi[j];",
                                    "x->ibox_hi[j] = l->ibox_hi[j];"),
    "float distance keeps last term only": ("        s = (j == 0) ? sq : s + sq;\n    }\n    return s;\n}\n\n/* Consider",
                                            "        s = sq;\n    }\n    return s;\n}\n\n/* Consider"),
    "sort ties by descending id": ("if (x->id != y->id) return x->id < y->id ? -1 : 1;",
                                   "if (x->id != y->id) return x->id < y->id ? 1 : -1;"),
    "wrong child searched while climbing": ("search_down(t, P->left == c ? P->right : P->left, q, N);",
                                            "search_down(t, P->left == c ? P->left : P->right, q, N);"),
    "quantize rounds instead of flooring": ("double v = floor(((double)pts[i * dim + j] - lo[j]) * scale);",
                                            "double v = round(((double)pts[i * dim + j] - lo[j]) * scale);"),
    "quantize in fp32": ("double v = floor(((double)pts[i * dim + j] - lo[j]) * scale);",
                         "double v = floor((float)((float)pts[i * dim + j] - (float)lo[j]) * (float)scale);"),
    "quantize clamps at 2^B": ("const double top = (double)(((int64_t)1 << coord_bits) - 1);",
                               "const double top = (double)((int64_t)1 << coord_bits);"),
    # the frame lives in the Python half of the oracle
    "per-axis scale (last axis's extent)": ("oracle.py", "ext = float(np.max(hi - lo))", "ext = float((hi - lo)[-1])"),
    "one minimum for all axes": ("oracle.py", "lo = pts.min(axis=0).astype(np.float64)",
                                 "lo = np.full(pts.shape[1], pts.min(), np.float64)"),
}


def _load_variant(tmp, name, mutate=None):
    d = os.path.join(tmp, name.replace(" ", "_"))
    os.makedirs(d)
    files = {f: open(os.path.join(ROOT, "oracle", f)).read() for f in ("zd_oracle.c", "oracle.py")}
    if mutate:
        target, old, new = mutate if len(mutate) == 3 else ("zd_oracle.c",) + tuple(mutate)
        assert files[target].count(old) >= 1, "mutation anchor not found: %r" % old[:60]
        files[target] = files[target].replace(old, new, 1)
    for f, src in files.items():
        open(os.path.join(d, f), "w").write(src)
    spec = importlib.util.spec_from_file_location("oracle_" + os.path.basename(d), os.path.join(d, "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


def _quantize_pins(o) -> bool:
    for case in GOLD["quantize"]["frames"]:
        pts = np.array(case["pts"], np.float32)
        lo, scale = o.quantization_of(pts, case["bits"])
        if lo.tolist() != case["lo"] or scale != case["scale"]:
            return False
        if o.quantize(pts, lo, scale, case["bits"]).tolist() != case["q"]:
            return False
        e = o.OracleTree(pts, 1, case["bits"], qlo=lo, qscale=scale).export()
        if [int(e["keys"][i]) for i in np.argsort(e["ids"])] != [int(k) for k in case["keys"]]:
            return False
    for case in GOLD["quantize"]["explicit"]:
        pts = np.array([[float(v) for v in r] for r in case["pts"]], np.float32)
        if o.quantize(pts, np.array(case["lo"]), case["scale"], case["bits"]).tolist() != case["q"]:
            return False
    return True


def _pins(o) -> bool:
    """A quick subset of the pins; True iff all hold."""
    try:
        if not _quantize_pins(o):
            return False
        for case in GOLD["morton"]["cases"]:
            if max(case["pt"]) >= 2 ** 31:
                continue
            k = o.morton_keys(np.array([case["pt"]], np.int32), case["bits"], case["shift"])
            if int(k[0]) != int(case["key"]):
                return False
        for case in GOLD["trees"]["cases"]:
            t = o.OracleTree(np.array(case["pts"], np.int32), case["L"], case["bits"])
            d = t.canonical_dump()
            got = sorted(zip(d["lo"].tolist(), d["hi"].tolist(), d["bit"].tolist()))
            if [list(g) for g in got] != sorted(case["nodes"]) or d["ids"].tolist() != case["sorted_ids"]:
                return False
        rng = np.random.default_rng(5)
        for dim in (2, 3):
            pts = rng.integers(0, 2 ** 10, size=(700, dim)).astype(np.int32)
            pts[:60] = pts[60:120]
            for L in (1, 6):
                t = o.OracleTree(pts, L, 10)
                e = t.export()
                check_tree(e["keys"], e["lo"], e["hi"], e["bit"], L, coords=pts[e["ids"].astype(np.int64)],
                           box_lo=e["box_lo"], box_hi=e["box_hi"], left=e["left"], right=e["right"],
                           parent=e["parent"], root=e["root"])
                idx, d2 = t.knn(5)
                bi, bd = brute_knn(pts, 5)
                if not (np.array_equal(idx, bi) and np.array_equal(d2, bd)):
                    return False
                q = rng.integers(0, 2 ** 10, size=(80, dim)).astype(np.int32)
                for mode in (1, 2):
                    idx, d2 = t.knn(4, queries=q, mode=mode)
                    bi, bd = brute_knn(pts, 4, queries=q)
                    if not (np.array_equal(idx, bi) and np.array_equal(d2, bd)):
                        return False
                ci, cd = o.knn_brute(pts, 5)
                bi, bd = brute_knn(pts, 5)
                if not (np.array_equal(ci, bi) and np.array_equal(cd, bd)):
                    return False
        # unit lattice: neighbours sit exactly one step outside leaf boxes
        for dim in (2, 3):
            g = np.stack(np.meshgrid(*[np.arange(6)] * dim, indexing="ij"), -1).reshape(-1, dim).astype(np.int32)
            t = o.OracleTree(g, 4, 4)
            idx, d2 = t.knn(2 * dim + 2)
            bi, bd = brute_knn(g, 2 * dim + 2)
            if not (np.array_equal(idx, bi) and np.array_equal(d2, bd)):
                return False
        a = rng.standard_normal((60, 3)).astype(np.float32)
        b = rng.standard_normal((150, 3)).astype(np.float32)
        bi, bd = brute_knn(b, 4, queries=a)
        ci, cd = o.knn_brute(b, 4, queries=a)
        if not (np.array_equal(ci, bi) and np.array_equal(cd, bd)):
            return False
        loss, ga, gb = o.knn_dist_grad(a, b, bi)
        A, B = a.astype(np.float64), b.astype(np.float64)

        def L64(A, B):
            dd = A[:, None, :] - B[bi]
            return np.sqrt((dd * dd).sum(-1)).sum()
        h = 1e-6
        for (arr, g, which) in ((A, ga, 0), (B, gb, 1)):
            for i in (int(bi[0, 0]) if which else 0, int(bi[3, 1]) if which else 5):
                for c in range(3):
                    P, M = arr.copy(), arr.copy()
                    P[i, c] += h
                    M[i, c] -= h
                    fd = ((L64(P, B) - L64(M, B)) if which == 0 else (L64(A, P) - L64(A, M))) / (2 * h)
                    if abs(fd - g[i, c]) > 1e-6 * max(1.0, abs(fd)):
                        return False
        return True
    except AssertionError:
        return False


@pytest.fixture(scope="module")
def tmp(tmp_path_factory):
    return str(tmp_path_factory.mktemp("mutants"))


def test_unmodified_oracle_passes_the_pins(tmp):
    assert _pins(_load_variant(tmp, "base"))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_each_planted_mistake_is_caught(tmp, name):
    assert not _pins(_load_variant(tmp, name, MUTATIONS[name])), "pins missed: " + name
