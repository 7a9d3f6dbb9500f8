"""ctypes wrapper of the plain CPU oracle (``zd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the product library never imports it.
It shares no code with the CUDA path.

Paper references (Blelloch & Dobson, "Parallel Nearest Neighbors in Low
Dimensions with Batch Updates"):

* ``morton_keys`` -- Sec. 1.1 "Morton ordering", Sec. 2 "Construction".
* ``OracleTree`` -- Algorithm 1 with the empty-cut pruning of Sec. 2.1;
  ``knn`` runs Algorithm 3 (leaf- and bit-based) or Algorithm 2 (root-based).
* ``knn_brute`` -- the plain definition of exact k-NN.
* ``OracleSet`` -- batch insert / delete (Sec. 2 "Batch-dynamic updates",
  Algorithm 4), read as: after any update the tree equals a fresh build of the
  current point set.
* ``knn_dist_grad`` -- fp64 gradient of a sum of k-NN distances.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, ERR_INVALID, ERR_RANGE, ERR_OOM = 0, 1, 2, 3
MODE_LEAF, MODE_BIT, MODE_ROOT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (fp contraction off, OpenMP over queries)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        vp, i64, i32, f64 = C.c_void_p, C.c_int64, C.c_int, C.c_double
        lib.zdo_morton_keys_i32.argtypes = [vp, i64, i32, i32, vp, vp]
        lib.zdo_quantize_f32.argtypes = [vp, i64, i32, vp, f64, i32, vp]
        lib.zdo_sort_perm.argtypes = [vp, vp, i64, vp]
        lib.zdo_build.argtypes = [vp, vp, vp, i64, i32, i32, vp, vp, f64, i32, C.POINTER(C.c_int)]
        lib.zdo_build.restype = vp
        lib.zdo_free.argtypes = [vp]
        lib.zdo_num_nodes.argtypes = [vp]
        lib.zdo_num_nodes.restype = i64
        lib.zdo_root.argtypes = [vp]
        lib.zdo_root.restype = i64
        lib.zdo_export.argtypes = [vp] + [vp] * 12
        lib.zdo_knn.argtypes = [vp, vp, vp, i64, i32, i32, i64, i64, vp, vp, vp, i32]
        lib.zdo_knn_brute.argtypes = [vp, vp, vp, i64, vp, vp, vp, i64, i32, i32, vp, vp, vp, i32]
        lib.zdo_knn_dist_grad.argtypes = [vp, vp, vp, i64, i64, i32, i32, vp, i32, vp, vp]
        lib.zdo_knn_dist_grad.restype = f64
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _shift3(shift):
    s = np.zeros(3, np.uint32)
    if shift is not None:
        s[: len(shift)] = np.asarray(shift, np.uint32)
    return s


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__("oracle status %d" % code)
        self.code = code


def morton_keys(pts: np.ndarray, coord_bits: int, shift=None) -> np.ndarray:
    """Morton keys of int32 points [n, dim] (Sec. 1.1)."""
    pts = np.ascontiguousarray(pts, np.int32)
    n, dim = pts.shape
    keys = np.empty(n, np.uint64)
    st = _load().zdo_morton_keys_i32(_p(pts), n, dim, coord_bits, _p(_shift3(shift)), _p(keys))
    if st:
        raise OracleError(st)
    return keys


def quantize(pts: np.ndarray, lo: np.ndarray, scale: float, coord_bits: int) -> np.ndarray:
    """Float points -> integer grid that feeds the Morton keys (Sec. 3.1)."""
    pts = np.ascontiguousarray(pts, np.float32)
    n, dim = pts.shape
    out = np.empty((n, dim), np.int32)
    lo = np.ascontiguousarray(lo, np.float64)
    st = _load().zdo_quantize_f32(_p(pts), n, dim, _p(lo), float(scale), coord_bits, _p(out))
    if st:
        raise OracleError(st)
    return out


def quantization_of(pts: np.ndarray, coord_bits: int):
    """The float-mode quantization frame: per-dimension minimum and one common
    scale (2^bits - 1) / (largest extent), all in fp64."""
    pts = np.asarray(pts, np.float32)
    lo = pts.min(axis=0).astype(np.float64)
    hi = pts.max(axis=0).astype(np.float64)
    ext = float(np.max(hi - lo))
    scale = float(((1 << coord_bits) - 1) / ext) if ext > 0 else 1.0
    return lo, scale


def sort_perm(keys: np.ndarray, ids=None) -> np.ndarray:
    """Positions in (key, id) order (Sec. 2 "Construction")."""
    keys = np.ascontiguousarray(keys, np.uint64)
    ids = None if ids is None else np.ascontiguousarray(ids, np.int32)
    perm = np.empty(len(keys), np.int64)
    st = _load().zdo_sort_perm(_p(keys), _p(ids), len(keys), _p(perm))
    if st:
        raise OracleError(st)
    return perm


class OracleTree:
    """The canonical pruned zd-tree built by Algorithm 1."""

    def __init__(self, pts, leaf_size: int, coord_bits: int, shift=None, ids=None,
                 qlo=None, qscale: float = 1.0):
        lib = _load()
        self.is_float = np.asarray(pts).dtype.kind == "f"
        if self.is_float:
            self.pts = np.ascontiguousarray(pts, np.float32)
        else:
            self.pts = np.ascontiguousarray(pts, np.int32)
        self.n, self.dim = self.pts.shape
        self.leaf_size, self.coord_bits = leaf_size, coord_bits
        self.shift = _shift3(shift)
        self.ids_in = None if ids is None else np.ascontiguousarray(ids, np.int32)
        self.qlo = None if qlo is None else np.ascontiguousarray(qlo, np.float64)
        self.qscale = float(qscale)
        st = C.c_int(0)
        self._h = lib.zdo_build(None if self.is_float else _p(self.pts),
                                _p(self.pts) if self.is_float else None,
                                _p(self.ids_in), self.n, self.dim, coord_bits, _p(self.shift),
                                _p(self.qlo), self.qscale, leaf_size, C.byref(st))
        if not self._h:
            raise OracleError(st.value)
        self.nnodes = lib.zdo_num_nodes(self._h)
        self.root = lib.zdo_root(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.zdo_free(h)
            self._h = None

    def export(self) -> dict:
        """Sorted keys / ids and every node's (lo, hi, bit, children, parent, box)."""
        n, v, d = self.n, self.nnodes, self.dim
        out = dict(keys=np.empty(n, np.uint64), ids=np.empty(n, np.int32),
                   lo=np.empty(v, np.int64), hi=np.empty(v, np.int64), bit=np.empty(v, np.int32),
                   left=np.empty(v, np.int64), right=np.empty(v, np.int64),
                   parent=np.empty(v, np.int64))
        if self.is_float:
            out["box_lo"] = np.empty((v, d), np.float64)
            out["box_hi"] = np.empty((v, d), np.float64)
            ib = (None, None)
            fb = (out["box_lo"], out["box_hi"])
        else:
            out["box_lo"] = np.empty((v, d), np.int64)
            out["box_hi"] = np.empty((v, d), np.int64)
            ib = (out["box_lo"], out["box_hi"])
            fb = (None, None)
        _lib.zdo_export(self._h, _p(out["keys"]), _p(out["ids"]), _p(out["lo"]), _p(out["hi"]),
                        _p(out["bit"]), _p(out["left"]), _p(out["right"]), _p(out["parent"]),
                        _p(ib[0]), _p(ib[1]), _p(fb[0]), _p(fb[1]))
        out["root"] = self.root
        return out

    def canonical_dump(self) -> dict:
        """Order-free description of the tree: nodes sorted by (lo, hi)."""
        e = self.export()
        order = np.lexsort((e["hi"], e["lo"]))
        return dict(ids=e["ids"], keys=e["keys"], lo=e["lo"][order], hi=e["hi"][order],
                    bit=e["bit"][order], box_lo=e["box_lo"][order], box_hi=e["box_hi"][order])

    def knn_sorted_range(self, k: int, r0: int, r1: int, nthreads: int = 0):
        """Leaf-based k-NN (Alg. 3) of the points at sorted positions [r0, r1)
        only: rows in sorted order.  Used to time a bounded sample."""
        lib = _load()
        m = r1 - r0
        idx = np.empty((m, k), np.int32)
        d2 = None if self.is_float else np.empty((m, k), np.int64)
        d2f = np.empty((m, k), np.float64) if self.is_float else None
        st = lib.zdo_knn(self._h, None, None, m, k, MODE_LEAF, r0, r1, _p(idx), _p(d2), _p(d2f), nthreads)
        if st:
            raise OracleError(st)
        return idx, (d2f if self.is_float else d2)

    def knn(self, k: int, queries=None, mode: int = MODE_LEAF, nthreads: int = 0):
        """k-NN by the tree.  queries=None: all points (Alg. 3 from each point's
        own leaf, self excluded), rows returned in id order when the ids are
        0..n-1 (else in sorted order, with ``ids``).  Otherwise external
        queries with the bit-based (Alg. 3) or root-based (Alg. 2) start."""
        lib = _load()
        if queries is None:
            m = self.n
            idx = np.empty((m, k), np.int32)
            d2 = None if self.is_float else np.empty((m, k), np.int64)
            d2f = np.empty((m, k), np.float64) if self.is_float else None
            st = lib.zdo_knn(self._h, None, None, m, k, MODE_LEAF, 0, -1, _p(idx), _p(d2), _p(d2f),
                             nthreads)
            if st:
                raise OracleError(st)
            dist = d2f if self.is_float else d2
            ids = self.export()["ids"]
            if self.ids_in is None:
                oi, od = np.empty_like(idx), np.empty_like(dist)
                oi[ids] = idx
                od[ids] = dist
                return oi, od
            return idx, dist, ids
        if self.is_float:
            q = np.ascontiguousarray(queries, np.float32)
        else:
            q = np.ascontiguousarray(queries, np.int32)
        m = q.shape[0]
        idx = np.empty((m, k), np.int32)
        d2 = None if self.is_float else np.empty((m, k), np.int64)
        d2f = np.empty((m, k), np.float64) if self.is_float else None
        st = lib.zdo_knn(self._h, None if self.is_float else _p(q), _p(q) if self.is_float else None,
                         m, k, mode, 0, -1, _p(idx), _p(d2), _p(d2f), nthreads)
        if st:
            raise OracleError(st)
        return idx, (d2f if self.is_float else d2)


def knn_brute(ref, k: int, queries=None, ref_ids=None, query_ids=None, nthreads: int = 0):
    """Plain definition: rank all reference points by (d^2, id).  queries=None
    means all points with self (by id) excluded."""
    lib = _load()
    is_float = np.asarray(ref).dtype.kind == "f"
    dt = np.float32 if is_float else np.int32
    ref = np.ascontiguousarray(ref, dt)
    n, dim = ref.shape
    rid = None if ref_ids is None else np.ascontiguousarray(ref_ids, np.int32)
    if queries is None:
        q = ref
        qid = rid if rid is not None else np.arange(n, dtype=np.int32)
    else:
        q = np.ascontiguousarray(queries, dt)
        qid = None if query_ids is None else np.ascontiguousarray(query_ids, np.int32)
    m = q.shape[0]
    idx = np.empty((m, k), np.int32)
    d2 = None if is_float else np.empty((m, k), np.int64)
    d2f = np.empty((m, k), np.float64) if is_float else None
    st = lib.zdo_knn_brute(None if is_float else _p(ref), _p(ref) if is_float else None, _p(rid), n,
                           None if is_float else _p(q), _p(q) if is_float else None, _p(qid), m,
                           dim, k, _p(idx), _p(d2), _p(d2f), nthreads)
    if st:
        raise OracleError(st)
    return idx, (d2f if is_float else d2)


def knn_dist_grad(a, b, idx, gout=1.0):
    """fp64 loss sum ||a_i - b_idx|| and its gradients (ga, gb)."""
    lib = _load()
    a = np.ascontiguousarray(a, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    idx = np.ascontiguousarray(idx, np.int32)
    m, dim = a.shape
    nb = b.shape[0]
    k = idx.shape[1]
    g = np.ascontiguousarray(np.atleast_1d(np.asarray(gout, np.float64)))
    per = 1 if g.size == m * k and m * k > 1 else 0
    ga = np.empty((m, dim), np.float64)
    gb = np.empty((nb, dim), np.float64)
    loss = lib.zdo_knn_dist_grad(_p(a), _p(b), _p(idx), m, nb, dim, k, _p(g), per, _p(ga), _p(gb))
    return loss, ga, gb


class OracleSet:
    """A live point set with ids, updated in batches.  Reading of Sec. 2
    "Batch-dynamic updates" / Algorithm 4: after every insert or delete the tree
    is the canonical tree of the current set, so the oracle rebuilds it."""

    def __init__(self, pts, leaf_size: int, coord_bits: int, shift=None):
        self.pts = np.ascontiguousarray(pts, np.int32)
        self.ids = np.arange(len(self.pts), dtype=np.int32)
        self.next_id = len(self.pts)
        self.leaf_size, self.coord_bits, self.shift = leaf_size, coord_bits, shift

    def insert(self, batch) -> np.ndarray:
        batch = np.ascontiguousarray(batch, np.int32)
        morton_keys(batch, self.coord_bits, self.shift)  # range check, as a build would
        new = np.arange(self.next_id, self.next_id + len(batch), dtype=np.int32)
        self.next_id += len(batch)
        self.pts = np.concatenate([self.pts, batch])
        self.ids = np.concatenate([self.ids, new])
        return new

    def delete(self, ids) -> None:
        ids = np.asarray(ids, np.int32)
        if len(np.unique(ids)) != len(ids):
            raise OracleError(6)
        keep = ~np.isin(self.ids, ids)
        if int((~keep).sum()) != len(ids):
            raise OracleError(5)
        self.pts, self.ids = self.pts[keep], self.ids[keep]

    def tree(self) -> OracleTree:
        return OracleTree(self.pts, self.leaf_size, self.coord_bits, self.shift, ids=self.ids)
