"""Thin ctypes binding of libzd (include/zd.h), with the C ABI's names.

Argument marshalling only: every step runs in the CUDA library.  Tensors are
PyTorch CUDA tensors (PyTorch provides device memory and the stream); the
library is loaded on first use and a missing library raises -- there is no
CPU fallback.  Paper references (Blelloch & Dobson, "Parallel Nearest
Neighbors in Low Dimensions with Batch Updates") are on each entry point.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# ZD_DEBUG=1 in the environment selects the debug build (index checks in the
# kernels; see build_lib.py)
LIB_PATH = os.path.join(_HERE, "_lib", "libzd_debug.so" if os.environ.get("ZD_DEBUG") == "1" else "libzd.so")

ZD_OK = 0
ZD_ERR_INVALID_ARG, ZD_ERR_RANGE, ZD_ERR_OOM, ZD_ERR_CUDA = 1, 2, 3, 4
ZD_ERR_NOT_FOUND, ZD_ERR_DUPLICATE_ID, ZD_ERR_TIMEOUT = 5, 6, 7
ZD_ERR_UNIMPLEMENTED, ZD_ERR_CAPACITY, ZD_ERR_INTERNAL = 8, 9, 10
ZD_COORD_I32, ZD_COORD_F32 = 0, 1
ZD_SEARCH_LEAF, ZD_SEARCH_BIT, ZD_SEARCH_ROOT = 0, 1, 2
ZD_KNN_THREAD_PER_QUERY, ZD_KNN_WARP_GROUP = 0x100, 0x200
ZD_KNN_ALL_POINTS = 0x400
ZD_MAX_K = 128

EXPORTED = ["zd_status_string", "zd_check", "zd_selftest_wait_timeout", "zd_morton_encode", "zd_morton_sort", "zd_morton_sort_noalloc",
            "zd_build",
            "zd_free", "zd_tree_info_get", "zd_export_tree", "zd_knn", "zd_insert_batch",
            "zd_delete_batch", "zd_knn_dist_backward", "zd_build_batched", "zd_knn_batched"]


class ZdParams(C.Structure):
    _fields_ = [("dim", C.c_int32), ("leaf_size", C.c_int32), ("coord_bits", C.c_int32),
                ("coord_type", C.c_int32), ("shift", C.c_uint32 * 3), ("capacity", C.c_int64)]


class ZdTreeInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("capacity", C.c_int64), ("next_id", C.c_int64),
                ("n_leaves", C.c_int64), ("n_internal", C.c_int64), ("dim", C.c_int32),
                ("leaf_size", C.c_int32), ("coord_bits", C.c_int32), ("coord_type", C.c_int32),
                ("n_clouds", C.c_int64)]


class ZdError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        msg = _lib().zd_status_string(code).decode() if _LIB is not None else str(code)
        super().__init__("%s: %s (status %d)" % (where, msg, code))


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libzd.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        lib = C.CDLL(LIB_PATH)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        lib.zd_status_string.argtypes = [i32]
        lib.zd_status_string.restype = C.c_char_p
        lib.zd_check.argtypes = [vp]
        lib.zd_selftest_wait_timeout.argtypes = [i32, vp]
        lib.zd_morton_encode.argtypes = [C.POINTER(ZdParams), vp, i64, vp, vp]
        lib.zd_morton_sort.argtypes = [vp, i64, i32, vp, vp, vp, vp]
        lib.zd_morton_sort_noalloc.argtypes = [vp, i64, i32, vp, vp, vp]
        lib.zd_build.argtypes = [C.POINTER(ZdParams), vp, vp, i64, vp, C.POINTER(vp)]
        lib.zd_free.argtypes = [vp, vp]
        lib.zd_tree_info_get.argtypes = [vp, C.POINTER(ZdTreeInfo), vp]
        lib.zd_export_tree.argtypes = [vp] + [vp] * 15
        lib.zd_knn.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp]
        lib.zd_insert_batch.argtypes = [vp, vp, i64, vp, vp]
        lib.zd_delete_batch.argtypes = [vp, vp, i64, vp]
        lib.zd_knn_dist_backward.argtypes = [vp, vp, vp, i64, i64, i64, i32, i32, vp, i32, vp, vp, vp]
        lib.zd_build_batched.argtypes = [C.POINTER(ZdParams), vp, vp, vp, vp, i64, vp, C.POINTER(vp)]
        lib.zd_knn_batched.argtypes = [vp, vp, vp, i64, i32, i32, vp, vp, vp]
        for name in EXPORTED:
            if name not in ("zd_status_string",):
                getattr(lib, name).restype = C.c_int
        _LIB = lib
    return _LIB


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _ok(code: int, where: str):
    if code != ZD_OK:
        raise ZdError(code, where)


def _cuda(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    return t.contiguous()


def _params(dim, leaf_size, coord_bits, coord_type, shift=None, capacity=0) -> ZdParams:
    p = ZdParams()
    p.dim, p.leaf_size, p.coord_bits, p.coord_type = dim, leaf_size, coord_bits, coord_type
    s = list(shift or [0, 0, 0]) + [0, 0, 0]
    for j in range(3):
        p.shift[j] = int(s[j])
    p.capacity = int(capacity)
    return p


def zd_check(stream=None) -> int:
    """Sync the stream; return and clear the device status word."""
    return _lib().zd_check(C.c_void_p(_stream(stream)))


def zd_selftest_wait_timeout(timeout_ms: int = 50, stream=None) -> None:
    """Enqueue a bounded wait on a flag nothing sets (failure-detection check);
    the next zd_check returns ZD_ERR_TIMEOUT."""
    _ok(_lib().zd_selftest_wait_timeout(int(timeout_ms), C.c_void_p(_stream(stream))), "zd_selftest_wait_timeout")


def zd_morton_encode(pts: torch.Tensor, coord_bits: int, shift=None, stream=None) -> torch.Tensor:
    """Morton keys of int32 points [n, dim] (Sec. 1.1); returned as int64
    tensors holding the uint64 bit patterns."""
    pts = _cuda(pts, torch.int32, "pts")
    n, dim = pts.shape
    keys = torch.empty(n, dtype=torch.int64, device=pts.device)
    p = _params(dim, 1, coord_bits, ZD_COORD_I32, shift)
    _ok(_lib().zd_morton_encode(C.byref(p), _ptr(pts), n, _ptr(keys), C.c_void_p(_stream(stream))),
        "zd_morton_encode")
    return keys


def zd_morton_sort(keys: torch.Tensor, key_bits: int = 64, stream=None):
    """Stable radix sort by key (Sec. 2 "Construction"): (sorted keys, perm)."""
    keys = _cuda(keys, torch.int64, "keys")
    n = keys.numel()
    out = torch.empty_like(keys)
    perm = torch.empty(n, dtype=torch.int32, device=keys.device)
    _ok(_lib().zd_morton_sort(_ptr(keys), n, key_bits, _ptr(out), _ptr(perm), None,
                              C.c_void_p(_stream(stream))), "zd_morton_sort")
    return out, perm


ZD_NOALLOC_MAX_KEYS = 1 << 20
ZD_MAX_KEYS = (1 << 30) - 1
ZD_POOL_KEEP_BYTES = 8 << 30
ZD_SMALL_BATCH = 16


def zd_morton_sort_noalloc(keys: torch.Tensor, key_bits: int = 64, stream=None, out=None):
    """zd_morton_sort for callers that may not allocate device memory: the
    library uses its own static scratch (at most ZD_NOALLOC_MAX_KEYS keys).
    Pass preallocated `out=(keys_out, perm_out)` to allocate nothing here
    either.  Calls that overlap on the GPU share the scratch and race."""
    keys = _cuda(keys, torch.int64, "keys")
    n = keys.numel()
    if out is None:
        out = (torch.empty_like(keys), torch.empty(n, dtype=torch.int32, device=keys.device))
    else:
        for t, dt, name in ((out[0], torch.int64, "out[0]"), (out[1], torch.int32, "out[1]")):
            if not (isinstance(t, torch.Tensor) and t.dtype == dt and t.device == keys.device
                    and t.is_contiguous() and t.numel() == n):
                raise ValueError("%s must be a contiguous %s tensor of %d elements on %s"
                                 % (name, dt, n, keys.device))
    _ok(_lib().zd_morton_sort_noalloc(_ptr(keys), n, key_bits, _ptr(out[0]), _ptr(out[1]),
                                      C.c_void_p(_stream(stream))), "zd_morton_sort_noalloc")
    return out


class ZdTree:
    """A zd-tree owned by libzd (Algorithm 1 + Sec. 2.1).  Use zd_build /
    zd_build_batched to make one."""

    def __init__(self, handle, dim, is_float, batched, device):
        self._h = handle
        self.dim, self.is_float, self.batched, self.device = dim, is_float, batched, device

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def free(self, stream=None):
        if self._h:
            _lib().zd_free(self._h, C.c_void_p(_stream(stream)))
            self._h = None

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("tree was freed")
        return self._h

    def info(self, stream=None) -> dict:
        i = ZdTreeInfo()
        _ok(_lib().zd_tree_info_get(self.handle, C.byref(i), C.c_void_p(_stream(stream))), "zd_tree_info_get")
        return {f: getattr(i, f) for f, _ in ZdTreeInfo._fields_}

    def export(self, stream=None) -> dict:
        """zd_export_tree into fresh tensors."""
        inf = self.info(stream)
        n, nl, ni, d = inf["n"], inf["n_leaves"], inf["n_internal"], self.dim
        dev = self.device
        bdt = torch.float32 if self.is_float else torch.int32
        e = dict(ids=torch.empty(n, dtype=torch.int32, device=dev),
                 keys=torch.empty(n, dtype=torch.int64, device=dev),
                 leaf_lo=torch.empty(nl + 1, dtype=torch.int32, device=dev),
                 node_lo=torch.empty(ni, dtype=torch.int32, device=dev),
                 node_hi=torch.empty(ni, dtype=torch.int32, device=dev),
                 node_bit=torch.empty(ni, dtype=torch.int32, device=dev),
                 node_left=torch.empty(ni, dtype=torch.int32, device=dev),
                 node_right=torch.empty(ni, dtype=torch.int32, device=dev),
                 node_parent=torch.empty(ni, dtype=torch.int32, device=dev),
                 leaf_parent=torch.empty(nl, dtype=torch.int32, device=dev),
                 node_box_lo=torch.empty((ni, d), dtype=bdt, device=dev),
                 node_box_hi=torch.empty((ni, d), dtype=bdt, device=dev),
                 leaf_box_lo=torch.empty((nl, d), dtype=bdt, device=dev),
                 leaf_box_hi=torch.empty((nl, d), dtype=bdt, device=dev))
        names = ["ids", "keys", "leaf_lo", "node_lo", "node_hi", "node_bit", "node_left", "node_right",
                 "node_parent", "leaf_parent", "node_box_lo", "node_box_hi", "leaf_box_lo", "leaf_box_hi"]
        _ok(_lib().zd_export_tree(self.handle, *[_ptr(e[k]) if e[k].numel() else None for k in names],
                                  C.c_void_p(_stream(stream))), "zd_export_tree")
        e["info"] = inf
        return e

    def knn(self, k: int, queries: torch.Tensor = None, mode: int = None, with_dist: bool = True,
            stream=None, out=None, mapping: int = 0):
        """Exact k-NN (Algorithms 2 and 3), ties by (squared distance, id).
        queries=None: all points (leaf-based, self excluded), rows by id.
        mapping: 0 (library choice), ZD_KNN_THREAD_PER_QUERY or ZD_KNN_WARP_GROUP."""
        if self.batched:
            raise RuntimeError("use zd_knn_batched for a forest")
        ddt = torch.float32 if self.is_float else torch.int64
        if queries is None:
            # all points; a bit- or root-based start is asked for explicitly
            mode = ZD_SEARCH_LEAF if mode in (None, ZD_SEARCH_LEAF) else mode | ZD_KNN_ALL_POINTS
            rows = self.info(stream)["next_id"] if out is None else None
            qp, m = None, 0
        else:
            mode = ZD_SEARCH_BIT if mode is None else mode
            queries = _cuda(queries, torch.float32 if self.is_float else torch.int32, "queries")
            m = queries.shape[0]
            rows, qp = m, _ptr(queries)
        if out is None:
            idx = torch.empty((rows, k), dtype=torch.int32, device=self.device)
            dist = torch.empty((rows, k), dtype=ddt, device=self.device) if with_dist else None
        else:
            idx, dist = out
        _ok(_lib().zd_knn(self.handle, qp, m, k, mode | mapping, _ptr(idx), _ptr(dist),
                          C.c_void_p(_stream(stream))), "zd_knn")
        return idx, dist

    def insert(self, pts: torch.Tensor, stream=None) -> torch.Tensor:
        """Batch insert (Algorithm 4); returns the new ids.  Batches of at most
        ZD_SMALL_BATCH points are applied on the device without a sync (a
        range error goes to zd_check); larger ones sync and raise."""
        pts = _cuda(pts, torch.int32, "pts")
        ids = torch.empty(pts.shape[0], dtype=torch.int32, device=pts.device)
        _ok(_lib().zd_insert_batch(self.handle, _ptr(pts), pts.shape[0], _ptr(ids),
                                   C.c_void_p(_stream(stream))), "zd_insert_batch")
        return ids

    def delete(self, ids: torch.Tensor, stream=None) -> None:
        """Batch delete by id.  Batches of at most ZD_SMALL_BATCH ids are
        applied on the device without a sync (unknown or repeated ids go to
        zd_check); larger ones sync and raise."""
        ids = _cuda(ids, torch.int32, "ids")
        _ok(_lib().zd_delete_batch(self.handle, _ptr(ids), ids.numel(), C.c_void_p(_stream(stream))),
            "zd_delete_batch")


def zd_build(pts: torch.Tensor, leaf_size: int, coord_bits: int, shift=None, capacity: int = 0,
             stream=None) -> ZdTree:
    """Canonical pruned zd-tree of int32 or float32 points [n, dim]."""
    if pts.dtype == torch.float32:
        ct = ZD_COORD_F32
    else:
        ct = ZD_COORD_I32
        pts = _cuda(pts, torch.int32, "pts")
    pts = pts.contiguous()
    n, dim = pts.shape
    p = _params(dim, leaf_size, coord_bits, ct, shift, capacity)
    h = C.c_void_p()
    _ok(_lib().zd_build(C.byref(p), None, _ptr(pts) if n else None, n, C.c_void_p(_stream(stream)),
                        C.byref(h)), "zd_build")
    return ZdTree(h, dim, ct == ZD_COORD_F32, False, pts.device)


def zd_build_batched(pts: torch.Tensor, offsets, leaf_size: int, coord_bits: int, stream=None,
                     offsets_device: torch.Tensor = None) -> ZdTree:
    """One forest of independent trees; offsets [n_clouds + 1] (host list /
    CPU tensor).  offsets_device: the same offsets already on the GPU (pass it
    when capturing a CUDA graph, so that no host copy is recorded)."""
    pts = pts.contiguous()
    ct = ZD_COORD_F32 if pts.dtype == torch.float32 else ZD_COORD_I32
    n, dim = pts.shape
    off_h = torch.as_tensor(offsets, dtype=torch.int64).cpu().contiguous()
    off_d = offsets_device if offsets_device is not None else off_h.to(pts.device)
    p = _params(dim, leaf_size, coord_bits, ct)
    h = C.c_void_p()
    t = ZdTree(None, dim, ct == ZD_COORD_F32, True, pts.device)
    _ok(_lib().zd_build_batched(C.byref(p), None, _ptr(pts) if n else None, C.c_void_p(off_h.data_ptr()),
                                _ptr(off_d), off_h.numel() - 1, C.c_void_p(_stream(stream)), C.byref(h)),
        "zd_build_batched")
    t._h = h
    t.offsets = off_h
    return t


def zd_knn_batched(tree: ZdTree, k: int, queries: torch.Tensor = None, query_offsets=None,
                   with_dist: bool = True, stream=None, out=None, mapping: int = 0):
    """k-NN inside every cloud of a forest; ids are cloud-local."""
    ddt = torch.float32 if tree.is_float else torch.int64
    if queries is None:
        rows, m, qp, qo = int(tree.offsets[-1]), 0, None, None
    else:
        queries = _cuda(queries, torch.float32 if tree.is_float else torch.int32, "queries")
        m = rows = queries.shape[0]
        qo = torch.as_tensor(query_offsets, dtype=torch.int64).to(queries.device).contiguous()
        qp = _ptr(queries)
    if out is None:
        idx = torch.empty((rows, k), dtype=torch.int32, device=tree.device)
        dist = torch.empty((rows, k), dtype=ddt, device=tree.device) if with_dist else None
    else:
        idx, dist = out
    _ok(_lib().zd_knn_batched(tree.handle, qp, _ptr(qo) if qo is not None else None, m, k, mapping,
                              _ptr(idx), _ptr(dist), C.c_void_p(_stream(stream))), "zd_knn_batched")
    return idx, dist


def zd_knn_dist_backward(q: torch.Tensor, ref: torch.Tensor, idx: torch.Tensor, gout: torch.Tensor,
                         stream=None):
    """Gradients of sum gout * ||q_i - ref_idx(i,j)|| over a batch
    [batch, m, dim] / [batch, r, dim] / idx [batch, m, k]."""
    q = _cuda(q, torch.float32, "q")
    ref = _cuda(ref, torch.float32, "ref")
    idx = _cuda(idx, torch.int32, "idx")
    if q.dim() == 2:
        q, ref, idx = q[None], ref[None], idx[None]
        squeeze = True
    else:
        squeeze = False
    batch, m, dim = q.shape
    r, k = ref.shape[1], idx.shape[2]
    g = _cuda(gout.to(torch.float32).reshape(-1), torch.float32, "gout")
    per = 1 if g.numel() == batch * m * k and g.numel() > 1 else 0
    gq = torch.empty_like(q)
    gr = torch.empty_like(ref)
    _ok(_lib().zd_knn_dist_backward(_ptr(q), _ptr(ref), _ptr(idx), batch, m, r, dim, k, _ptr(g), per,
                                    _ptr(gq), _ptr(gr), C.c_void_p(_stream(stream))), "zd_knn_dist_backward")
    if squeeze:
        return gq[0], gr[0]
    return gq, gr


class KnnDist(torch.autograd.Function):
    """loss-ready k-NN distances of a batch of float clouds.

    forward(A [P, m, 3], B [P, r, 3], k, leaf_size): builds one forest over the
    P clouds of B, finds the k nearest points of B for every point of A (fp64
    ranking), returns the fp32 distances [P, m, k] and saves only the ids.
    backward recomputes the distances in fp32 (zd_knn_dist_backward)."""

    @staticmethod
    def forward(ctx, A, B, k: int, leaf_size: int = 16, coord_bits: int = 21):
        P, m, dim = A.shape
        r = B.shape[1]
        offB = [i * r for i in range(P + 1)]
        offA = [i * m for i in range(P + 1)]
        tree = zd_build_batched(B.reshape(P * r, dim), offB, leaf_size, coord_bits)
        idx, dist = zd_knn_batched(tree, k, queries=A.reshape(P * m, dim), query_offsets=offA)
        tree.free()
        idx = idx.view(P, m, k)
        ctx.save_for_backward(A, B, idx)
        ctx.mark_non_differentiable(idx)
        return dist.view(P, m, k), idx

    @staticmethod
    def backward(ctx, gdist, gidx):
        A, B, idx = ctx.saved_tensors
        ga, gb = zd_knn_dist_backward(A, B, idx, gdist.contiguous())
        return ga, gb, None, None, None
