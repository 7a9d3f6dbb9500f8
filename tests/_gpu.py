"""Helpers for the GPU parity tests: turn a zd_export_tree dump into the
(lo, hi, bit) node list and unified link arrays used by tests/_checks.py."""
import numpy as np


def nodes_of(e):
    """All nodes as sorted (lo, hi, bit) plus boxes keyed by (lo, hi)."""
    nl = int(e["info"]["n_leaves"])
    ni = nl - 1
    leaf_lo = e["leaf_lo"].cpu().numpy().astype(np.int64)
    lo = np.concatenate([e["node_lo"].cpu().numpy(), leaf_lo[:-1]]).astype(np.int64)
    hi = np.concatenate([e["node_hi"].cpu().numpy(), leaf_lo[1:]]).astype(np.int64)
    bit = np.concatenate([e["node_bit"].cpu().numpy(), -np.ones(nl, np.int32)]).astype(np.int64)
    box_lo = np.concatenate([e["node_box_lo"].cpu().numpy(), e["leaf_box_lo"].cpu().numpy()])
    box_hi = np.concatenate([e["node_box_hi"].cpu().numpy(), e["leaf_box_hi"].cpu().numpy()])
    # unified ids: internal i -> i, leaf j -> ni + j
    def uni(c):
        c = np.asarray(c, np.int64)
        return np.where(c >= 0, c, ni + (~c))
    left = np.concatenate([uni(e["node_left"].cpu().numpy()), -np.ones(nl, np.int64)])
    right = np.concatenate([uni(e["node_right"].cpu().numpy()), -np.ones(nl, np.int64)])
    parent = np.concatenate([e["node_parent"].cpu().numpy(), e["leaf_parent"].cpu().numpy()]).astype(np.int64)
    root = 0 if ni > 0 else ni
    return dict(lo=lo, hi=hi, bit=bit, box_lo=box_lo, box_hi=box_hi, left=left, right=right,
                parent=parent, root=root, keys=e["keys"].cpu().numpy().view(np.uint64),
                ids=e["ids"].cpu().numpy())


def canonical(d):
    order = np.lexsort((d["hi"], d["lo"]))
    return dict(lo=d["lo"][order], hi=d["hi"][order], bit=d["bit"][order],
                box_lo=d["box_lo"][order], box_hi=d["box_hi"][order])
