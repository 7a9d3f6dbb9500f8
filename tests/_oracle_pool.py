"""Oracle checks of the large workloads, run in a process pool.

The pool uses the spawn start method, so it may be started after the test
process has initialised CUDA (a forked child of a CUDA process can hang).
Workers read the point coordinates from one shared-memory block instead of
receiving copies through pipes.
"""
import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np


def workers(cap: int = 8) -> int:
    return max(1, min(cap, len(os.sched_getaffinity(0))))


class SharedPoints:
    """An int32 [rows, dim] array in a shared-memory block (owner side)."""

    def __init__(self, arr: np.ndarray):
        arr = np.ascontiguousarray(arr, np.int32)
        self.shape = arr.shape
        self.shm = shared_memory.SharedMemory(create=True, size=max(arr.nbytes, 1))
        np.ndarray(arr.shape, np.int32, buffer=self.shm.buf)[...] = arr

    @property
    def name(self):
        return self.shm.name

    def close(self):
        self.shm.close()
        self.shm.unlink()


def _dynamic_round(args):
    """The exact k-NN of one round's queries over that round's live set: ids
    below n_rows that are not in `deleted`, coordinates from the shared
    array.  The oracle tree of the live set, bit-based search (Sec. 2)."""
    shm_name, shape, n_rows, deleted, queries, leaf_size, coord_bits, k = args
    from oracle import oracle

    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        all_pts = np.ndarray(shape, np.int32, buffer=shm.buf)
        live = np.ones(n_rows, bool)
        live[deleted] = False
        ids = np.nonzero(live)[0].astype(np.int32)
        t = oracle.OracleTree(all_pts[ids], leaf_size, coord_bits, ids=ids)
        idx, d2 = t.knn(k, queries=queries, mode=oracle.MODE_BIT, nthreads=1)
        return idx, d2
    finally:
        shm.close()


def dynamic_rounds(all_pts: np.ndarray, rounds, leaf_size: int, coord_bits: int, k: int):
    """rounds: list of (n_rows, deleted ids so far, queries).  Returns the
    oracle's (idx, d2) per round, in order."""
    sp = SharedPoints(all_pts)
    try:
        jobs = [(sp.name, sp.shape, n_rows, dele, q, leaf_size, coord_bits, k) for n_rows, dele, q in rounds]
        with mp.get_context("spawn").Pool(workers()) as pool:
            return pool.map(_dynamic_round, jobs, chunksize=1)
    finally:
        sp.close()
