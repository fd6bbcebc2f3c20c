"""Oracle work for the full-size parity tests, spread over the host's cores.

The functions here run in worker processes started with the "spawn" method (a
process forked after the first GPU call would hang), and call only the CPU
oracle and the seeded input generator.  A full-size input is split into
key-disjoint parts by a multiplicative hash of the key: a group-by result is
the union of the results of any partition of the key set, so each worker runs
the plain oracle on the rows of its part and the union is compared with the
GPU result part by part."""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

PART_MUL = np.uint64(0x9E3779B97F4A7C15)


def part_of(keys: np.ndarray, nparts_log2: int) -> np.ndarray:
    """Part of each key: the top bits of key * odd constant (mod 2**64)."""
    with np.errstate(over="ignore"):
        return ((np.asarray(keys, np.int64).view(np.uint64) * PART_MUL) >> np.uint64(64 - nparts_log2)).astype(
            np.int64)


def pool(workers: int | None = None):
    return mp.get_context("spawn").Pool(workers or max(1, min(16, os.cpu_count() or 1)))


class Shared:
    """A numpy array in shared memory that spawned workers attach to by name."""

    def __init__(self, n: int, dtype):
        self.dtype = np.dtype(dtype)
        self.n = n
        self.shm = shared_memory.SharedMemory(create=True, size=max(1, n * self.dtype.itemsize))
        self.array = np.ndarray((n,), dtype=self.dtype, buffer=self.shm.buf)

    def ref(self):
        return (self.shm.name, self.n, self.dtype.str)

    def close(self):
        self.array = None
        self.shm.close()
        self.shm.unlink()


def _attach(ref):
    name, n, dt = ref
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray((n,), dtype=np.dtype(dt), buffer=shm.buf)


def oracle_part(task):
    """Oracle result of the rows whose key falls in part `part` (of 2**plog)."""
    import oracle
    kref, vref, part, plog, budget = task
    ks, keys = _attach(kref)
    vs, vals = _attach(vref)
    try:
        step = 1 << 24
        sel_k, sel_v = [], []
        for a in range(0, keys.size, step):
            k = keys[a:a + step]
            m = part_of(k, plog) == part
            sel_k.append(k[m].copy())
            sel_v.append(vals[a:a + step][m].astype(np.int64))
        k = np.concatenate(sel_k) if sel_k else np.zeros(0, np.int64)
        v = np.concatenate(sel_v) if sel_v else np.zeros(0, np.int64)
        res, _ = oracle.default().groupby(k, v, budget_bytes=budget)
        return part, res
    finally:
        del keys, vals
        ks.close()
        vs.close()


def oracle_workload(task):
    """Oracle result of one seeded workload, generated on this host."""
    import datagen as dg
    import oracle
    idx, params = task
    w = dg.Workload(**params)
    keys, vals = w.host()
    res, _ = oracle.default().groupby(keys, vals.astype(np.int64), budget_bytes=w.budget)
    return idx, res


def workload_params(w) -> dict:
    return dict(name=w.name, n=w.n, domain=w.domain, dist=w.dist, zipf_s=w.zipf_s, vtype=w.vtype, seed=w.seed,
                budget=w.budget, ops=w.ops)
