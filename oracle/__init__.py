"""CPU oracle for the budgeted group-by (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of bench.py may import this package; the library's product path never
does.  The C++ source (oracle.cpp) shares no code with the GPU path.

Functions return numpy arrays sorted ascending by signed int64 key:
``groupby`` (budgeted Hash-Sort discipline, Section 4.2), ``groupby_bruteforce``
(nested-loop definition, Section 3.1), ``groups_of`` (full-scan recomputation of
chosen groups) and ``count_distinct``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
LIB_PATH = os.path.join(HERE, "liboracle.so")
ENTRY_BYTES = 64  # memory charged per group held in the oracle's hash map

_P = ctypes.c_void_p
_U64 = ctypes.c_uint64


def build(out: str = LIB_PATH, mutant: int = 0) -> str:
    """Compile oracle.cpp (optionally with a planted mistake, for pin tests)."""
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", f"-DORACLE_MUTANT={int(mutant)}", "-o", out, SRC]
    subprocess.run(cmd, check=True)
    return out


def _ptr(a):
    return a.ctypes.data_as(_P) if a is not None else None


class Oracle:
    def __init__(self, path: str = LIB_PATH):
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(SRC):
            build(path)
        lib = ctypes.CDLL(path)
        lib.oracle_groupby.restype = ctypes.c_int
        lib.oracle_groupby.argtypes = [_P, _P, _U64, _U64, _U64, _P, _P, _P, _P, _P, _U64, _P, _P]
        lib.oracle_groupby_bruteforce.restype = ctypes.c_int
        lib.oracle_groupby_bruteforce.argtypes = [_P, _P, _U64, _P, _P, _P, _P, _P, _U64, _P]
        lib.oracle_groups_of.restype = ctypes.c_int
        lib.oracle_groups_of.argtypes = [_P, _P, _U64, _P, _U64, _P, _P, _P, _P]
        lib.oracle_count_distinct.restype = ctypes.c_uint64
        lib.oracle_count_distinct.argtypes = [_P, _U64]
        self.lib = lib
        self.path = path

    @staticmethod
    def _inputs(keys, vals):
        keys = np.ascontiguousarray(keys, dtype=np.int64)
        vals = None if vals is None else np.ascontiguousarray(vals).astype(np.int64)
        return keys, vals

    @staticmethod
    def _outs(cap):
        cap = max(int(cap), 1)
        return dict(keys=np.empty(cap, np.int64), count=np.empty(cap, np.uint64), sum=np.empty(cap, np.int64),
                    min=np.empty(cap, np.int64), max=np.empty(cap, np.int64))

    def groupby(self, keys, vals, budget_bytes: int = 1 << 40, entry_bytes: int = ENTRY_BYTES):
        """Budgeted group-by; returns (dict of arrays, number of sorted runs)."""
        keys, vals = self._inputs(keys, vals)
        n = keys.shape[0]
        o = self._outs(n)
        ng = np.zeros(1, np.uint64)
        nr = np.zeros(1, np.uint64)
        rc = self.lib.oracle_groupby(_ptr(keys), _ptr(vals), n, int(budget_bytes), int(entry_bytes),
                                     _ptr(o["keys"]), _ptr(o["count"]), _ptr(o["sum"]), _ptr(o["min"]),
                                     _ptr(o["max"]), max(n, 1), _ptr(ng), _ptr(nr))
        if rc != 0:
            raise RuntimeError(f"oracle_groupby returned {rc}")
        g = int(ng[0])
        return {k: v[:g] for k, v in o.items()}, int(nr[0])

    def groupby_bruteforce(self, keys, vals):
        keys, vals = self._inputs(keys, vals)
        n = keys.shape[0]
        o = self._outs(n)
        ng = np.zeros(1, np.uint64)
        rc = self.lib.oracle_groupby_bruteforce(_ptr(keys), _ptr(vals), n, _ptr(o["keys"]), _ptr(o["count"]),
                                                _ptr(o["sum"]), _ptr(o["min"]), _ptr(o["max"]), max(n, 1), _ptr(ng))
        if rc != 0:
            raise RuntimeError(f"oracle_groupby_bruteforce returned {rc}")
        g = int(ng[0])
        return {k: v[:g] for k, v in o.items()}

    def groups_of(self, keys, vals, sample):
        keys, vals = self._inputs(keys, vals)
        sample = np.ascontiguousarray(sample, dtype=np.int64)
        m = sample.shape[0]
        o = self._outs(m)
        rc = self.lib.oracle_groups_of(_ptr(keys), _ptr(vals), keys.shape[0], _ptr(sample), m, _ptr(o["count"]),
                                       _ptr(o["sum"]), _ptr(o["min"]), _ptr(o["max"]))
        if rc != 0:
            raise RuntimeError(f"oracle_groups_of returned {rc}")
        o["keys"] = sample.copy()
        return {k: v[:m] for k, v in o.items()}

    def count_distinct(self, keys) -> int:
        keys = np.ascontiguousarray(keys, dtype=np.int64)
        return int(self.lib.oracle_count_distinct(_ptr(keys), keys.shape[0]))


_DEFAULT = None


def default() -> Oracle:
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Oracle()
    return _DEFAULT


def mutant(k: int) -> Oracle:
    """An oracle built with planted mistake ``k`` (1..8), in a temporary file."""
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    path = os.path.join(d, f"liboracle_m{k}.so")
    build(path, mutant=k)
    return Oracle(path)
