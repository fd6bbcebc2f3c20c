"""ctypes declarations of include/agg.h (argument marshalling only).

The shared library is paper_1311_0059_gb300/libagg.so, built in-tree by
paper_1311_0059_gb300/build.py.  Loading fails loudly when it is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libagg.so")
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "agg.h")

AGG_OK = 0
AGG_ERR_INVALID_ARG = 1
AGG_ERR_BUDGET_TOO_SMALL = 2
AGG_ERR_OOM = 3
AGG_ERR_OUTPUT_CAPACITY = 4
AGG_ERR_STAGING_EXHAUSTED = 5
AGG_ERR_TIMEOUT = 6
AGG_ERR_CUDA = 7
AGG_ERR_INTERNAL = 8

AGG_COUNT, AGG_SUM, AGG_MIN, AGG_MAX = 1, 2, 4, 8
AGG_I32, AGG_I64 = 0, 1
AGG_PATH_HASH, AGG_PATH_SORT, AGG_PATH_AUTO = 0, 1, 2
AGG_MAX_LEVELS = 12
AGG_LEVEL0_SLOTS = 1 << 22  # default cap of the level-0 table (slots)
AGG_MIN_BUDGET = 1 << 20

_P = ctypes.c_void_p
_U64 = ctypes.c_uint64


class agg_spec(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_uint32), ("value_type", ctypes.c_int32), ("path", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("expected_groups", ctypes.c_uint64), ("seed", ctypes.c_uint64)]


class agg_tuning(ctypes.Structure):
    _fields_ = [("max_load_factor", ctypes.c_double), ("smem_entries", ctypes.c_uint32),
                ("fan_out", ctypes.c_uint32), ("warp_dedup", ctypes.c_uint32), ("wait_limit_us", ctypes.c_uint32),
                ("fudge", ctypes.c_double), ("in_budget", ctypes.c_uint32), ("sorted_input", ctypes.c_uint32),
                ("max_levels", ctypes.c_uint32), ("staging_tier", ctypes.c_uint32),
                ("level0_slots", ctypes.c_uint32)]


class agg_output(ctypes.Structure):
    _fields_ = [("keys", _P), ("count", _P), ("sum", _P), ("min", _P), ("max", _P), ("capacity", ctypes.c_uint64),
                ("d_n_groups", _P)]


class agg_stats(ctypes.Structure):
    _fields_ = [("n_rows", _U64), ("n_groups", _U64), ("levels", _U64), ("rounds", _U64),
                ("spill_records", _U64 * AGG_MAX_LEVELS), ("resident_groups", _U64 * AGG_MAX_LEVELS),
                ("spill_bytes_written", _U64), ("spill_bytes_read", _U64), ("rows_at_full", _U64),
                ("table_slots", _U64), ("table_capacity", _U64), ("table_bytes", _U64), ("budget_bytes", _U64),
                ("staging_bytes", _U64), ("fan_out", _U64), ("status_bits", _U64), ("kernel_launches", _U64),
                ("phase_ns", _U64 * 12), ("sorted_input", _U64), ("fallback_records", _U64),
                ("fallback_level", _U64), ("staging_in_host", _U64), ("path", _U64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["spill_records"] = list(self.spill_records)
        d["resident_groups"] = list(self.resident_groups)
        d["phase_ns"] = list(self.phase_ns)
        return d


class agg_plan_info(ctypes.Structure):
    _fields_ = [("entry_bytes", _U64), ("table_slots", _U64), ("table_capacity", _U64), ("fan_out", _U64),
                ("active_slots", _U64), ("working_bytes", _U64), ("staging_bytes", _U64),
                ("in_budget_path", _U64), ("partitions", _U64), ("hash_bytes", ctypes.c_double),
                ("sort_bytes", ctypes.c_double), ("hash_seconds", ctypes.c_double), ("sort_seconds", ctypes.c_double),
                ("chosen_path", _U64)]


class agg_batch_item(ctypes.Structure):
    _fields_ = [("d_keys", _P), ("d_vals", _P), ("n", _U64), ("budget", ctypes.c_size_t),
                ("expected_groups", _U64), ("out", agg_output)]


class agg_batch_tuning(ctypes.Structure):
    _fields_ = [("team_blocks", ctypes.c_uint32), ("smem_entries", ctypes.c_uint32),
                ("max_load_factor", ctypes.c_double), ("fan_out", ctypes.c_uint32), ("use_graph", ctypes.c_uint32)]


class agg_query(ctypes.Structure):
    _fields_ = [("d_keys", _P), ("d_vals", _P), ("n", _U64), ("budget", ctypes.c_size_t),
                ("expected_groups", _U64), ("out", agg_output), ("ready", _P)]


class agg_query_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("n_groups", _U64), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double), ("team_blocks", ctypes.c_uint32),
                ("path", ctypes.c_uint32)]


class agg_server_stats(ctypes.Structure):
    _fields_ = [("submitted", _U64), ("completed", _U64), ("running", _U64), ("queued", _U64),
                ("pool_bytes", _U64), ("pool_in_use", _U64), ("pool_peak", _U64), ("max_concurrent", _U64),
                ("staging_bytes", _U64), ("staging_in_use", _U64), ("staging_peak", _U64), ("blocks", _U64),
                ("blocks_in_use", _U64)]


AGG_QUERY_QUEUED, AGG_QUERY_RUNNING, AGG_QUERY_DONE, AGG_QUERY_FAILED = 0, 1, 2, 3


# name -> (restype, argtypes); the names are exactly those declared in include/agg.h
SIGNATURES = {
    "agg_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(agg_spec), ctypes.POINTER(_P)]),
    "agg_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(agg_tuning)]),
    "agg_reserve": (ctypes.c_int, [_P, _U64]),
    "agg_run": (ctypes.c_int, [_P, _P, _P, _U64, ctypes.POINTER(agg_output), _P]),
    "agg_run_host": (ctypes.c_int, [_P, _P, _P, _U64, ctypes.POINTER(agg_output), ctypes.POINTER(_U64), _P]),
    "agg_sync": (ctypes.c_int, [_P, ctypes.POINTER(_U64)]),
    "agg_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(agg_stats)]),
    "agg_destroy": (ctypes.c_int, [_P]),
    "agg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "agg_plan": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(agg_spec), ctypes.POINTER(agg_tuning), _U64,
                                ctypes.POINTER(agg_plan_info)]),
    "agg_run_noalloc": (ctypes.c_int, [ctypes.POINTER(agg_spec), _P, _P, _U64, ctypes.POINTER(agg_output),
                                       ctypes.POINTER(_U64), _P]),
    "agg_batch_create": (ctypes.c_int, [ctypes.POINTER(agg_spec), ctypes.POINTER(agg_batch_item), ctypes.c_uint32,
                                        ctypes.POINTER(agg_batch_tuning), ctypes.POINTER(_P)]),
    "agg_batch_run": (ctypes.c_int, [_P, _P]),
    "agg_batch_sync": (ctypes.c_int, [_P, ctypes.POINTER(_U64)]),
    "agg_batch_destroy": (ctypes.c_int, [_P]),
    "agg_server_create": (ctypes.c_int, [ctypes.POINTER(agg_spec), ctypes.c_size_t, ctypes.c_uint32,
                                         ctypes.POINTER(_P)]),
    "agg_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(agg_query), ctypes.POINTER(_U64)]),
    "agg_server_progress": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32)]),
    "agg_server_poll": (ctypes.c_int, [_P, _U64, ctypes.POINTER(agg_query_info)]),
    "agg_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(agg_server_stats)]),
    "agg_server_destroy": (ctypes.c_int, [_P]),
}

AGG_NOALLOC_SLOTS = 1 << 18
AGG_NOALLOC_MAX_ROWS = AGG_NOALLOC_SLOTS // 4

_LIB = None


class AggError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


def load(path: str = LIB_PATH):
    global _LIB
    if _LIB is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1311_0059_gb300/build.py "
                               "(the group-by has no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def strerror(status: int) -> str:
    return load().agg_strerror(int(status)).decode()


def check(status: int, where: str):
    if status != AGG_OK:
        raise AggError(status, where)
