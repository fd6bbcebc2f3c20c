"""Thin torch-facing wrapper over the C ABI: allocates output tensors and passes
raw device pointers and the current CUDA stream to libagg.so.  Every step of
the group-by runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes

import torch

from . import _abi
from ._abi import (AGG_COUNT, AGG_I32, AGG_I64, AGG_MAX, AGG_MIN, AGG_PATH_HASH, AGG_PATH_SORT, AGG_SUM,
                   agg_batch_item, agg_batch_tuning, agg_output, agg_plan_info, agg_query, agg_query_info,
                   agg_server_stats, agg_spec, agg_stats, agg_tuning, check)

ALL_OPS = AGG_COUNT | AGG_SUM | AGG_MIN | AGG_MAX


def make_spec(ops=ALL_OPS, value_type=AGG_I64, path=AGG_PATH_HASH, expected_groups=0, seed=0):
    return agg_spec(ops=ops, value_type=value_type, path=path, flags=0, expected_groups=expected_groups, seed=seed)


def plan(budget: int, n: int, spec: agg_spec, tuning: agg_tuning | None = None) -> dict:
    info = agg_plan_info()
    check(_abi.load().agg_plan(budget, ctypes.byref(spec), ctypes.byref(tuning) if tuning else None, n,
                               ctypes.byref(info)), "agg_plan")
    return {f: getattr(info, f) for f, _ in info._fields_}


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Output:
    """Device output tensors for up to `capacity` groups."""

    def __init__(self, capacity: int, ops: int, device):
        cap = max(int(capacity), 1)
        self.capacity = cap
        self.keys = torch.empty(cap, dtype=torch.int64, device=device)
        self.count = torch.empty(cap, dtype=torch.int64, device=device) if ops & AGG_COUNT else None
        self.sum = torch.empty(cap, dtype=torch.int64, device=device) if ops & AGG_SUM else None
        self.min = torch.empty(cap, dtype=torch.int64, device=device) if ops & AGG_MIN else None
        self.max = torch.empty(cap, dtype=torch.int64, device=device) if ops & AGG_MAX else None
        self.n_groups = torch.zeros(1, dtype=torch.int64, device=device)
        self.abi = agg_output(keys=self.keys.data_ptr(),
                              count=self.count.data_ptr() if self.count is not None else None,
                              sum=self.sum.data_ptr() if self.sum is not None else None,
                              min=self.min.data_ptr() if self.min is not None else None,
                              max=self.max.data_ptr() if self.max is not None else None,
                              capacity=cap, d_n_groups=self.n_groups.data_ptr())

    def result(self, n_groups: int) -> dict:
        g = int(n_groups)
        out = {"keys": self.keys[:g]}
        for f in ("count", "sum", "min", "max"):
            t = getattr(self, f)
            if t is not None:
                out[f] = t[:g]
        return out


class GroupBy:
    """One budgeted group-by handle (agg_create .. agg_destroy)."""

    def __init__(self, budget_bytes: int, ops: int = ALL_OPS, value_type: int = AGG_I64, path: int = AGG_PATH_HASH,
                 expected_groups: int = 0, seed: int = 0, tuning: agg_tuning | None = None):
        self.lib = _abi.load()
        self.spec = make_spec(ops, value_type, path, expected_groups, seed)
        self.ops = ops
        self.budget = budget_bytes
        h = ctypes.c_void_p()
        check(self.lib.agg_create(budget_bytes, ctypes.byref(self.spec), ctypes.byref(h)), "agg_create")
        self.h = h
        if tuning is not None:
            self.set_tuning(tuning)

    def set_tuning(self, tuning: agg_tuning):
        check(self.lib.agg_set_tuning(self.h, ctypes.byref(tuning)), "agg_set_tuning")

    def reserve(self, max_rows: int):
        check(self.lib.agg_reserve(self.h, max_rows), "agg_reserve")

    def output(self, capacity: int, device) -> Output:
        return Output(capacity, self.ops, device)

    def run_async(self, keys: torch.Tensor, vals: torch.Tensor | None, out: Output, n: int | None = None,
                  stream=None) -> int:
        """Enqueues agg_run on `stream` (default: current stream); returns the status."""
        n = keys.numel() if n is None else n
        return self.lib.agg_run(self.h, ctypes.c_void_p(keys.data_ptr()),
                                ctypes.c_void_p(vals.data_ptr()) if vals is not None else None, n,
                                ctypes.byref(out.abi), _stream_ptr(stream))

    def sync(self) -> int:
        ng = ctypes.c_uint64()
        check(self.lib.agg_sync(self.h, ctypes.byref(ng)), "agg_sync")
        return ng.value

    def run(self, keys: torch.Tensor, vals: torch.Tensor | None, capacity: int | None = None, stream=None) -> dict:
        """agg_run + agg_sync; returns device tensors of the n_groups result rows."""
        n = keys.numel()
        out = self.output(n if capacity is None else capacity, keys.device)
        check(self.run_async(keys, vals, out, n, stream), "agg_run")
        ng = self.sync()
        return out.result(ng)

    def run_host(self, keys, vals, out_capacity: int | None = None, stream=None) -> dict:
        """agg_run_host on host arrays (numpy or CPU tensors); returns numpy arrays."""
        import numpy as np
        k = np.ascontiguousarray(keys, dtype=np.int64)
        v = None if vals is None else np.ascontiguousarray(vals)
        n = k.shape[0]
        cap = max(n if out_capacity is None else out_capacity, 1)
        res = {f: np.empty(cap, np.int64) for f in ("keys", "count", "sum", "min", "max")}
        ho = agg_output(keys=res["keys"].ctypes.data, count=res["count"].ctypes.data, sum=res["sum"].ctypes.data,
                        min=res["min"].ctypes.data, max=res["max"].ctypes.data, capacity=cap, d_n_groups=None)
        ng = ctypes.c_uint64()
        check(self.lib.agg_run_host(self.h, ctypes.c_void_p(k.ctypes.data),
                                    ctypes.c_void_p(v.ctypes.data) if v is not None else None, n, ctypes.byref(ho),
                                    ctypes.byref(ng), _stream_ptr(stream)), "agg_run_host")
        g = ng.value
        out = {"keys": res["keys"][:g]}
        for f, bit in (("count", AGG_COUNT), ("sum", AGG_SUM), ("min", AGG_MIN), ("max", AGG_MAX)):
            if self.ops & bit:
                out[f] = res[f][:g]
        return out

    def stats(self) -> dict:
        s = agg_stats()
        check(self.lib.agg_get_stats(self.h, ctypes.byref(s)), "agg_get_stats")
        return s.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.lib.agg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many independent group-bys run by one persistent launch (agg_batch_*).

    `instances` is a list of (keys, vals, budget_bytes, expected_groups) with
    device tensors; outputs are allocated here, one Output per instance."""

    def __init__(self, instances, ops: int = ALL_OPS, value_type: int = AGG_I64, seed: int = 0,
                 tuning: agg_batch_tuning | None = None, capacities=None):
        self.lib = _abi.load()
        self.spec = make_spec(ops, value_type, AGG_PATH_HASH, 0, seed)
        self.ops = ops
        self.outs = []
        items = (agg_batch_item * max(len(instances), 1))()
        for i, (k, v, budget, eg) in enumerate(instances):
            cap = k.numel() if capacities is None else capacities[i]
            o = Output(cap, ops, k.device)
            self.outs.append(o)
            items[i] = agg_batch_item(d_keys=k.data_ptr(), d_vals=v.data_ptr() if v is not None else None,
                                      n=k.numel(), budget=budget, expected_groups=eg, out=o.abi)
        self.inputs = instances
        h = ctypes.c_void_p()
        check(self.lib.agg_batch_create(ctypes.byref(self.spec), items, len(instances),
                                        ctypes.byref(tuning) if tuning is not None else None, ctypes.byref(h)),
              "agg_batch_create")
        self.h = h
        self.count = len(instances)

    def run_async(self, stream=None) -> int:
        return self.lib.agg_batch_run(self.h, _stream_ptr(stream))

    def sync(self):
        ng = (ctypes.c_uint64 * max(self.count, 1))()
        check(self.lib.agg_batch_sync(self.h, ng), "agg_batch_sync")
        return [ng[i] for i in range(self.count)]

    def run(self, stream=None):
        check(self.run_async(stream), "agg_batch_run")
        ng = self.sync()
        return [o.result(g) for o, g in zip(self.outs, ng)]

    def close(self):
        if getattr(self, "h", None):
            self.lib.agg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Queries that arrive over time, admitted against a device memory pool by
    their declared budgets and run concurrently (agg_server_*)."""

    def __init__(self, pool_bytes: int, max_active: int = 64, ops: int = ALL_OPS, value_type: int = AGG_I64,
                 seed: int = 0, path: int = AGG_PATH_HASH):
        self.lib = _abi.load()
        self.spec = make_spec(ops, value_type, path, 0, seed)
        self.ops = ops
        h = ctypes.c_void_p()
        check(self.lib.agg_server_create(ctypes.byref(self.spec), pool_bytes, max_active, ctypes.byref(h)),
              "agg_server_create")
        self.h = h
        self.keep = {}  # tensors that must live until their query completes

    def submit(self, keys, vals, budget: int, out: Output, expected_groups: int = 0, ready_event=None) -> int:
        q = agg_query(d_keys=keys.data_ptr(), d_vals=vals.data_ptr() if vals is not None else None, n=keys.numel(),
                      budget=budget, expected_groups=expected_groups, out=out.abi,
                      ready=ready_event.cuda_event if ready_event is not None else None)
        t = ctypes.c_uint64()
        check(self.lib.agg_server_submit(self.h, ctypes.byref(q), ctypes.byref(t)), "agg_server_submit")
        self.keep[t.value] = (keys, vals, out, ready_event)
        return t.value

    def progress(self) -> int:
        c = ctypes.c_uint32()
        check(self.lib.agg_server_progress(self.h, ctypes.byref(c)), "agg_server_progress")
        return c.value

    def poll(self, ticket: int) -> agg_query_info:
        info = agg_query_info()
        check(self.lib.agg_server_poll(self.h, ticket, ctypes.byref(info)), "agg_server_poll")
        return info

    def release(self, ticket: int):
        self.keep.pop(ticket, None)

    def stats(self) -> dict:
        st = agg_server_stats()
        check(self.lib.agg_server_get_stats(self.h, ctypes.byref(st)), "agg_server_get_stats")
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.agg_server_destroy(self.h)
            self.h = None
            self.keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
