"""Helpers for the GPU parity tests: run the library through its C ABI and
compare with the CPU oracle after a canonical sort by signed key."""
import numpy as np

import datagen as dg

FIELDS = ("keys", "count", "sum", "min", "max")
OPS_BITS = {"count": 1, "sum": 2, "min": 4, "max": 8}


def torch_mod():
    import torch
    return torch


def to_dev(a):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def canon(d):
    order = np.argsort(d["keys"], kind="stable")
    return {k: np.asarray(v)[order] for k, v in d.items()}


def gpu_groupby(keys, vals, budget, ops=15, vtype=None, path=0, tuning=None, expected_groups=0, seed=0,
                capacity=None):
    """Runs one group-by on the GPU; returns (canonical numpy result, stats)."""
    from paper_1311_0059_gb300 import AGG_I32, AGG_I64
    from paper_1311_0059_gb300.groupby import GroupBy
    torch = torch_mod()
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    if vtype is None:
        vtype = AGG_I32 if (vals is not None and np.asarray(vals).dtype == np.int32) else AGG_I64
    with GroupBy(budget, ops=ops, value_type=vtype, path=path, expected_groups=expected_groups, seed=seed,
                 tuning=tuning) as g:
        dk = to_dev(keys) if keys.size else torch.empty(0, dtype=torch.int64, device="cuda")
        dv = None
        if vals is not None:
            v = np.ascontiguousarray(vals)
            dv = to_dev(v) if v.size else torch.empty(0, dtype=torch.from_numpy(v).dtype, device="cuda")
        res = g.run(dk, dv, capacity=capacity)
        out = {k: t.cpu().numpy() for k, t in res.items()}
        st = g.stats()
    return canon(out), st


def assert_parity(got, exp, ops=15, what=""):
    gk, ek = np.asarray(got["keys"]), np.asarray(exp["keys"])
    assert gk.shape == ek.shape, f"{what}: {gk.size} groups, oracle has {ek.size}"
    assert np.array_equal(gk, ek), f"{what}: group keys differ"
    for f, bit in OPS_BITS.items():
        if ops & bit:
            g = np.asarray(got[f]).view(np.int64) if np.asarray(got[f]).dtype != np.int64 else np.asarray(got[f])
            e = np.asarray(exp[f]).astype(np.uint64).view(np.int64) if f == "count" else np.asarray(exp[f])
            bad = np.flatnonzero(g != e)
            assert bad.size == 0, f"{what}: {f} differs at {bad.size} groups, first key {gk[bad[0]]}"


def oracle_expected(oracle, keys, vals):
    v = None if vals is None else np.asarray(vals).astype(np.int64)
    res, _ = oracle.groupby(keys, v)
    return res


def check_invariants(res, n, vals_sum_u64=None, global_min=None, global_max=None):
    """Invariants of any group-by result (sorted by key): COUNTs add up to n,
    SUMs to the sum of all values (mod 2**64), the smallest MIN and largest MAX
    are the global minimum and maximum of the values, and keys are unique."""
    assert int(np.asarray(res["count"]).astype(np.uint64).sum(dtype=np.uint64)) == n
    if vals_sum_u64 is not None and "sum" in res:
        assert np.asarray(res["sum"]).view(np.uint64).sum(dtype=np.uint64) == vals_sum_u64
    if global_min is not None and "min" in res and n:
        assert int(np.asarray(res["min"]).min()) == global_min, "smallest MIN is not the global minimum"
    if global_max is not None and "max" in res and n:
        assert int(np.asarray(res["max"]).max()) == global_max, "largest MAX is not the global maximum"
    k = np.asarray(res["keys"])
    assert np.all(np.diff(k) > 0), "duplicate or unsorted group keys"


def device_workload(w: dg.Workload):
    """Generates w on the device with the CUDA generator; returns (keys, vals, cdf) tensors."""
    torch = torch_mod()
    keys = torch.empty(w.n, dtype=torch.int64, device="cuda")
    vals = torch.empty(w.n, dtype=torch.int32 if w.vtype == "i32_1000" else torch.int64, device="cuda")
    cdf = None
    if w.dist == "zipf":
        cdf = torch.from_numpy(w.cdf()).cuda()
    w.device(keys.data_ptr(), vals.data_ptr(), cdf_ptr=cdf.data_ptr() if cdf is not None else 0,
             stream_handle=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return keys, vals, cdf
