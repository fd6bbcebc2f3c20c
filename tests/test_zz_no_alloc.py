"""agg_run_noalloc, the entry point for callers that cannot allocate device
memory, against the CPU oracle and against the allocating agg_run.

Some callers may not call cudaMalloc or cudaFree (a plug-in inside a framework
that owns every device allocation, a latency-critical path that cannot afford
an allocation or the synchronisation of a free).  agg_run_noalloc serves them
from a fixed array inside the library; its results must equal the oracle's and
agg_run's, and a second call in a row must not see the first call's leftovers.
This file is collected last, so a run that stops at the first failure has run
every other test before it; it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from _gpu import assert_parity, canon, oracle_expected

pytestmark = pytest.mark.gpu


def _call_noalloc(keys, vals, ops, vt, seed=0, capacity=None):
    import torch
    from paper_1311_0059_gb300 import _abi
    from paper_1311_0059_gb300.groupby import Output, make_spec
    lib = _abi.load()
    n = keys.numel()
    spec = make_spec(ops=ops, value_type=vt, seed=seed)
    out = Output(n if capacity is None else capacity, ops, keys.device)
    ng = ctypes.c_uint64()
    st = lib.agg_run_noalloc(ctypes.byref(spec), ctypes.c_void_p(keys.data_ptr()),
                             ctypes.c_void_p(vals.data_ptr()) if vals is not None else None, n,
                             ctypes.byref(out.abi), ctypes.byref(ng),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        return st, ng.value, None
    assert int(out.n_groups.item()) == ng.value
    return st, ng.value, canon({k: t.cpu().numpy() for k, t in out.result(ng.value).items()})


@pytest.mark.parametrize("ops,vdtype", [(15, np.int64), (15, np.int32), (3, np.int64)])
def test_noalloc_matches_oracle_and_agg_run_twice(oracle, ops, vdtype):
    import torch
    from paper_1311_0059_gb300 import AGG_I32, AGG_I64, _abi
    from paper_1311_0059_gb300.groupby import GroupBy
    vt = AGG_I32 if vdtype == np.int32 else AGG_I64
    rng = np.random.default_rng(ops)
    n = _abi.AGG_NOALLOC_MAX_ROWS
    for call in range(2):
        # a different key set on each call: leftovers of the first call would show
        keys = rng.integers(-2**63, 2**63 - 1, 9000 + 4000 * call, dtype=np.int64)[rng.integers(0, 9000, n)]
        keys[:3] = np.iinfo(np.int64).min  # the empty-marker key value takes the side slot
        vals = rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(vdtype)
        dk, dv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda()
        st, _, got = _call_noalloc(dk, dv, ops, vt)
        assert st == 0, f"call {call}: status {st}"
        assert_parity(got, oracle_expected(oracle, keys, vals), ops, f"call {call} against the oracle")
        with GroupBy(64 << 20, ops=ops, value_type=vt) as g:
            ref = canon({k: t.cpu().numpy() for k, t in g.run(dk, dv).items()})
        assert got.keys() == ref.keys()
        for f in ref:
            assert np.array_equal(got[f], ref[f]), f"call {call}: {f} differs from agg_run"


def test_noalloc_keys_built_to_share_one_bucket_stay_resident(oracle):
    # 400 keys whose level-0 hashes share bits 32..63 below 2^12: on the
    # spilling path they would crowd one 32-slot bucket; here they probe on
    # across slots, every group stays resident and the result is exact.
    import torch
    from paper_1311_0059_gb300 import AGG_I64
    from test_hash_adversarial_gpu import key_with_hash
    rng = np.random.default_rng(12)
    keys_set = np.unique(np.array([key_with_hash((int(rng.integers(0, 1 << 12)) << 32) |
                                                 int(rng.integers(0, 1 << 32))) for _ in range(400)], np.int64))
    n = 60_000
    keys = keys_set[rng.integers(0, keys_set.size, n)]
    vals = rng.integers(0, 1 << 20, n, dtype=np.int64)
    for call in range(2):
        st, ng, got = _call_noalloc(torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda(), 15, AGG_I64)
        assert st == 0 and ng == keys_set.size, f"call {call}: status {st}, {ng} groups"
        assert_parity(got, oracle_expected(oracle, keys, vals), 15, f"call {call}: one-bucket keys")


def test_noalloc_reports_output_capacity():
    import torch
    from paper_1311_0059_gb300 import AGG_I64, _abi
    keys = torch.arange(1000, dtype=torch.int64, device="cuda")
    st, ng, _ = _call_noalloc(keys, keys, 15, AGG_I64, capacity=999)
    assert st == _abi.AGG_ERR_OUTPUT_CAPACITY and ng == 1000
    st, ng, got = _call_noalloc(keys, keys, 15, AGG_I64)  # the next call is clean
    assert st == 0 and ng == 1000 and np.array_equal(got["keys"], np.arange(1000))


def test_noalloc_rejects_too_many_rows():
    import torch
    from paper_1311_0059_gb300 import AGG_I64, _abi
    from paper_1311_0059_gb300.groupby import Output, make_spec
    n = _abi.AGG_NOALLOC_MAX_ROWS + 1
    keys = torch.zeros(n, dtype=torch.int64, device="cuda")
    spec = make_spec(ops=1, value_type=AGG_I64)
    out = Output(n, 1, keys.device)
    st = _abi.load().agg_run_noalloc(ctypes.byref(spec), ctypes.c_void_p(keys.data_ptr()), None, n,
                                     ctypes.byref(out.abi), None, None)
    assert st == _abi.AGG_ERR_INVALID_ARG
