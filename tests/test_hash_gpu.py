"""Parity of the GPU hash path (Pre-Partitioning hybrid hash) with the CPU
oracle: element by element after a canonical sort, bit-exact (all aggregates
are integers)."""
import numpy as np
import pytest

import datagen as dg
from _gpu import assert_parity, canon, check_invariants, device_workload, gpu_groupby, oracle_expected

pytestmark = pytest.mark.gpu

I64_MIN = np.iinfo(np.int64).min
I64_MAX = np.iinfo(np.int64).max
MB = 1 << 20


def rand_case(seed, n, pool, vdtype=np.int64):
    rng = np.random.default_rng(seed)
    special = np.array([I64_MIN, I64_MIN + 1, -1, 0, 1, I64_MAX], np.int64)
    dom = np.concatenate([special, rng.integers(I64_MIN, I64_MAX, max(pool, 1), dtype=np.int64, endpoint=True)])
    keys = dom[rng.integers(0, dom.size, n)]
    if vdtype == np.int32:
        vals = rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(np.int32)
    else:
        vals = rng.integers(I64_MIN, I64_MAX, n, dtype=np.int64, endpoint=True)
    return keys, vals


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 2047, 2048, 2049, 100_003])
@pytest.mark.parametrize("ops,vd", [(15, np.int64), (15, np.int32), (3, np.int64), (1, np.int64), (12, np.int32)])
def test_small_shapes(oracle, n, ops, vd):
    keys, vals = rand_case(n * 7 + ops, n, pool=max(1, n // 3), vdtype=vd)
    got, st = gpu_groupby(keys, vals, budget=4 * MB, ops=ops)
    assert_parity(got, oracle_expected(oracle, keys, vals), ops, f"n={n} ops={ops}")
    assert st["n_groups"] == got["keys"].size


def test_one_key_is_scalar_aggregation(oracle):
    rng = np.random.default_rng(1)
    vals = rng.integers(I64_MIN, I64_MAX, 300_000, dtype=np.int64)
    keys = np.full(vals.size, 42, np.int64)
    got, _ = gpu_groupby(keys, vals, budget=MB)
    assert got["keys"].tolist() == [42] and int(got["count"][0]) == vals.size
    assert got["sum"][0] == vals.view(np.uint64).sum(dtype=np.uint64).view(np.int64)
    assert got["min"][0] == vals.min() and got["max"][0] == vals.max()


def test_sentinel_like_keys(oracle):
    keys = np.array([I64_MIN, I64_MIN, I64_MAX, 0, -1, I64_MIN + 1] * 1000, np.int64)
    vals = np.arange(keys.size, dtype=np.int64)
    got, _ = gpu_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals))


def test_all_unique_spills_and_recurses(oracle):
    # 100% cardinality (Section 6.1): every row is its own group; with a 1 MiB
    # budget the table holds ~8k groups, so the rest spill and recurse.
    rng = np.random.default_rng(2)
    keys = np.unique(rng.integers(I64_MIN, I64_MAX, 400_000, dtype=np.int64))
    rng.shuffle(keys)
    vals = rng.integers(0, 1 << 40, keys.size)
    got, st = gpu_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals))
    assert st["levels"] >= 2 and sum(st["spill_records"]) > 0


def test_forced_multilevel_recursion(oracle):
    # many groups under the minimum budget and a small fan-out force >= 3 levels
    from paper_1311_0059_gb300 import agg_tuning
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 3_000_000, 2_000_000).astype(np.int64) * 7919
    vals = rng.integers(0, 1 << 20, keys.size)
    got, st = gpu_groupby(keys, vals, budget=MB, tuning=agg_tuning(fan_out=16))
    assert_parity(got, oracle_expected(oracle, keys, vals))
    assert st["levels"] >= 3


def test_heavy_hitter(oracle):
    # Section 6.4 heavy hitter, scaled: one key carries n - (D - 1) rows.
    rng = np.random.default_rng(4)
    d, n = 200_000, 3_000_000
    dom = dg.key_of_rank(4, np.arange(d, dtype=np.uint64))
    keys = np.concatenate([np.full(n - (d - 1), dom[0]), dom[1:]])
    rng.shuffle(keys)
    vals = rng.integers(0, 1 << 20, n)
    got, st = gpu_groupby(keys, vals, budget=2 * MB)
    assert_parity(got, oracle_expected(oracle, keys, vals))


def test_heavy_hitter_arrives_after_full(oracle):
    # the heavy key first appears once the table is already full: it must spill whole
    rng = np.random.default_rng(5)
    others = np.unique(rng.integers(I64_MIN, I64_MAX, 300_000, dtype=np.int64))
    hot = np.int64(123456789)
    others = others[others != hot]
    keys = np.concatenate([others, np.full(1_000_000, hot)])
    vals = rng.integers(0, 1 << 20, keys.size)
    got, st = gpu_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals))


def test_sorted_input(oracle):
    w = dg.Workload("sorted", n=2_000_000, domain=300_000)
    keys, vals = w.host()
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    got, _ = gpu_groupby(keys, vals, budget=2 * MB)
    assert_parity(got, oracle_expected(oracle, keys, vals))


def test_plain_1m_10k_int32_full_size(oracle):
    # the plain in-budget workload at its full size (1M rows, 10k keys, int32 values, 64 MB)
    w = dg.PLAIN_1M_10K
    keys, vals = w.host()
    got, st = gpu_groupby(keys, vals, budget=w.budget, ops=w.ops)
    assert_parity(got, oracle_expected(oracle, keys, vals), w.ops)
    assert st["levels"] == 1 and sum(st["spill_records"]) == 0


def test_spill_workload_scaled(oracle):
    # the spilling workload scaled to 4M rows / 1M-key domain under a 4 MB budget
    w = dg.Workload("spill-scaled", n=4_000_000, domain=1_000_000, budget=4 * MB)
    keys, vals = w.host()
    got, st = gpu_groupby(keys, vals, budget=w.budget)
    assert_parity(got, oracle_expected(oracle, keys, vals))
    assert st["levels"] >= 2


def test_zipf_workload_scaled(oracle):
    w = dg.Workload("zipf-scaled", n=4_000_000, domain=500_000, dist="zipf", zipf_s=1.0, budget=64 * MB, ops=3)
    keys, vals = w.host()
    got, st = gpu_groupby(keys, vals, budget=w.budget, ops=3)
    assert_parity(got, oracle_expected(oracle, keys, vals), 3)


@pytest.mark.parametrize("tune", [dict(), dict(max_load_factor=0.9), dict(smem_entries=1), dict(smem_entries=256),
                                  dict(warp_dedup=1), dict(warp_dedup=2), dict(fan_out=256),
                                  dict(max_load_factor=0.2, fan_out=16), dict(level0_slots=4096),
                                  dict(level0_slots=1)])
def test_result_invariant_under_tuning(oracle, tune):
    from paper_1311_0059_gb300 import agg_tuning
    w = dg.Workload("tune", n=1_500_000, domain=400_000, dist="zipf", zipf_s=0.8)
    keys, vals = w.host()
    got, _ = gpu_groupby(keys, vals, budget=2 * MB, tuning=agg_tuning(**tune))
    assert_parity(got, oracle_expected(oracle, keys, vals), what=str(tune))


def test_level0_cap_spills_groups_the_whole_table_would_hold(oracle):
    # 20k groups fit the 8 MB budget's table: uncapped, level 0 completes them
    # all; capped at 4096 slots, the groups that fill the small table first
    # stay resident and the rows of the others spill to level 1.  The result
    # is the same.
    from paper_1311_0059_gb300 import agg_tuning
    keys, vals = rand_case(21, 400_000, 20_000)
    exp = oracle_expected(oracle, keys, vals)
    whole, st_w = gpu_groupby(keys, vals, budget=8 * MB, tuning=agg_tuning(level0_slots=1, sorted_input=2))
    assert_parity(whole, exp, what="whole table")
    assert st_w["spill_records"][0] == 0 and st_w["levels"] == 1
    capped, st_c = gpu_groupby(keys, vals, budget=8 * MB, tuning=agg_tuning(level0_slots=4096, sorted_input=2))
    assert_parity(capped, exp, what="level-0 table capped at 4096 slots")
    assert st_c["spill_records"][0] > 0 and st_c["levels"] >= 2
    assert st_c["resident_groups"][0] <= 4096 + 1  # the capped table, and the side slot of INT64_MIN


@pytest.mark.parametrize("hint", [1, 1000, 400_000, 10**9])
def test_result_invariant_under_expected_groups(oracle, hint):
    # Section 6.6: the estimate of G only changes the plan, never the result
    w = dg.Workload("hint", n=1_000_000, domain=300_000)
    keys, vals = w.host()
    got, _ = gpu_groupby(keys, vals, budget=4 * MB, expected_groups=hint)
    assert_parity(got, oracle_expected(oracle, keys, vals), what=f"hint {hint}")


def test_seed_changes_nothing_but_placement(oracle):
    keys, vals = rand_case(9, 500_000, 200_000)
    exp = oracle_expected(oracle, keys, vals)
    for seed in (0, 1, 0xDEADBEEF):
        got, _ = gpu_groupby(keys, vals, budget=MB, seed=seed)
        assert_parity(got, exp, what=f"seed {seed}")


def test_repeated_runs_on_one_handle(oracle):
    # the table is reset by emit: a handle gives the same result run after run
    import torch
    from paper_1311_0059_gb300.groupby import GroupBy
    from _gpu import to_dev
    keys, vals = rand_case(10, 300_000, 100_000)
    exp = oracle_expected(oracle, keys, vals)
    with GroupBy(MB) as g:
        dk, dv = to_dev(keys), to_dev(vals)
        for _ in range(3):
            res = g.run(dk, dv)
            assert_parity(canon({k: t.cpu().numpy() for k, t in res.items()}), exp)


def test_output_capacity_error():
    from paper_1311_0059_gb300._abi import AGG_ERR_OUTPUT_CAPACITY, AggError
    keys, vals = rand_case(11, 10_000, 5_000)
    with pytest.raises(AggError) as e:
        gpu_groupby(keys, vals, budget=MB, capacity=10)
    assert e.value.status == AGG_ERR_OUTPUT_CAPACITY


def test_host_pointer_rejected():
    import ctypes
    from paper_1311_0059_gb300._abi import AGG_ERR_INVALID_ARG
    from paper_1311_0059_gb300.groupby import GroupBy
    import torch
    keys = np.arange(100, dtype=np.int64)
    with GroupBy(MB) as g:
        out = g.output(100, "cuda")
        st = g.lib.agg_run(g.h, ctypes.c_void_p(keys.ctypes.data), ctypes.c_void_p(keys.ctypes.data), 100,
                           ctypes.byref(out.abi), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == AGG_ERR_INVALID_ARG


def test_run_host_matches_device(oracle):
    from paper_1311_0059_gb300.groupby import GroupBy
    keys, vals = rand_case(12, 700_000, 300_000)
    with GroupBy(2 * MB) as g:
        got = canon(g.run_host(keys, vals))
    assert_parity(got, oracle_expected(oracle, keys, vals))


def test_device_generator_matches_host():
    import torch
    for w in (dg.Workload("u", n=300_001, domain=77_777, vtype="i32_1000", seed=5),
              dg.Workload("z", n=300_001, domain=50_000, dist="zipf", zipf_s=1.1, seed=6)):
        k, v, _ = device_workload(w)
        hk, hv = w.host()
        assert np.array_equal(k.cpu().numpy(), hk)
        assert np.array_equal(v.cpu().numpy(), hv)


def _sampled_full_size(oracle, w, m=48):
    import torch
    from paper_1311_0059_gb300.groupby import GroupBy
    from paper_1311_0059_gb300 import AGG_I64
    keys, vals, _ = device_workload(w)
    with GroupBy(w.budget, ops=w.ops, value_type=AGG_I64) as g:
        res = g.run(keys, vals)
        st = g.stats()
    got = canon({k: t.cpu().numpy() for k, t in res.items()})
    hk, hv = keys.cpu().numpy(), vals.cpu().numpy()
    check_invariants(got, w.n, hv.view(np.uint64).sum(dtype=np.uint64))
    ranks = dg.rank_of_key(w.seed, got["keys"])
    assert np.all(ranks < w.domain), "a group key outside the key domain"
    distinct = np.count_nonzero(np.bincount(dg.rank_of_key(w.seed, hk).astype(np.int64), minlength=w.domain))
    assert got["keys"].size == distinct
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([rng.choice(got["keys"].size, m, replace=False),
                                    np.argsort(got["count"])[-8:]]))
    ref = oracle.groups_of(hk, hv, got["keys"][idx])
    for f in ("count", "sum", "min", "max"):
        if f in got:
            assert np.array_equal(got[f][idx].astype(np.int64), ref[f].astype(np.int64)), f
    return st


def test_spill_200m_50m_full_size_sampled(oracle):
    st = _sampled_full_size(oracle, dg.SPILL_200M_50M)
    assert st["levels"] >= 2


def test_zipf_500m_10m_full_size_sampled(oracle):
    st = _sampled_full_size(oracle, dg.ZIPF_500M_10M)
    assert st["levels"] == 2  # level-0 table capped at 2^22 slots: the tail spills once


def _run_host_pinned(g, keys, vals, capacity):
    """agg_run_host on pinned host tensors (the path the end-to-end bench takes)."""
    import ctypes

    import torch
    from paper_1311_0059_gb300._abi import agg_output
    hk = torch.from_numpy(keys).pin_memory()
    hv = torch.from_numpy(vals).pin_memory()
    out = {f: torch.empty(max(capacity, 1), dtype=torch.int64).pin_memory() for f in ("keys", "count", "sum", "min", "max")}
    ho = agg_output(keys=out["keys"].data_ptr(), count=out["count"].data_ptr(), sum=out["sum"].data_ptr(),
                    min=out["min"].data_ptr(), max=out["max"].data_ptr(), capacity=capacity, d_n_groups=None)
    ng = ctypes.c_uint64()
    st = g.lib.agg_run_host(g.h, ctypes.c_void_p(hk.data_ptr()), ctypes.c_void_p(hv.data_ptr()), keys.size,
                            ctypes.byref(ho), ctypes.byref(ng), None)
    res = {f: t.numpy()[:min(ng.value, capacity)] for f, t in out.items()}
    return st, ng.value, res


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("vd", [np.int64, np.int32])
def test_run_host_pinned_spilling(oracle, path, vd):
    # pinned host buffers: the hash path reads the input and writes the result
    # in host memory directly; the sort path copies
    from paper_1311_0059_gb300 import AGG_I32, AGG_I64
    from paper_1311_0059_gb300.groupby import GroupBy
    keys, vals = rand_case(21 + path, 900_000, 400_000, vdtype=vd)
    with GroupBy(MB, value_type=AGG_I32 if vd == np.int32 else AGG_I64, path=path) as g:
        st, ng, res = _run_host_pinned(g, keys, vals, keys.size)
        assert st == 0
        if path == 0:
            assert g.stats()["levels"] >= 2
    assert_parity(canon(res), oracle_expected(oracle, keys, vals), what=f"path={path}")


def test_run_host_pinned_output_capacity(oracle):
    from paper_1311_0059_gb300 import _abi
    from paper_1311_0059_gb300.groupby import GroupBy
    keys, vals = rand_case(23, 100_000, 5_000)
    exp = oracle_expected(oracle, keys, vals)
    with GroupBy(8 * MB) as g:
        st, ng, _ = _run_host_pinned(g, keys, vals, exp["keys"].size - 1)
        assert st == _abi.AGG_ERR_OUTPUT_CAPACITY
        assert ng == exp["keys"].size
        st, ng, res = _run_host_pinned(g, keys, vals, exp["keys"].size)  # the handle is usable again
        assert st == 0 and ng == exp["keys"].size
    assert_parity(canon(res), exp)


def test_run_host_count_only_without_values(oracle):
    # COUNT needs no values: the direct mode runs with h_vals = NULL
    import ctypes

    import torch
    from paper_1311_0059_gb300 import AGG_COUNT
    from paper_1311_0059_gb300._abi import agg_output
    from paper_1311_0059_gb300.groupby import GroupBy
    keys, vals = rand_case(31, 500_000, 200_000)
    exp = oracle_expected(oracle, keys, vals)
    with GroupBy(MB, ops=AGG_COUNT) as g:
        hk = torch.from_numpy(keys).pin_memory()
        ok_ = torch.empty(keys.size, dtype=torch.int64).pin_memory()
        oc = torch.empty(keys.size, dtype=torch.int64).pin_memory()
        ho = agg_output(keys=ok_.data_ptr(), count=oc.data_ptr(), sum=None, min=None, max=None, capacity=keys.size,
                        d_n_groups=None)
        ng = ctypes.c_uint64()
        st = g.lib.agg_run_host(g.h, ctypes.c_void_p(hk.data_ptr()), None, keys.size, ctypes.byref(ho),
                                ctypes.byref(ng), None)
        assert st == 0 and ng.value == exp["keys"].size
    got = canon({"keys": ok_.numpy()[:ng.value], "count": oc.numpy()[:ng.value]})
    assert_parity(got, exp, AGG_COUNT)


@pytest.mark.parametrize("path", [0, 1])
def test_run_host_pageable_both_paths(oracle, path):
    from paper_1311_0059_gb300.groupby import GroupBy
    keys, vals = rand_case(32 + path, 300_000, 120_000)
    with GroupBy(MB, path=path) as g:
        got = canon(g.run_host(keys, vals))
        empty = g.run_host(keys[:0], vals[:0])
    assert_parity(got, oracle_expected(oracle, keys, vals), what=f"path={path}")
    assert empty["keys"].size == 0


def test_run_host_pinned_empty_input(oracle):
    from paper_1311_0059_gb300.groupby import GroupBy
    with GroupBy(MB) as g:
        st, ng, _ = _run_host_pinned(g, np.zeros(0, np.int64), np.zeros(0, np.int64), 1)
    assert st == 0 and ng == 0
