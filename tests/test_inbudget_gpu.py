"""Parity of the in-budget paths with the CPU oracle.

When every group of a run fits the table at once (n at most half the slots),
the group-by completes in place with no partitioning of the spilled kind
(Section 4.3.4: a table that never fills).  Small inputs are split by hash into
partitions that thread blocks aggregate in shared memory (keys that do not fit
a block's table go to a global table probed linearly); larger ones use that
global table directly.  Every case is compared element by element with the
oracle and with the spilling path (the in_budget tuning knob set to off)."""
import numpy as np
import pytest

import datagen as dg
from _gpu import assert_parity, canon, gpu_groupby, oracle_expected, to_dev

pytestmark = pytest.mark.gpu

I64_MIN = np.iinfo(np.int64).min
I64_MAX = np.iinfo(np.int64).max
MB = 1 << 20


def _tuning(**kw):
    from paper_1311_0059_gb300 import agg_tuning
    return agg_tuning(**kw)


def _case(seed, n, pool, vd=np.int64):
    rng = np.random.default_rng(seed)
    special = np.array([I64_MIN, I64_MIN + 1, -1, 0, 1, I64_MAX], np.int64)
    dom = np.concatenate([special, rng.integers(I64_MIN, I64_MAX, max(pool, 1), dtype=np.int64, endpoint=True)])
    keys = dom[rng.integers(0, dom.size, n)]
    vals = (rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(np.int32) if vd == np.int32 else
            rng.integers(I64_MIN, I64_MAX, n, dtype=np.int64, endpoint=True))
    return keys, vals


def _plan_path(budget, n, ops, vt, tuning=None):
    from paper_1311_0059_gb300.groupby import make_spec, plan
    return plan(budget, n, make_spec(ops=ops, value_type=vt), tuning)["in_budget_path"]


@pytest.mark.parametrize("n", [1, 2, 4095, 4096, 4097, 100_003, 1_000_000, 2_097_152])
@pytest.mark.parametrize("ops,vd", [(15, np.int64), (15, np.int32), (3, np.int64), (1, np.int64), (12, np.int32)])
def test_partitioned_path_shapes(oracle, n, ops, vd):
    from paper_1311_0059_gb300 import AGG_I32, AGG_I64
    vt = AGG_I32 if vd == np.int32 else AGG_I64
    budget = 256 * MB
    assert _plan_path(budget, n, ops, vt) == 1
    keys, vals = _case(n * 5 + ops, n, pool=max(1, n // 4), vd=vd)
    exp = oracle_expected(oracle, keys, vals)
    got, st = gpu_groupby(keys, vals, budget=budget, ops=ops)
    assert_parity(got, exp, ops, f"partitioned n={n} ops={ops}")
    assert st["levels"] == 1 and sum(st["spill_records"]) == 0 and st["n_groups"] == got["keys"].size


@pytest.mark.parametrize("ops,vd", [(15, np.int64), (3, np.int64), (15, np.int32)])
def test_table_path_matches_oracle_and_spilling_path(oracle, ops, vd):
    # past the partitioned path's 2M rows, below half the slots: the single table
    from paper_1311_0059_gb300 import AGG_I32, AGG_I64
    vt = AGG_I32 if vd == np.int32 else AGG_I64
    n, budget = 2_600_000, 512 * MB
    assert _plan_path(budget, n, ops, vt) == 2
    keys, vals = _case(77 + ops, n, pool=700_000, vd=vd)
    exp = oracle_expected(oracle, keys, vals)
    got, st = gpu_groupby(keys, vals, budget=budget, ops=ops)
    assert_parity(got, exp, ops, "table path")
    assert st["levels"] == 1
    spill, _ = gpu_groupby(keys, vals, budget=budget, ops=ops, tuning=_tuning(in_budget=2))
    assert_parity(spill, exp, ops, "same input on the spilling path")


def test_table_path_without_shared_memory_tables(oracle):
    keys, vals = _case(5, 300_000, 50_000)
    assert _plan_path(64 * MB, keys.size, 15, 1, _tuning(smem_entries=1)) == 2
    got, _ = gpu_groupby(keys, vals, budget=64 * MB, tuning=_tuning(smem_entries=1))
    assert_parity(got, oracle_expected(oracle, keys, vals), what="single table, no shared-memory cache")


def test_heavy_hitter_and_one_key_on_the_in_budget_paths(oracle):
    rng = np.random.default_rng(3)
    n = 1_500_000
    keys = np.where(rng.random(n) < 0.7, 99, rng.integers(0, 200_000, n)).astype(np.int64)
    vals = rng.integers(-2**40, 2**40, n, dtype=np.int64)
    for tune in (None, _tuning(smem_entries=1)):
        got, _ = gpu_groupby(keys, vals, budget=128 * MB, tuning=tune)
        assert_parity(got, oracle_expected(oracle, keys, vals), what=f"heavy hitter, tuning {tune}")
    one = np.full(n, -5, np.int64)
    got, _ = gpu_groupby(one, vals, budget=128 * MB)
    assert got["keys"].tolist() == [-5] and int(got["count"][0]) == n
    assert got["min"][0] == vals.min() and got["max"][0] == vals.max()


def test_partition_overflow_goes_to_the_global_table(oracle):
    # 6,000 distinct keys whose level-0 hashes share their top 12 bits: all fall
    # in one partition, three times what a block's 2,048-entry table holds; the
    # keys that do not fit are aggregated in the global table and emitted by the
    # last block.  The empty-marker key value rides along in the side slot.
    from test_hash_adversarial_gpu import key_with_hash
    rng = np.random.default_rng(21)
    ks = np.unique(np.array([key_with_hash((int(rng.integers(0, 1 << 20)) << 32) | int(rng.integers(0, 1 << 32)))
                             for _ in range(6000)], np.int64))
    n = 200_000
    keys = ks[rng.integers(0, ks.size, n)]
    keys[::997] = I64_MIN
    vals = rng.integers(-2**50, 2**50, n, dtype=np.int64)
    exp = oracle_expected(oracle, keys, vals)
    assert _plan_path(64 * MB, n, 15, 1) == 1
    for _ in range(2):  # twice on fresh handles: the overflow table is emptied by its emit
        got, st = gpu_groupby(keys, vals, budget=64 * MB)
        assert_parity(got, exp, what="partition overflow")


def test_one_handle_alternates_paths(oracle):
    # the partitioned path leaves its scratch records in the top entries; a
    # spilling run, a table run and partitioned runs of other sizes on the same
    # handle must each start from a clean table
    from paper_1311_0059_gb300.groupby import GroupBy
    cases = [_case(31, 50_000, 20_000), _case(32, 3_000_000, 2_000_000), _case(33, 1_800_000, 900_000),
             _case(34, 2_500_000, 100_000), _case(35, 7, 3), _case(36, 1_000_000, 10_000)]
    with GroupBy(96 * MB) as g:
        for i, (keys, vals) in enumerate(cases):
            res = g.run(to_dev(keys), to_dev(vals))
            got = canon({k: t.cpu().numpy() for k, t in res.items()})
            assert_parity(got, oracle_expected(oracle, keys, vals), what=f"run {i} ({keys.size} rows)")


def test_plain_workload_on_the_partitioned_path(oracle):
    # the plain 1M-row, 10k-key, int32 workload at full size, generated on the device
    from _gpu import device_workload
    w = dg.PLAIN_1M_10K
    keys, vals, _ = device_workload(w)
    from paper_1311_0059_gb300 import AGG_I32
    from paper_1311_0059_gb300.groupby import GroupBy
    assert _plan_path(w.budget, w.n, w.ops, AGG_I32) == 1
    with GroupBy(w.budget, ops=w.ops, value_type=AGG_I32) as g:
        for _ in range(3):
            res = g.run(keys, vals)
            got = canon({k: t.cpu().numpy() for k, t in res.items()})
    hk, hv = w.host()
    assert_parity(got, oracle_expected(oracle, hk, hv), w.ops, "plain 1M/10k")


def test_output_capacity_on_the_in_budget_paths():
    from paper_1311_0059_gb300._abi import AGG_ERR_OUTPUT_CAPACITY, AggError
    keys, vals = _case(11, 10_000, 5_000)
    for tune in (None, _tuning(smem_entries=1)):
        with pytest.raises(AggError) as e:
            gpu_groupby(keys, vals, budget=32 * MB, capacity=10, tuning=tune)
        assert e.value.status == AGG_ERR_OUTPUT_CAPACITY
