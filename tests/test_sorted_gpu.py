"""Parity of the sorted-input path with the CPU oracle.

On sorted input the Sort-based algorithm's sort degenerates to a scan (Section
6.4), so the hash kernel first checks a sample of adjacent key pairs and, if it
is in order, aggregates with one segmented reduction and no table; a descent
found by the full check sends the run back to the hash path.  Every case is
compared element by element with the oracle; the stats counter tells which
path ran."""
import numpy as np
import pytest

from _gpu import assert_parity, gpu_groupby, oracle_expected

pytestmark = pytest.mark.gpu

I64_MIN = np.iinfo(np.int64).min
I64_MAX = np.iinfo(np.int64).max
MB = 1 << 20


def _tuning(**kw):
    from paper_1311_0059_gb300 import agg_tuning
    return agg_tuning(**kw)


def _sorted_case(seed, n, pool, vd=np.int64):
    rng = np.random.default_rng(seed)
    dom = np.concatenate([[I64_MIN, I64_MIN + 1, -1, 0, 1, I64_MAX],
                          rng.integers(I64_MIN, I64_MAX, max(pool, 1), dtype=np.int64)])
    keys = np.sort(dom[rng.integers(0, dom.size, n)])
    vals = (rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(np.int32) if vd == np.int32 else
            rng.integers(I64_MIN, I64_MAX, n, dtype=np.int64, endpoint=True))
    return keys, vals


NO_IN_BUDGET = dict(in_budget=2)  # small inputs would otherwise take the in-budget paths


@pytest.mark.parametrize("n", [2, 3, 2047, 2048, 2049, 100_001, 1_000_003])
@pytest.mark.parametrize("ops,vd", [(15, np.int64), (15, np.int32), (3, np.int64), (1, np.int64), (12, np.int32)])
def test_sorted_shapes(oracle, n, ops, vd):
    keys, vals = _sorted_case(n + ops, n, pool=max(1, n // 3), vd=vd)
    got, st = gpu_groupby(keys, vals, budget=MB, ops=ops, tuning=_tuning(**NO_IN_BUDGET))
    assert_parity(got, oracle_expected(oracle, keys, vals), ops, f"sorted n={n} ops={ops}")
    assert st["sorted_input"] == 1 and st["levels"] == 1 and st["n_groups"] == got["keys"].size


def test_segments_spanning_many_blocks(oracle):
    # three keys over 3M rows: every block's range lies inside one segment or
    # two, and the blocks' leading partials are added across block boundaries
    rng = np.random.default_rng(1)
    n = 3_000_000
    keys = np.sort(rng.choice(np.array([-7, 5, 9], np.int64), n, p=[0.1, 0.85, 0.05]))
    vals = rng.integers(-2**40, 2**40, n, dtype=np.int64)
    got, st = gpu_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals), what="three long segments")
    assert st["sorted_input"] == 1
    one = np.full(n, 3, np.int64)
    got, st = gpu_groupby(one, vals, budget=MB)
    assert st["sorted_input"] == 1 and got["keys"].tolist() == [3] and int(got["count"][0]) == n
    assert got["sum"][0] == vals.view(np.uint64).sum(dtype=np.uint64).view(np.int64)
    assert got["min"][0] == vals.min() and got["max"][0] == vals.max()


def test_all_unique_sorted(oracle):
    rng = np.random.default_rng(2)
    keys = np.unique(rng.integers(I64_MIN, I64_MAX, 2_500_000, dtype=np.int64))
    vals = rng.integers(0, 1 << 20, keys.size, dtype=np.int64)
    got, st = gpu_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals), what="all unique, sorted")
    assert st["sorted_input"] == 1 and st["n_groups"] == keys.size


def test_one_late_descent_falls_back_to_the_hash_path(oracle):
    # the sample sees sorted pairs; the full check finds the one descent and
    # the run completes on the hash path
    keys, vals = _sorted_case(3, 1_500_000, 400_000)
    keys[1_234_567], keys[1_234_568] = keys[1_234_568] + 1, keys[1_234_567]
    assert keys[1_234_567] > keys[1_234_568] or keys[1_234_567] > keys[1_234_566]
    got, st = gpu_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals), what="one descent")
    assert st["sorted_input"] == 0


def test_unsorted_and_descending_take_the_hash_path(oracle):
    keys, vals = _sorted_case(4, 800_000, 200_000)
    for k in (keys[::-1].copy(), np.random.default_rng(5).permutation(keys)):
        got, st = gpu_groupby(k, vals, budget=MB)
        assert_parity(got, oracle_expected(oracle, k, vals), what="not sorted")
        assert st["sorted_input"] == 0


def test_sorted_path_off_gives_the_same_result(oracle):
    keys, vals = _sorted_case(6, 1_000_000, 300_000)
    exp = oracle_expected(oracle, keys, vals)
    on, st_on = gpu_groupby(keys, vals, budget=MB)
    off, st_off = gpu_groupby(keys, vals, budget=MB, tuning=_tuning(sorted_input=2))
    assert st_on["sorted_input"] == 1 and st_off["sorted_input"] == 0
    assert_parity(on, exp, what="sorted path")
    assert_parity(off, exp, what="hash path on sorted input")


def test_sorted_output_capacity():
    from paper_1311_0059_gb300._abi import AGG_ERR_OUTPUT_CAPACITY, AggError
    keys = np.arange(50_000, dtype=np.int64)
    with pytest.raises(AggError) as e:
        gpu_groupby(keys, keys, budget=MB, capacity=100, tuning=_tuning(**NO_IN_BUDGET))
    assert e.value.status == AGG_ERR_OUTPUT_CAPACITY


def test_sorted_path_twice_on_one_handle_then_hash(oracle):
    # the control block's sorted-path fields are reset run after run
    from _gpu import canon, to_dev
    from paper_1311_0059_gb300.groupby import GroupBy
    a = _sorted_case(7, 600_000, 100_000)
    b = _sorted_case(8, 900_000, 500_000)
    c = (np.random.default_rng(9).permutation(b[0]), b[1])
    with GroupBy(MB) as g:
        for keys, vals in (a, b, c, a):
            res = canon({k: t.cpu().numpy() for k, t in g.run(to_dev(keys), to_dev(vals)).items()})
            assert_parity(res, oracle_expected(oracle, keys, vals))
