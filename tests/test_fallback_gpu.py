"""The recursion fallback of the hash path (Section 4.3): records that
partitioning no longer shrinks are sorted by key inside the run and reduced by
segments.  It engages when a level reaches the depth cap (agg_tuning
.max_levels), or when the records the level before completed formed more than
0.8 groups per record (all-unique keys: the output is the whole input).  Each
case is compared element by element with the oracle; the stats counters tell
where the fallback ran."""
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


def test_depth_cap_two_on_a_multilevel_input(oracle):
    # many groups under the minimum budget and fan-out 16 need three or more
    # levels; with a cap of 2 the records reaching level 2 are sorted instead
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 600_000, 1_000_000).astype(np.int64) * 7919
    vals = rng.integers(0, 1 << 20, keys.size)
    exp = oracle_expected(oracle, keys, vals)
    deep, st = gpu_groupby(keys, vals, budget=MB, tuning=_tuning(fan_out=16, sorted_input=2))
    assert_parity(deep, exp, what="uncapped")
    assert st["levels"] >= 3 and st["fallback_records"] == 0
    got, st = gpu_groupby(keys, vals, budget=MB, tuning=_tuning(fan_out=16, max_levels=2, sorted_input=2))
    assert_parity(got, exp, what="depth cap 2")
    assert st["fallback_level"] == 2 and st["fallback_records"] > 0 and st["levels"] == 3


@pytest.mark.parametrize("ops,vd", [(15, np.int64), (15, np.int32), (3, np.int64), (12, np.int32), (1, np.int64)])
def test_depth_cap_one_sorts_every_spilled_record(oracle, ops, vd):
    rng = np.random.default_rng(10 + ops)
    n = 700_003
    dom = np.concatenate([[I64_MIN, I64_MIN + 1, -1, 0, I64_MAX], rng.integers(I64_MIN, I64_MAX, 250_000,
                                                                                  dtype=np.int64)])
    keys = dom[rng.integers(0, dom.size, n)]
    vals = (rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(np.int32) if vd == np.int32 else
            rng.integers(I64_MIN, I64_MAX, n, dtype=np.int64, endpoint=True))
    got, st = gpu_groupby(keys, vals, budget=MB, ops=ops, tuning=_tuning(max_levels=1))
    assert_parity(got, oracle_expected(oracle, keys, vals), ops, f"cap 1, ops={ops}")
    assert st["fallback_level"] == 1 and st["fallback_records"] == st["spill_records"][0] > 0
    assert st["levels"] == 2


def test_all_unique_keys_fall_back_after_level_0(oracle):
    # every row its own group: the resident part of level 0 shows one group per
    # row, so level 1 sorts the spilled rows instead of partitioning them again
    rng = np.random.default_rng(2)
    keys = np.unique(rng.integers(I64_MIN, I64_MAX, 600_000, dtype=np.int64))
    rng.shuffle(keys)
    vals = rng.integers(0, 1 << 40, keys.size)
    got, st = gpu_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals), what="all unique")
    assert st["fallback_level"] == 1 and st["fallback_records"] > 0 and st["n_groups"] == keys.size


def test_low_cardinality_spill_does_not_fall_back(oracle):
    # four rows per key: partitioning shrinks the data, the hash levels run
    rng = np.random.default_rng(6)
    keys = rng.integers(0, 250_000, 1_000_000).astype(np.int64) * 104729
    vals = rng.integers(0, 1 << 20, keys.size)
    got, st = gpu_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals), what="4 rows per key")
    assert st["levels"] >= 2 and st["fallback_records"] == 0


def test_fallback_twice_on_one_handle_then_without(oracle):
    from _gpu import canon, to_dev
    from paper_1311_0059_gb300.groupby import GroupBy
    rng = np.random.default_rng(7)
    uniq = np.unique(rng.integers(I64_MIN, I64_MAX, 300_000, dtype=np.int64))
    rng.shuffle(uniq)
    dup = rng.integers(0, 200_000, 900_000).astype(np.int64) * 31
    cases = [(uniq, rng.integers(0, 99, uniq.size)), (uniq[::-1].copy(), rng.integers(0, 99, uniq.size)),
             (dup, rng.integers(0, 99, dup.size))]
    with GroupBy(MB) as g:
        for keys, vals in cases + cases[:1]:
            res = canon({k: t.cpu().numpy() for k, t in g.run(to_dev(keys), to_dev(vals)).items()})
            assert_parity(res, oracle_expected(oracle, keys, vals))


def test_batched_instances_with_unique_keys(oracle):
    # the batched form shares the kernel: instances of all-unique keys fall back too
    import torch
    from paper_1311_0059_gb300 import AGG_I64
    from paper_1311_0059_gb300.groupby import Batch
    rng = np.random.default_rng(8)
    inst, data = [], []
    for i in range(12):
        n = int(rng.integers(50_000, 300_000))
        keys = np.unique(rng.integers(I64_MIN, I64_MAX, n, dtype=np.int64)) if i % 2 else \
            rng.integers(0, n // 3, n).astype(np.int64)
        rng.shuffle(keys)
        vals = rng.integers(-1000, 1000, keys.size)
        data.append((keys, vals))
        inst.append((torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda(), MB, 0))
    b = Batch(inst, ops=15, value_type=AGG_I64)
    res = b.run()
    for i, ((keys, vals), r) in enumerate(zip(data, res)):
        got = {f: t.cpu().numpy() for f, t in r.items()}
        o = np.argsort(got["keys"], kind="stable")
        assert_parity({f: a[o] for f, a in got.items()}, oracle_expected(oracle, keys, vals), what=f"instance {i}")
    b.close()
