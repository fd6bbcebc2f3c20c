"""Parity of the GPU sort path (radix sort + segmented reduction, Section 4.1)
with the CPU oracle.  The sort path emits groups in ascending signed key
order, so its raw output is compared without re-sorting."""
import numpy as np
import pytest

import datagen as dg
from _gpu import assert_parity, canon, check_invariants, device_workload, gpu_groupby, oracle_expected, to_dev

pytestmark = pytest.mark.gpu

I64_MIN = np.iinfo(np.int64).min
I64_MAX = np.iinfo(np.int64).max
MB = 1 << 20
SORT = 1


def sort_groupby(keys, vals, budget, ops=15, **kw):
    """Sort path; returns the raw (uncanonicalised) result and stats."""
    from paper_1311_0059_gb300 import AGG_I32, AGG_I64
    from paper_1311_0059_gb300.groupby import GroupBy
    import torch
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    vt = AGG_I32 if (vals is not None and np.asarray(vals).dtype == np.int32) else AGG_I64
    with GroupBy(budget, ops=ops, value_type=vt, path=SORT, **kw) as g:
        dk = to_dev(keys) if keys.size else torch.empty(0, dtype=torch.int64, device="cuda")
        dv = None
        if vals is not None:
            v = np.ascontiguousarray(vals)
            dv = to_dev(v) if v.size else torch.empty(0, dtype=torch.from_numpy(v).dtype, device="cuda")
        res = g.run(dk, dv)
        out = {k: t.cpu().numpy() for k, t in res.items()}
        st = g.stats()
    return out, st


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


@pytest.mark.parametrize("n", [0, 1, 31, 4095, 4096, 4097, 100_003])
@pytest.mark.parametrize("ops,vd", [(15, np.int64), (15, np.int32), (3, np.int64)])
def test_sort_small_shapes_in_key_order(oracle, n, ops, vd):
    keys, vals = rand_case(n * 3 + ops, n, pool=max(1, n // 3), vdtype=vd)
    got, st = sort_groupby(keys, vals, budget=4 * MB, ops=ops)
    assert_parity(got, oracle_expected(oracle, keys, vals), ops, f"sort n={n}")


def test_sort_msd_split_and_rounds(oracle):
    # a 1 MiB budget sorts ~29k rows per round: 600k rows need an MSD split
    keys, vals = rand_case(21, 600_000, 250_000)
    got, st = sort_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals), what="msd split")
    assert st["rounds"] > 1


def test_sort_heavy_hitter_single_key_bucket(oracle):
    rng = np.random.default_rng(22)
    d, n = 20_000, 1_500_000
    dom = dg.key_of_rank(22, np.arange(d, dtype=np.uint64))
    keys = np.concatenate([np.full(n - (d - 1), dom[0]), dom[1:]])
    rng.shuffle(keys)
    vals = rng.integers(I64_MIN, I64_MAX, n, dtype=np.int64)
    got, st = sort_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals), what="heavy hitter")


def test_sort_one_key(oracle):
    vals = np.arange(2_000_000, dtype=np.int64) - 7
    keys = np.full(vals.size, -5, np.int64)
    got, _ = sort_groupby(keys, vals.astype(np.int32), budget=MB)
    assert got["keys"].tolist() == [-5] and int(got["count"][0]) == vals.size
    assert int(got["sum"][0]) == int(vals.sum()) and got["min"][0] == -7 and got["max"][0] == vals.max()


def test_sort_sorted_and_all_unique(oracle):
    rng = np.random.default_rng(23)
    keys = np.unique(rng.integers(I64_MIN, I64_MAX, 300_000, dtype=np.int64))
    vals = rng.integers(0, 1 << 20, keys.size)
    got, _ = sort_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals), what="sorted all-unique")
    rng.shuffle(keys)
    got, _ = sort_groupby(keys, vals, budget=MB)
    assert_parity(got, oracle_expected(oracle, keys, vals), what="shuffled all-unique")


def test_hash_path_equals_sort_path():
    # two independent GPU algorithms on the same input
    w = dg.Workload("cmp", n=3_000_000, domain=900_000, dist="zipf", zipf_s=0.7)
    keys, vals = w.host()
    s, _ = sort_groupby(keys, vals, budget=2 * MB)
    h, _ = gpu_groupby(keys, vals, budget=2 * MB)
    assert_parity(h, s, what="hash vs sort")


def test_sort_spill_200m_full_size_sampled(oracle):
    from paper_1311_0059_gb300.groupby import GroupBy
    from paper_1311_0059_gb300 import AGG_I64
    w = dg.SPILL_200M_50M
    keys, vals, _ = device_workload(w)
    with GroupBy(w.budget, ops=w.ops, value_type=AGG_I64, path=SORT) as g:
        res = g.run(keys, vals)
        st = g.stats()
    got = {k: t.cpu().numpy() for k, t in res.items()}
    check_invariants(got, w.n, vals.cpu().numpy().view(np.uint64).sum(dtype=np.uint64))
    hk, hv = keys.cpu().numpy(), vals.cpu().numpy()
    distinct = np.count_nonzero(np.bincount(dg.rank_of_key(w.seed, hk).astype(np.int64), minlength=w.domain))
    assert got["keys"].size == distinct
    rng = np.random.default_rng(1)
    idx = rng.choice(got["keys"].size, 48, replace=False)
    ref = oracle.groups_of(hk, hv, got["keys"][idx])
    for f in ("count", "sum", "min", "max"):
        assert np.array_equal(got[f][idx].astype(np.int64), ref[f].astype(np.int64)), f
