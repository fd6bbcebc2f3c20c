"""Pins for the CPU oracle: checks against facts that do not come from the oracle.

Each pin takes an ``oracle.Oracle`` and raises AssertionError on a mismatch, so
the same pins run against the real oracle (tests/test_oracle.py) and against
oracle builds with planted mistakes (tests/test_oracle_mutants.py), which must
each fail at least one pin.

Sources of truth used here:
* the hand-worked example in golden/uservisits_example.txt (Section 3.1 query);
* the nested-loop brute force and an independent numpy mask-per-key grouping;
* special cases with closed forms: scalar aggregation as the one-group case
  (Section 3.1), the all-unique dataset (100% cardinality, Section 6.1), the
  heavy-hitter and sorted-uniform datasets (Section 6.4), the empty input;
* invariants: sum of COUNT = N, sum of SUM = sum of values (mod 2^64), number
  of groups = number of distinct keys, global MIN/MAX;
* result invariance when the memory budget forces sorted runs (Section 4.2).
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "uservisits_example.txt")
I64_MIN = np.iinfo(np.int64).min
I64_MAX = np.iinfo(np.int64).max


def read_golden(path=GOLDEN):
    rows, groups, cur = [], [], None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line in ("[rows]", "[groups]"):
                cur = rows if line == "[rows]" else groups
                continue
            cur.append([int(t) for t in line.split()])
    keys = np.array([r[0] for r in rows], np.int64)
    vals = np.array([r[1] for r in rows], np.int64)
    exp = dict(keys=np.array([g[0] for g in groups], np.int64),
               count=np.array([g[1] for g in groups], np.uint64),
               sum=np.array([g[2] for g in groups], np.int64),
               min=np.array([g[3] for g in groups], np.int64),
               max=np.array([g[4] for g in groups], np.int64))
    return keys, vals, exp


def numpy_groups(keys, vals):
    """Independent grouping: one boolean mask per distinct key (small inputs)."""
    keys = np.asarray(keys, np.int64)
    vals = np.asarray(vals).astype(np.int64)
    uk = np.unique(keys)
    out = dict(keys=uk, count=np.zeros(len(uk), np.uint64), sum=np.zeros(len(uk), np.int64),
               min=np.zeros(len(uk), np.int64), max=np.zeros(len(uk), np.int64))
    for i, k in enumerate(uk):
        v = vals[keys == k]
        out["count"][i] = v.size
        out["sum"][i] = v.view(np.uint64).sum(dtype=np.uint64).view(np.int64)
        out["min"][i] = v.min()
        out["max"][i] = v.max()
    return out


def assert_same(got, exp, what=""):
    for f in ("keys", "count", "sum", "min", "max"):
        g, e = np.asarray(got[f]), np.asarray(exp[f])
        assert g.shape == e.shape, f"{what}: {f} has {g.shape} groups, expected {e.shape}"
        assert np.array_equal(g.astype(e.dtype), e), f"{what}: field {f} differs"


def edge_keys(rng, n, pool_size):
    special = np.array([I64_MIN, I64_MIN + 1, -1, 0, 1, I64_MAX, I64_MAX - 1], np.int64)
    pool = np.concatenate([special, rng.integers(I64_MIN, I64_MAX, pool_size, dtype=np.int64, endpoint=True)])
    return pool[rng.integers(0, pool.size, n)]


def big_values(rng, n):
    return rng.integers(I64_MIN, I64_MAX, n, dtype=np.int64, endpoint=True)


# ---------------------------------------------------------------- pins

def pin_golden_example(o):
    keys, vals, exp = read_golden()
    got, _ = o.groupby(keys, vals)
    assert_same(got, exp, "golden, unbounded budget")
    got, runs = o.groupby(keys, vals, budget_bytes=2 * 64)
    assert runs > 1
    assert_same(got, exp, "golden, two-group budget")
    assert_same(o.groupby_bruteforce(keys, vals), exp, "golden, brute force")


def pin_bruteforce_random(o):
    for seed in range(6):
        rng = np.random.default_rng(seed)
        n = [1, 31, 32, 33, 700, 2000][seed]
        keys = edge_keys(rng, n, pool_size=max(1, n // 4))
        vals = big_values(rng, n) if seed % 2 else rng.integers(-1000, 1000, n)
        bf = o.groupby_bruteforce(keys, vals)
        npg = numpy_groups(keys, vals)
        assert_same(bf, npg, f"brute force vs numpy, seed {seed}")
        got, _ = o.groupby(keys, vals)
        assert_same(got, npg, f"groupby vs numpy, seed {seed}")


def pin_spill_invariance(o):
    rng = np.random.default_rng(11)
    n = 5000
    keys = edge_keys(rng, n, pool_size=600)
    vals = big_values(rng, n)
    full, runs_full = o.groupby(keys, vals)
    assert runs_full <= 1
    for groups_in_budget in (1, 3, 50, 599):
        got, runs = o.groupby(keys, vals, budget_bytes=groups_in_budget * 64)
        assert runs > 1, "a tight budget must produce several sorted runs"
        assert_same(got, full, f"budget of {groups_in_budget} groups")


def pin_scalar(o):
    rng = np.random.default_rng(5)
    vals = big_values(rng, 1000)
    keys = np.full(1000, -77, np.int64)
    got, _ = o.groupby(keys, vals, budget_bytes=64)
    assert got["keys"].tolist() == [-77]
    assert int(got["count"][0]) == 1000
    assert got["sum"][0] == vals.view(np.uint64).sum(dtype=np.uint64).view(np.int64)
    assert got["min"][0] == vals.min() and got["max"][0] == vals.max()


def pin_all_unique(o):
    rng = np.random.default_rng(6)
    keys = np.unique(rng.integers(I64_MIN, I64_MAX, 3000, dtype=np.int64))
    rng.shuffle(keys)
    vals = rng.integers(1, 1 << 40, keys.size)
    got, _ = o.groupby(keys, vals, budget_bytes=100 * 64)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(got["keys"], keys[order])
    assert np.all(got["count"] == 1)
    for f in ("sum", "min", "max"):
        assert np.array_equal(got[f], vals[order])


def pin_heavy_hitter(o):
    # Scaled-down heavy-hitter dataset (Section 6.4): one key carries
    # n - (D - 1) rows, every other key of the D-key domain occurs once.
    rng = np.random.default_rng(7)
    d, n = 500, 20000
    domain = np.unique(rng.integers(I64_MIN, I64_MAX, d + 10, dtype=np.int64))[:d]
    keys = np.concatenate([np.full(n - (d - 1), domain[0]), domain[1:]])
    rng.shuffle(keys)
    vals = rng.integers(0, 1 << 20, n)
    got, _ = o.groupby(keys, vals, budget_bytes=40 * 64)
    assert got["keys"].size == d
    hh = np.searchsorted(got["keys"], domain[0])
    assert int(got["count"][hh]) == n - (d - 1)
    assert int(got["sum"][hh]) == int(vals[keys == domain[0]].sum())
    others = np.ones(d, bool)
    others[hh] = False
    assert np.all(got["count"][others] == 1)


def pin_sorted_input(o):
    rng = np.random.default_rng(8)
    keys = edge_keys(rng, 4000, pool_size=300)
    vals = big_values(rng, 4000)
    order = np.argsort(keys, kind="stable")
    a, _ = o.groupby(keys, vals, budget_bytes=20 * 64)
    b, _ = o.groupby(keys[order], vals[order], budget_bytes=20 * 64)
    assert_same(a, b, "sorted vs shuffled input")
    assert_same(b, numpy_groups(keys, vals), "sorted input vs numpy")


def pin_empty(o):
    got, runs = o.groupby(np.zeros(0, np.int64), np.zeros(0, np.int64))
    assert got["keys"].size == 0 and runs == 0
    assert o.groupby_bruteforce(np.zeros(0, np.int64), np.zeros(0, np.int64))["keys"].size == 0


def pin_invariants(o):
    rng = np.random.default_rng(9)
    n = 20000
    keys = edge_keys(rng, n, pool_size=3000)
    vals = big_values(rng, n)
    got, _ = o.groupby(keys, vals, budget_bytes=500 * 64)
    assert int(got["count"].sum(dtype=np.uint64)) == n
    assert got["sum"].view(np.uint64).sum(dtype=np.uint64) == vals.view(np.uint64).sum(dtype=np.uint64)
    assert got["keys"].size == np.unique(keys).size == o.count_distinct(keys)
    assert got["min"].min() == vals.min() and got["max"].max() == vals.max()
    assert np.all(got["min"] <= got["max"])


def pin_signed_order(o):
    keys = np.array([5, -3, I64_MAX, I64_MIN, -3, 0, -1], np.int64)
    got, _ = o.groupby(keys, np.arange(7))
    assert got["keys"].tolist() == [I64_MIN, -3, -1, 0, 5, I64_MAX]
    assert np.all(np.diff(got["keys"]) > 0)


def pin_groups_of(o):
    rng = np.random.default_rng(10)
    keys = edge_keys(rng, 3000, pool_size=200)
    vals = big_values(rng, 3000)
    ref = numpy_groups(keys, vals)
    pick = rng.choice(ref["keys"].size, 25, replace=False)
    sample = np.concatenate([ref["keys"][pick], ref["keys"][pick[:3]]])  # repeats allowed
    got = o.groups_of(keys, vals, sample)
    idx = np.searchsorted(ref["keys"], sample)
    for f in ("count", "sum", "min", "max"):
        assert np.array_equal(got[f].astype(ref[f].dtype), ref[f][idx]), f
    # a key that does not occur yields the identity state
    absent = np.setdiff1d(np.array([12345, 67890], np.int64), keys)
    g = o.groups_of(keys, vals, absent)
    assert np.all(g["count"] == 0) and np.all(g["sum"] == 0)
    assert np.all(g["min"] == I64_MAX) and np.all(g["max"] == I64_MIN)


ALL_PINS = [pin_golden_example, pin_bruteforce_random, pin_spill_invariance, pin_scalar, pin_all_unique,
            pin_heavy_hitter, pin_sorted_input, pin_empty, pin_invariants, pin_signed_order, pin_groups_of]
