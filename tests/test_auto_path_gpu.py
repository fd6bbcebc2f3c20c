"""AGG_PATH_AUTO: each run takes the path the cost model predicts to be faster
(the sort path for nearly unique keys that spill, the hash path otherwise),
in the same working memory.  Every run is compared with the oracle, on a
handle and in the served form, where an AUTO server mixes both paths."""
import time

import numpy as np
import pytest

import datagen as dg
from _gpu import assert_parity, canon, oracle_expected, to_dev

pytestmark = pytest.mark.gpu
MB = 1 << 20
I64_MIN = np.iinfo(np.int64).min
I64_MAX = np.iinfo(np.int64).max


def _unique(seed, n):
    rng = np.random.default_rng(seed)
    k = np.unique(rng.integers(I64_MIN, I64_MAX, n + n // 50, dtype=np.int64))[:n]
    rng.shuffle(k)
    return k, rng.integers(-2**40, 2**40, k.size)


def test_auto_handle_switches_paths_in_one_memory(oracle):
    from paper_1311_0059_gb300 import AGG_PATH_AUTO, AGG_PATH_HASH, AGG_PATH_SORT
    from paper_1311_0059_gb300.groupby import GroupBy
    big = _unique(1, 3_000_000)
    small = _unique(2, 100_000)
    rng = np.random.default_rng(3)
    dup = (rng.integers(0, 80_000, 3_000_000).astype(np.int64) * 17, rng.integers(0, 1 << 20, 3_000_000))
    with GroupBy(128 * MB, path=AGG_PATH_AUTO, expected_groups=3_000_000) as g:
        for (keys, vals), want in ((big, AGG_PATH_SORT), (small, AGG_PATH_HASH), (dup, AGG_PATH_SORT),
                                   (small, AGG_PATH_HASH), (big, AGG_PATH_SORT)):
            res = canon({k: t.cpu().numpy() for k, t in g.run(to_dev(keys), to_dev(vals)).items()})
            assert_parity(res, oracle_expected(oracle, keys, vals), what=f"{keys.size} rows")
            assert g.stats()["path"] == want
    with GroupBy(128 * MB, path=AGG_PATH_AUTO, expected_groups=80_000) as g:  # low cardinality: hash
        res = canon({k: t.cpu().numpy() for k, t in g.run(to_dev(dup[0]), to_dev(dup[1])).items()})
        assert_parity(res, oracle_expected(oracle, *dup), what="low cardinality")
        assert g.stats()["path"] == AGG_PATH_HASH


def test_auto_server_mixes_both_paths(oracle):
    from paper_1311_0059_gb300 import AGG_I64, AGG_PATH_AUTO, AGG_PATH_HASH, AGG_PATH_SORT, _abi
    from paper_1311_0059_gb300.groupby import Output, Server
    srv = Server(2 << 30, max_active=8, ops=15, value_type=AGG_I64, path=AGG_PATH_AUTO)
    cases = []
    for i in range(8):
        if i % 2 == 0:
            keys, vals = _unique(10 + i, 3_000_000)
            cases.append((keys, vals, 128 * MB, keys.size))                 # nearly unique: sort
        else:
            w = dg.Workload(f"q{i}", n=1_500_000 if i % 4 == 1 else 60_000, domain=40_000, seed=i, budget=64 * MB)
            keys, vals = w.host()
            cases.append((keys, vals, w.budget, 40_000))                     # low cardinality: hash
    outs, ts = [], []
    for keys, vals, budget, hint in cases:
        o = Output(keys.size, 15, "cuda")
        ts.append(srv.submit(to_dev(keys), to_dev(vals), budget, o, expected_groups=hint))
        outs.append(o)
    deadline = time.perf_counter() + 120
    while srv.stats()["completed"] < len(cases) and time.perf_counter() < deadline:
        srv.progress()
    paths = set()
    for (keys, vals, _, _), o, t in zip(cases, outs, ts):
        info = srv.poll(t)
        assert info.state == _abi.AGG_QUERY_DONE and info.status == 0
        got = canon({f: x.cpu().numpy() for f, x in o.result(info.n_groups).items()})
        assert_parity(got, oracle_expected(oracle, keys, vals), what=f"ticket {t}, path {info.path}")
        paths.add(info.path)
    assert paths == {AGG_PATH_HASH, AGG_PATH_SORT}
    srv.close()
