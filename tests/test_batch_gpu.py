"""The batched form: many independent group-bys in one persistent launch.
Every instance's result must equal its own single-query result and the
oracle's, bit for bit, whatever the team shape and whether the launch is
replayed from a CUDA graph."""
import numpy as np
import pytest

import datagen as dg
from _gpu import assert_parity, canon, oracle_expected, to_dev

pytestmark = pytest.mark.gpu
MB = 1 << 20


def small_batch(count=40, seed=3):
    ws = dg.batch_workloads(count, seed=seed, rows=(1_000, 150_000), card=(0.01, 0.5), budget=(1 * MB, 3 * MB))
    data = []
    for w in ws:
        k, v = w.host()
        data.append((k, v, w.budget))
    return data


def _run_batch(data, tuning=None, reps=1):
    from paper_1311_0059_gb300 import AGG_I64
    from paper_1311_0059_gb300.groupby import Batch
    dev = [(to_dev(k), to_dev(v), b, 0) for k, v, b in data]
    bt = Batch(dev, ops=15, value_type=AGG_I64, tuning=tuning)
    res = None
    for _ in range(reps):
        res = bt.run()
    out = [canon({f: t.cpu().numpy() for f, t in r.items()}) for r in res]
    bt.close()
    return out


@pytest.mark.parametrize("team", [1, 2, 4])
def test_batch_matches_oracle(oracle, team):
    from paper_1311_0059_gb300 import _abi
    data = small_batch()
    got = _run_batch(data, tuning=_abi.agg_batch_tuning(team_blocks=team))
    for i, (k, v, b) in enumerate(data):
        assert_parity(got[i], oracle_expected(oracle, k, v), what=f"instance {i} (team {team})")


def test_batch_spills_and_replays_from_graph(oracle):
    # budgets at the minimum force most instances of this batch to spill and recurse
    from paper_1311_0059_gb300 import _abi
    ws = dg.batch_workloads(24, seed=9, rows=(100_000, 400_000), card=(0.3, 0.5), budget=(MB, MB))
    data = [(*w.host(), w.budget) for w in ws]
    for use_graph in (0, 2):
        got = _run_batch(data, tuning=_abi.agg_batch_tuning(team_blocks=2, use_graph=use_graph), reps=3)
        for i, (k, v, b) in enumerate(data):
            assert_parity(got[i], oracle_expected(oracle, k, v), what=f"spilling instance {i}")


def test_batch_equals_single_query_results():
    from paper_1311_0059_gb300.groupby import GroupBy
    data = small_batch(count=16, seed=5)
    got = _run_batch(data)
    for i, (k, v, b) in enumerate(data):
        with GroupBy(b) as g:
            ref = canon({f: t.cpu().numpy() for f, t in g.run(to_dev(k), to_dev(v)).items()})
        assert_parity(got[i], ref, what=f"instance {i} alone vs in the batch")


def test_batch_workload_generator_is_deterministic():
    a = dg.batch_workloads(64, seed=0)
    b = dg.batch_workloads(64, seed=0)
    assert [(w.n, w.domain, w.dist, w.budget, w.seed) for w in a] == [(w.n, w.domain, w.dist, w.budget, w.seed)
                                                                      for w in b]
    ns = np.array([w.n for w in dg.batch_workloads(4096)])
    assert ns.min() >= 1000 and ns.max() <= 4_000_000


def test_batch_rejects_pointers_the_kernel_cannot_use():
    # an instance with host keys, host values or no values (SUM needs them)
    # makes agg_batch_create fail with an argument error, before any launch
    import torch
    from paper_1311_0059_gb300 import AGG_I64, _abi
    from paper_1311_0059_gb300.groupby import Batch
    k = torch.arange(1000, dtype=torch.int64, device="cuda")
    v = torch.ones(1000, dtype=torch.int64, device="cuda")
    for bad in ((k.cpu(), v, 4 * MB, 0), (k, v.cpu(), 4 * MB, 0), (k, None, 4 * MB, 0)):
        with pytest.raises(_abi.AggError) as e:
            Batch([(k, v, 4 * MB, 0), bad], ops=15, value_type=AGG_I64)
        assert e.value.status == _abi.AGG_ERR_INVALID_ARG
