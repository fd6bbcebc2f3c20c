"""Failure detection without a GPU fault: a bounded device-side wait that runs
out must end the run with AGG_ERR_TIMEOUT, and the handle must work again.

Every grid barrier of the hash kernel waits with a limit (agg_tuning
.wait_limit_us; 4 s by default).  The input would fit the table at once, so
the in-budget paths (which have no grid barrier) are turned off to run it
through the spilling kernel.  A limit of 1 us makes the waits run out: on an
input of a few tiles most blocks draw no tile and reach the first grid barrier
microseconds before the busy blocks arrive, and one arrival of 304 blocks at a
barrier already takes about that long.  Nothing hangs and nothing faults: each
block that gives up records the status and returns, and a block released by a
barrier that others left only works on data completed before that barrier, so
every access stays in bounds.
"""
import numpy as np
import pytest

from _gpu import assert_parity, canon, oracle_expected, to_dev

pytestmark = pytest.mark.gpu

MB = 1 << 20


def test_bounded_wait_runs_out_and_the_handle_recovers(oracle):
    from paper_1311_0059_gb300 import _abi, agg_tuning
    from paper_1311_0059_gb300.groupby import GroupBy
    rng = np.random.default_rng(41)
    keys = rng.integers(-2**63, 2**63 - 1, 1000, dtype=np.int64)[rng.integers(0, 1000, 4096)]
    vals = rng.integers(-2**40, 2**40, keys.size, dtype=np.int64)
    exp = oracle_expected(oracle, keys, vals)
    dk, dv = to_dev(keys), to_dev(vals)
    with GroupBy(4 * MB, tuning=agg_tuning(wait_limit_us=1, in_budget=2)) as g:
        timed_out = False
        for _ in range(5):
            try:
                got = canon({k: t.cpu().numpy() for k, t in g.run(dk, dv).items()})
            except _abi.AggError as err:
                assert err.status == _abi.AGG_ERR_TIMEOUT, err
                timed_out = True
                break
            # a run whose waits all ended in time is a correct run
            assert_parity(got, exp, what="a run within the 1 us limit")
        assert timed_out, "no wait ran out with a limit of 1 us"
        g.set_tuning(agg_tuning(in_budget=2))  # the default limit again
        for _ in range(2):
            got = canon({k: t.cpu().numpy() for k, t in g.run(dk, dv).items()})
            assert_parity(got, exp, what="after the timed-out run")
