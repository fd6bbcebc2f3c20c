"""The host staging tier: spill staging in pinned host memory that the kernel
reaches over the host link (the paper's disk, outside the memory budget), as a
true tier below device memory.  Results must equal the oracle's and the
device-tier run's, at every level of recursion and through the sort fallback."""
import numpy as np
import pytest

from _gpu import assert_parity, canon, gpu_groupby, oracle_expected, to_dev

pytestmark = pytest.mark.gpu
MB = 1 << 20


def _tuning(**kw):
    from paper_1311_0059_gb300 import agg_tuning
    return agg_tuning(**kw)


@pytest.mark.parametrize("extra", [dict(), dict(fan_out=16), dict(max_levels=1)])
def test_spilling_with_staging_in_host_memory(oracle, extra):
    rng = np.random.default_rng(17)
    keys = rng.integers(0, 900_000, 2_000_000).astype(np.int64) * 1_000_003
    vals = rng.integers(-2**40, 2**40, keys.size)
    exp = oracle_expected(oracle, keys, vals)
    got, st = gpu_groupby(keys, vals, budget=MB, tuning=_tuning(staging_tier=2, **extra))
    assert_parity(got, exp, what=f"host staging {extra}")
    assert st["staging_in_host"] == 1 and st["levels"] >= 2
    dev, st_d = gpu_groupby(keys, vals, budget=MB, tuning=_tuning(staging_tier=1, **extra))
    assert st_d["staging_in_host"] == 0
    assert_parity(dev, got, what="device tier against host tier")


def test_switching_tiers_on_one_handle(oracle):
    from paper_1311_0059_gb300.groupby import GroupBy
    rng = np.random.default_rng(18)
    keys = rng.integers(0, 500_000, 1_200_000).astype(np.int64)
    vals = rng.integers(0, 1 << 20, keys.size)
    exp = oracle_expected(oracle, keys, vals)
    with GroupBy(MB) as g:
        for tier, where in ((1, 0), (2, 1), (1, 0), (0, 0)):
            g.set_tuning(_tuning(staging_tier=tier))
            res = canon({k: t.cpu().numpy() for k, t in g.run(to_dev(keys), to_dev(vals)).items()})
            assert_parity(res, exp, what=f"tier {tier}")
            assert g.stats()["staging_in_host"] == where
