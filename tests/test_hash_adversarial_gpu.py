"""Adversarial key sets for the hash path's per-slot policies, checked against
the CPU oracle element by element.

The hash path places a key by h = fmix64(key ^ seed_0), with the MurmurHash3
64-bit finaliser and seed_0 = fmix64(seed + c).  That finaliser is a bijection,
so these tests build keys with chosen hash bits by inverting it:
* many hot keys that share one set of the 4-way level-0 cache (hash bits 16..24
  equal), so that most of them cannot be cached and must go to the global table;
* hundreds of keys in one 32-slot bucket of the global table (hash bits 32..63
  nearly equal), so that all but 32 of them spill although the table is almost
  empty, and inserts race for the bucket's slots;
* a tiny level-0 table (a small expected_groups hint) with many concurrent
  inserts per bucket.
The inverse is used only to construct inputs; expected values come from the
oracle.
"""
import numpy as np
import pytest

from _gpu import assert_parity, gpu_groupby, oracle_expected

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1
C1, C2 = 0xFF51AFD7ED558CCD, 0xC4CEB9FE1A85EC53
LEVEL_C = 0xD6E8FEB86659FD93
MB = 1 << 20


def fmix64(k: int) -> int:
    k &= M64
    k ^= k >> 33
    k = (k * C1) & M64
    k ^= k >> 33
    k = (k * C2) & M64
    return k ^ (k >> 33)


def fmix64_inv(h: int) -> int:
    # x ^ (x >> 33) is its own inverse on 64 bits; the multipliers are odd
    h &= M64
    h ^= h >> 33
    h = (h * pow(C2, -1, 1 << 64)) & M64
    h ^= h >> 33
    h = (h * pow(C1, -1, 1 << 64)) & M64
    return h ^ (h >> 33)


def key_with_hash(h: int, seed: int = 0) -> int:
    seed0 = fmix64((seed + LEVEL_C) & M64)
    k = fmix64_inv(h) ^ seed0
    return k - (1 << 64) if k >= 1 << 63 else k


def test_inverse_is_exact():
    rng = np.random.default_rng(0)
    for x in rng.integers(0, 2**63, 1000, dtype=np.int64).tolist():
        assert fmix64(fmix64_inv(x)) == x and fmix64_inv(fmix64(x)) == x


def test_hot_keys_sharing_one_cache_set(oracle):
    # 64 hot keys whose hash bits 16..27 are equal (one set of the level-0
    # cache for any cache size), spread over global buckets; only four fit the
    # set, the other hot keys are aggregated in the global table throughout.
    rng = np.random.default_rng(11)
    hot = []
    for i in range(64):
        hi = int(rng.integers(0, 1 << 32))
        lo = (int(rng.integers(0, 1 << 16)) & 0xFFFF) | (0x5A5 << 16)
        hot.append(key_with_hash((hi << 32) | (int(rng.integers(0, 16)) << 28) | lo))
    hot = np.array(hot, np.int64)
    cold = rng.integers(-2**63, 2**63 - 1, 3000, dtype=np.int64)
    n = 600_000
    keys = np.where(rng.random(n) < 0.9, hot[rng.integers(0, hot.size, n)], cold[rng.integers(0, cold.size, n)])
    vals = rng.integers(-2**40, 2**40, n, dtype=np.int64)
    for ops in (15, 3):
        got, _ = gpu_groupby(keys, vals, budget=64 * MB, ops=ops)
        assert_parity(got, oracle_expected(oracle, keys, vals), ops, f"one cache set, ops={ops}")


def test_many_keys_in_one_bucket(oracle):
    # 400 keys with hash bits 32..63 below 2^12: all in bucket 0 of the global
    # table whatever its size.  32 become resident, the rest spill and are
    # aggregated at level 1 (a fresh seed spreads them).
    rng = np.random.default_rng(12)
    keys_set = np.array([key_with_hash((int(rng.integers(0, 1 << 12)) << 32) | int(rng.integers(0, 1 << 32)))
                         for _ in range(400)], np.int64)
    keys_set = np.unique(keys_set)
    n = 300_000
    keys = keys_set[rng.integers(0, keys_set.size, n)]
    vals = rng.integers(0, 1 << 20, n, dtype=np.int64)
    got, st = gpu_groupby(keys, vals, budget=16 * MB)
    assert_parity(got, oracle_expected(oracle, keys, vals), 15, "one bucket")
    assert st["spill_records"][0] > 0, "the keys were meant to overflow one bucket"
    assert st["resident_groups"][0] <= 32


@pytest.mark.parametrize("expected_groups", [1, 1000, 20_000])
def test_tiny_level0_table_under_concurrent_inserts(oracle, expected_groups):
    # A small expected_groups hint sizes the level-0 table to a few thousand
    # slots: every block inserts new keys into the same few buckets at once,
    # and most keys spill.
    rng = np.random.default_rng(13 + expected_groups)
    n = 400_000
    keys = rng.integers(0, 60_000, n).astype(np.int64) * 1_000_003 - 7
    vals = rng.integers(-1000, 1000, n, dtype=np.int64)
    got, st = gpu_groupby(keys, vals, budget=64 * MB, expected_groups=expected_groups)
    assert_parity(got, oracle_expected(oracle, keys, vals), 15, f"expected_groups={expected_groups}")
    assert st["n_groups"] == got["keys"].size
