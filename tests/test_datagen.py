"""The seeded input generator (host side), checked against its published
definitions and the statistics of the distributions it draws."""
import numpy as np

import datagen as dg


def test_splitmix64_published_outputs():
    # SplitMix64 started at state 0 (Steele, Lea & Flood 2014; reference C code
    # by Vigna): the first three outputs are these published constants.
    x, out = 0, []
    for _ in range(3):
        x = (x + dg.GAMMA) & dg.MASK64
        out.append(dg.mix_int(x))
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # the vectorised form and the stream definition agree with it
    assert dg.mix(np.array([dg.GAMMA], np.uint64))[0] == 0xE220A8397B1DCDAF


def test_stream_is_counter_based():
    a = dg.stream(3, 0, 0, 1000)
    b = dg.stream(3, 0, 400, 100)
    assert np.array_equal(a[400:500], b)
    base = dg.stream_base(3, 0)
    assert int(a[7]) == dg.mix_int(base + 8 * dg.GAMMA)
    assert not np.array_equal(dg.stream(3, 1, 0, 1000), a)
    assert not np.array_equal(dg.stream(4, 0, 0, 1000), a)


def test_mulhi_exact():
    rng = np.random.default_rng(0)
    u = rng.integers(0, 1 << 64, 5000, dtype=np.uint64, endpoint=False)
    u[:3] = [0, (1 << 64) - 1, 1 << 63]
    for d in (1, 7, 1000, 10_000, 50_000_000, (1 << 32) - 1):
        got = dg.mulhi_u32(u, d)
        exp = [(int(x) * d) >> 64 for x in u]
        assert got.tolist() == exp


def test_key_map_is_bijective_on_a_domain():
    keys = dg.key_of_rank(0, np.arange(2_000_000, dtype=np.uint64))
    assert np.unique(keys).size == keys.size
    assert keys.dtype == np.int64
    assert (keys < 0).any() and (keys > 0).any()


def test_uniform_ranks_and_values():
    w = dg.Workload("t", n=400_000, domain=1000, vtype="i32_1000")
    r = w.ranks()
    assert r.min() >= 0 and r.max() < 1000
    cnt = np.bincount(r.astype(np.int64), minlength=1000)
    # chi-square against the uniform law (999 dof; mean 999, sd ~44.7)
    chi2 = ((cnt - 400.0) ** 2 / 400.0).sum()
    assert chi2 < 999 + 6 * 44.7
    keys, vals = w.host()
    assert vals.dtype == np.int32 and vals.min() >= 0 and vals.max() < 1000
    assert abs(vals.mean() - 499.5) < 2.0
    v64 = dg.values(0, "i64_2p20", 0, 100_000)
    assert v64.dtype == np.int64 and v64.min() >= 0 and v64.max() < (1 << 20)


def test_zipf_frequencies():
    d, s, n = 1000, 1.0, 400_000
    w = dg.Workload("z", n=n, domain=d, dist="zipf", zipf_s=s)
    r = w.ranks()
    assert r.min() >= 0 and r.max() < d
    h = (np.arange(1, d + 1, dtype=np.float64) ** -s).sum()
    p0 = 1.0 / h
    f0 = (r == 0).mean()
    assert abs(f0 - p0) < 5 * np.sqrt(p0 * (1 - p0) / n)
    p1 = 0.5 / h
    f1 = (r == 1).mean()
    assert abs(f1 - p1) < 5 * np.sqrt(p1 * (1 - p1) / n)
    cdf = dg.zipf_cdf(d, s)
    assert cdf[-1] == 2.0 and np.all(np.diff(cdf) > 0)


def test_instance_seeds_distinct():
    s = [dg.instance_seed(0, i) for i in range(10_000)]
    assert len(set(s)) == len(s)


def test_rank_of_key_inverts_key_of_rank():
    r = np.concatenate([np.arange(1000, dtype=np.uint64), np.array([2**64 - 1, 2**63, 12345678901234], np.uint64)])
    for seed in (0, 7):
        assert np.array_equal(dg.rank_of_key(seed, dg.key_of_rank(seed, r)), r)
