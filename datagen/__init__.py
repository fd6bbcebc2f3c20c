"""Seeded synthetic (key, value) inputs for the budgeted group-by.

This module only draws inputs; it holds none of the group-by arithmetic.  Both
the CPU oracle (through the numpy functions here) and the GPU path (through the
device kernels in ``csrc/datagen.cu``) consume the same bytes: every element is
a pure function of (seed, stream, index), so the host and device implementations
produce identical arrays, which a GPU test checks element by element.

Definitions
-----------
* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): the state advances by the odd constant GAMMA and
  each output is ``mix(state)`` with the 64-bit finaliser below.  Element ``i``
  of stream ``sid`` under ``seed`` is ``mix(base + (i + 1) * GAMMA)`` with
  ``base = mix(seed ^ ((sid + 1) * GAMMA))`` (arithmetic mod 2**64), i.e. the
  (i+1)-th output of a SplitMix64 generator started at state ``base``.
* Key domain: rank ``r`` (0-based) maps to key ``mix(r ^ salt)`` with
  ``salt = element 0 of stream 2``.  ``mix`` is a bijection of 64-bit words, so
  distinct ranks give distinct, random-looking int64 keys.
* Uniform rank in ``[0, D)``: ``floor(u * D / 2**64)`` (multiply-high) of a
  stream-0 draw ``u``; ``D < 2**32``.
* Zipf(s) rank over ``D`` ranks (the skewed workloads of the paper's skew study,
  Section 6.4, generated after Gray et al.): P(rank r) proportional to
  ``(r+1)**-s``.  A float64 CDF table (``zipf_cdf``) is built once on the host;
  a draw ``u`` becomes ``t = (u >> 11) * 2**-53`` and the rank is the first
  index whose CDF entry exceeds ``t`` (the last entry is forced to 2.0).  The
  device kernel searches the same table bytes, so both sides agree exactly.
* Values (stream 1): ``int32`` uniform in ``[0, 1000)`` as multiply-high by
  1000; ``int64`` uniform in ``[0, 2**20)`` as ``u >> 44``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB

STREAM_KEY = 0
STREAM_VAL = 1
STREAM_SALT = 2
STREAM_INSTANCE = 3
STREAM_PARAMS = 4

_U64 = np.uint64


def mix_int(z: int) -> int:
    """SplitMix64 finaliser on one Python int (mod 2**64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser, elementwise on a uint64 array (wraps mod 2**64)."""
    z = np.asarray(z, dtype=_U64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U64(30))) * _U64(M1)
        z = (z ^ (z >> _U64(27))) * _U64(M2)
        return z ^ (z >> _U64(31))


def stream_base(seed: int, sid: int) -> int:
    return mix_int((seed & MASK64) ^ (((sid + 1) * GAMMA) & MASK64))


def stream(seed: int, sid: int, start: int, count: int) -> np.ndarray:
    """Elements [start, start+count) of stream ``sid`` as uint64."""
    base = _U64(stream_base(seed, sid))
    idx = np.arange(start + 1, start + count + 1, dtype=_U64)
    with np.errstate(over="ignore"):
        return mix(base + idx * _U64(GAMMA))


def key_salt(seed: int) -> int:
    return mix_int(stream_base(seed, STREAM_SALT) + GAMMA)


def key_of_rank(seed: int, ranks: np.ndarray) -> np.ndarray:
    """Bijective rank -> int64 key map of the key domain."""
    r = np.asarray(ranks, dtype=_U64)
    return mix(r ^ _U64(key_salt(seed))).view(np.int64)


def _unxorshift(y: np.ndarray, s: int) -> np.ndarray:
    x = y.copy()
    t = y >> _U64(s)
    while np.any(t):
        x ^= t
        t = t >> _U64(s)
    return x


def unmix(z: np.ndarray) -> np.ndarray:
    """Inverse of ``mix`` (each xorshift and odd multiply is invertible mod 2**64)."""
    z = np.asarray(z, dtype=_U64)
    inv1 = _U64(pow(M1, -1, 1 << 64))
    inv2 = _U64(pow(M2, -1, 1 << 64))
    with np.errstate(over="ignore"):
        z = _unxorshift(z, 31) * inv2
        z = _unxorshift(z, 27) * inv1
        return _unxorshift(z, 30)


def rank_of_key(seed: int, keys: np.ndarray) -> np.ndarray:
    """Inverse of ``key_of_rank``: the domain rank of each key (uint64)."""
    k = np.asarray(keys, dtype=np.int64).view(_U64)
    return unmix(k) ^ _U64(key_salt(seed))


def mulhi_u32(u: np.ndarray, d: int) -> np.ndarray:
    """floor(u * d / 2**64) for uint64 ``u`` and 0 < d < 2**32, exactly."""
    assert 0 < d < (1 << 32)
    u = np.asarray(u, dtype=_U64)
    dd = _U64(d)
    with np.errstate(over="ignore"):
        hi = (u >> _U64(32)) * dd
        lo = ((u & _U64(0xFFFFFFFF)) * dd) >> _U64(32)
        return (hi + lo) >> _U64(32)


def uniform_ranks(seed: int, domain: int, start: int, count: int) -> np.ndarray:
    return mulhi_u32(stream(seed, STREAM_KEY, start, count), domain)


_HARMONIC = np.zeros(0)


def harmonic(n: int) -> np.ndarray:
    """Partial sums H[r-1] = 1 + 1/2 + ... + 1/r for r = 1..n, float64, summed in
    order; one growing master table, so every prefix has the same bytes."""
    global _HARMONIC
    if _HARMONIC.size < n:
        size = max(n, 2 * _HARMONIC.size)
        _HARMONIC = np.cumsum(1.0 / np.arange(1, size + 1, dtype=np.float64))
    return _HARMONIC[:n]


def zipf_cdf(domain: int, s: float) -> np.ndarray:
    """Float64 CDF table of Zipf(s) over ``domain`` ranks; last entry 2.0.
    For s = 1 the table is the harmonic prefix divided by its last entry."""
    if float(s) == 1.0:
        h = harmonic(domain)
        cdf = h / h[-1]
    else:
        w = np.arange(1, domain + 1, dtype=np.float64) ** (-float(s))
        cdf = np.cumsum(w)
        cdf /= cdf[-1]
    cdf[-1] = 2.0
    return cdf


def zipf_ranks(seed: int, cdf: np.ndarray, start: int, count: int) -> np.ndarray:
    u = stream(seed, STREAM_KEY, start, count)
    t = (u >> _U64(11)).astype(np.float64) * (2.0 ** -53)
    return np.searchsorted(cdf, t, side="right").astype(_U64)


def values(seed: int, vtype: str, start: int, count: int) -> np.ndarray:
    u = stream(seed, STREAM_VAL, start, count)
    if vtype == "i32_1000":
        return mulhi_u32(u, 1000).astype(np.int32)
    if vtype == "i64_2p20":
        return (u >> _U64(44)).astype(np.int64)
    raise ValueError(f"unknown value type {vtype!r}")


def instance_seed(seed: int, i: int) -> int:
    """Seed of instance/query ``i`` under a workload seed (SplitMix64 output i)."""
    return mix_int(stream_base(seed, STREAM_INSTANCE) + (i + 1) * GAMMA)


@dataclass
class Workload:
    """One synthetic group-by input: ``n`` rows over a ``domain``-key space."""
    name: str
    n: int
    domain: int
    dist: str = "uniform"          # "uniform" | "zipf"
    zipf_s: float = 1.0
    vtype: str = "i64_2p20"        # "i32_1000" | "i64_2p20"
    seed: int = 0
    budget: int = 64 << 20
    ops: int = 15                  # COUNT|SUM|MIN|MAX bitmask
    _cdf: np.ndarray | None = field(default=None, repr=False)

    @property
    def value_dtype(self):
        return np.int32 if self.vtype == "i32_1000" else np.int64

    def cdf(self) -> np.ndarray:
        if self._cdf is None:
            self._cdf = zipf_cdf(self.domain, self.zipf_s)
        return self._cdf

    def ranks(self, start: int = 0, count: int | None = None) -> np.ndarray:
        count = self.n - start if count is None else count
        if self.dist == "uniform":
            return uniform_ranks(self.seed, self.domain, start, count)
        if self.dist == "zipf":
            return zipf_ranks(self.seed, self.cdf(), start, count)
        raise ValueError(self.dist)

    def host(self, start: int = 0, count: int | None = None):
        """(keys int64, vals int32|int64) rows [start, start+count) on the host."""
        count = self.n - start if count is None else count
        keys = key_of_rank(self.seed, self.ranks(start, count))
        vals = values(self.seed, self.vtype, start, count)
        return keys, vals

    def device(self, keys_ptr: int, vals_ptr: int, start: int = 0, count: int | None = None,
               cdf_ptr: int = 0, stream_handle: int = 0) -> None:
        """Write the same rows into device buffers with the CUDA generator."""
        count = self.n - start if count is None else count
        lib = _device_lib()
        dist = 0 if self.dist == "uniform" else 1
        vt = 0 if self.vtype == "i32_1000" else 1
        if dist == 1 and not cdf_ptr:
            raise ValueError("zipf generation on the device needs the CDF table on the device")
        rc = lib.datagen_rows(ctypes.c_uint64(self.seed), ctypes.c_uint64(self.domain), ctypes.c_int(dist),
                              ctypes.c_void_p(cdf_ptr), ctypes.c_int(vt), ctypes.c_uint64(start),
                              ctypes.c_uint64(count), ctypes.c_void_p(keys_ptr), ctypes.c_void_p(vals_ptr),
                              ctypes.c_void_p(stream_handle))
        if rc != 0:
            raise RuntimeError(f"datagen_rows failed with CUDA error {rc}")


# The workloads of the benchmark configurations, named by what they are.
PLAIN_1M_10K = Workload("plain in-budget: 1M rows, 10k keys, int32 values, 64 MB",
                        n=1_000_000, domain=10_000, vtype="i32_1000", budget=64 << 20, ops=15)
SPILL_200M_50M = Workload("spilling: 200M rows, 50M-key uniform domain, 256 MB",
                          n=200_000_000, domain=50_000_000, vtype="i64_2p20", budget=256 << 20, ops=15)
ZIPF_500M_10M = Workload("skewed: 500M rows, Zipf(1.0) over 10M keys, 1 GB",
                         n=500_000_000, domain=10_000_000, dist="zipf", zipf_s=1.0, vtype="i64_2p20",
                         budget=1 << 30, ops=3)

_LIB = None
_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdatagen.so")


def _device_lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run datagen/build.py")
        lib = ctypes.CDLL(LIB_PATH)
        lib.datagen_rows.restype = ctypes.c_int
        lib.datagen_rows.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
        _LIB = lib
    return _LIB


def unit_doubles(seed: int, sid: int, count: int) -> np.ndarray:
    """count doubles in [0, 1) from stream ``sid``: (u >> 11) * 2**-53."""
    return (stream(seed, sid, 0, count) >> _U64(11)).astype(np.float64) * (2.0 ** -53)


def batch_workloads(count: int = 4096, seed: int = 0, rows=(1_000, 4_000_000), card=(0.01, 0.50),
                    budget=(4 << 20, 64 << 20), zipf_s=(0.5, 1.2)) -> list:
    """The batched workload: `count` independent group-by instances.  Per
    instance (five draws of stream 4 under `seed`): rows log-uniform in `rows`,
    distinct keys a uniform fraction `card` of the rows, uniform or Zipf keys
    (probability 1/2 each) with Zipf exponent uniform in `zipf_s`, int64 values
    in [0, 2**20), COUNT+SUM+MIN+MAX, budget log-uniform in `budget`."""
    u = unit_doubles(seed, STREAM_PARAMS, 5 * count).reshape(count, 5)
    out = []
    for i in range(count):
        n = int(np.exp(np.log(rows[0]) + u[i, 0] * (np.log(rows[1]) - np.log(rows[0]))))
        frac = card[0] + u[i, 1] * (card[1] - card[0])
        dom = max(1, int(round(frac * n)))
        zipf = u[i, 2] < 0.5
        s = zipf_s[0] + u[i, 3] * (zipf_s[1] - zipf_s[0])
        b = int(np.exp(np.log(budget[0]) + u[i, 4] * (np.log(budget[1]) - np.log(budget[0]))))
        out.append(Workload(f"batch instance {i}", n=n, domain=dom, dist="zipf" if zipf else "uniform",
                            zipf_s=float(s), vtype="i64_2p20", seed=instance_seed(seed, i), budget=b, ops=15))
    return out


STREAM_ARRIVALS = 5


def served_workloads(duration: float = 60.0, rate: float = 200.0, seed: int = 0, rows=(10_000, 100_000_000),
                     card=(0.001, 0.50), budget=(16 << 20, 2 << 30)):
    """The served workload: queries arriving as a Poisson process of `rate` per
    second over `duration` seconds (exponential gaps from stream 5).  Per query
    (five draws of stream 4): rows log-uniform in `rows`, distinct keys a
    uniform fraction `card` of the rows, uniform or Zipf(1.0) keys (1/2 each),
    int64 values in [0, 2**20), budget log-uniform in `budget`.
    Returns [(arrival_seconds, Workload)]."""
    expect = int(duration * rate * 1.5) + 64
    gaps = -np.log1p(-unit_doubles(seed, STREAM_ARRIVALS, expect)) / rate
    t = np.cumsum(gaps)
    count = int(np.searchsorted(t, duration))
    u = unit_doubles(seed + 1, STREAM_PARAMS, 5 * max(count, 1)).reshape(-1, 5)
    out = []
    for i in range(count):
        n = int(np.exp(np.log(rows[0]) + u[i, 0] * (np.log(rows[1]) - np.log(rows[0]))))
        frac = card[0] + u[i, 1] * (card[1] - card[0])
        dom = max(1, int(round(frac * n)))
        zipf = u[i, 2] < 0.5
        b = int(np.exp(np.log(budget[0]) + u[i, 4] * (np.log(budget[1]) - np.log(budget[0]))))
        out.append((float(t[i]), Workload(f"query {i}", n=n, domain=dom, dist="zipf" if zipf else "uniform",
                                          zipf_s=1.0, vtype="i64_2p20", seed=instance_seed(seed + 1, i), budget=b,
                                          ops=15)))
    return out
