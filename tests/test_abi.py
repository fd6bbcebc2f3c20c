"""The C-ABI library loads and exports every entry point include/agg.h declares
(no GPU needed: only host-side functions are called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions(path):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(agg_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1311_0059_gb300 import _abi
    if not os.path.exists(_abi.LIB_PATH):
        from paper_1311_0059_gb300 import build
        build.build()
    return _abi.load()


def test_header_lists_the_boundary():
    names = header_functions(os.path.join(ROOT, "include", "agg.h"))
    for must in ("agg_create", "agg_run", "agg_destroy", "agg_sync", "agg_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1311_0059_gb300 import _abi
    names = header_functions(os.path.join(ROOT, "include", "agg.h"))
    for n in names:
        assert hasattr(lib, n), f"{n} declared in agg.h but not exported"
        assert n in _abi.SIGNATURES, f"{n} has no Python binding"


def test_strerror(lib):
    from paper_1311_0059_gb300 import _abi
    for s in range(0, 9):
        assert _abi.strerror(s)
    assert _abi.strerror(0) == "ok"


def test_plan_is_host_only_and_follows_the_budget(lib):
    from paper_1311_0059_gb300 import groupby as gb, _abi
    spec = gb.make_spec(ops=15, value_type=_abi.AGG_I64)
    p = gb.plan(256 << 20, 200_000_000, spec)
    assert p["entry_bytes"] == 64
    assert p["working_bytes"] <= 256 << 20
    assert p["table_slots"] * 65 <= 256 << 20
    assert p["fan_out"] == 64            # 200M * 64 B * 1.2 / 256 MiB = 57.2 -> 64
    spec32 = gb.make_spec(ops=15, value_type=_abi.AGG_I32)
    assert gb.plan(64 << 20, 1_000_000, spec32)["entry_bytes"] == 32
    assert gb.plan(1 << 30, 10, gb.make_spec(ops=3))["fan_out"] == 16
    with pytest.raises(_abi.AggError) as e:
        gb.plan(1000, 10, spec)
    assert e.value.status == _abi.AGG_ERR_BUDGET_TOO_SMALL
    bad = gb.make_spec(ops=0)
    with pytest.raises(_abi.AggError) as e:
        gb.plan(1 << 20, 10, bad)
    assert e.value.status == _abi.AGG_ERR_INVALID_ARG


def test_tuning_limits_are_checked_on_the_host(lib):
    from paper_1311_0059_gb300 import groupby as gb, _abi
    spec = gb.make_spec(ops=15, value_type=_abi.AGG_I64)
    ok = [_abi.agg_tuning(), _abi.agg_tuning(wait_limit_us=1), _abi.agg_tuning(wait_limit_us=60_000_000),
          _abi.agg_tuning(smem_entries=1), _abi.agg_tuning(fan_out=256, warp_dedup=1, max_load_factor=0.95)]
    bad = [_abi.agg_tuning(wait_limit_us=60_000_001), _abi.agg_tuning(smem_entries=512 + 256),
           _abi.agg_tuning(fan_out=8), _abi.agg_tuning(warp_dedup=3), _abi.agg_tuning(max_load_factor=0.96),
           _abi.agg_tuning(fudge=-1.0)]
    for t in ok:
        gb.plan(64 << 20, 1000, spec, t)
    for t in bad:
        with pytest.raises(_abi.AggError) as e:
            gb.plan(64 << 20, 1000, spec, t)
        assert e.value.status == _abi.AGG_ERR_INVALID_ARG


def test_plan_picks_the_in_budget_paths(lib):
    # A table that can hold every row's key at once (n at most half the slots)
    # completes in place: small inputs go to the partitioned path (partitions of
    # about one shared-memory table, 2048 entries), larger ones to the single
    # table; more rows than that, or the knob set to off, give the spilling path.
    from paper_1311_0059_gb300 import groupby as gb, _abi
    spec32 = gb.make_spec(ops=15, value_type=_abi.AGG_I32)
    p = gb.plan(64 << 20, 1_000_000, spec32)        # the plain 1M-row, 10k-key workload
    assert p["in_budget_path"] == 1 and p["partitions"] == 512 and p["staging_bytes"] == 0
    assert p["active_slots"] >= 1_250_000             # room for every key if all overflowed
    spec = gb.make_spec(ops=3, value_type=_abi.AGG_I64)
    p = gb.plan(256 << 20, 3_000_000, spec)           # past the partitioned path's 2M rows
    assert p["in_budget_path"] == 2 and p["active_slots"] >= 6_000_000
    p = gb.plan(256 << 20, 200_000_000, gb.make_spec(ops=15, value_type=_abi.AGG_I64))
    assert p["in_budget_path"] == 0 and p["staging_bytes"] > 0
    p = gb.plan(64 << 20, 1_000_000, spec32, _abi.agg_tuning(in_budget=2))
    assert p["in_budget_path"] == 0
    p = gb.plan(64 << 20, 1_000_000, spec32, _abi.agg_tuning(smem_entries=1))
    assert p["in_budget_path"] == 2                   # no shared-memory tables: the single table
    assert gb.plan(1 << 20, 0, spec)["in_budget_path"] == 2   # empty input: only the empty result
    # the sort path never takes them
    assert gb.plan(64 << 20, 1000, gb.make_spec(ops=15, path=_abi.AGG_PATH_SORT))["in_budget_path"] == 0
    with pytest.raises(_abi.AggError):
        gb.plan(64 << 20, 10, spec, _abi.agg_tuning(in_budget=3))
    with pytest.raises(_abi.AggError):
        gb.plan(64 << 20, 10, spec, _abi.agg_tuning(sorted_input=3))


def test_depth_cap_knob_is_checked_on_the_host(lib):
    from paper_1311_0059_gb300 import groupby as gb, _abi
    spec = gb.make_spec(ops=15, value_type=_abi.AGG_I64)
    for ok in (0, 1, 2, 11):
        gb.plan(64 << 20, 10, spec, _abi.agg_tuning(max_levels=ok))
    for bad in (12, 100):
        with pytest.raises(_abi.AggError):
            gb.plan(64 << 20, 10, spec, _abi.agg_tuning(max_levels=bad))
    for tier in (0, 1, 2):
        gb.plan(64 << 20, 10, spec, _abi.agg_tuning(staging_tier=tier))
    with pytest.raises(_abi.AggError):
        gb.plan(64 << 20, 10, spec, _abi.agg_tuning(staging_tier=3))


def test_level0_table_cap(lib):
    # the level-0 table takes at most AGG_LEVEL0_SLOTS slots unless asked for
    # the whole budget (1) or another cap (>= 4096)
    from paper_1311_0059_gb300 import groupby as gb, _abi
    spec = gb.make_spec(ops=3, value_type=_abi.AGG_I64)
    whole = gb.plan(1 << 30, 100_000_000, spec, _abi.agg_tuning(level0_slots=1))
    assert whole["active_slots"] == whole["table_slots"] > _abi.AGG_LEVEL0_SLOTS
    assert gb.plan(1 << 30, 100_000_000, spec)["active_slots"] == _abi.AGG_LEVEL0_SLOTS
    assert gb.plan(1 << 30, 100_000_000, spec, _abi.agg_tuning(level0_slots=8192))["active_slots"] == 8192
    assert gb.plan(1 << 30, 1000, spec)["active_slots"] < _abi.AGG_LEVEL0_SLOTS   # sized to n below the cap
    # the cost model's resident capacity K follows the cap: more spill, more bytes
    auto = gb.make_spec(ops=3, value_type=_abi.AGG_I64, path=_abi.AGG_PATH_AUTO, expected_groups=10_000_000)
    capped = gb.plan(1 << 30, 100_000_000, auto)["hash_bytes"]
    assert capped > gb.plan(1 << 30, 100_000_000, auto, _abi.agg_tuning(level0_slots=1))["hash_bytes"]
    for bad in (2, 4095):
        with pytest.raises(_abi.AggError):
            gb.plan(64 << 20, 10, spec, _abi.agg_tuning(level0_slots=bad))


def test_cost_model_chooses_between_the_paths(lib):
    # AGG_PATH_AUTO: the model in bytes (input, the Pre-Partitioning spill
    # R(1 - K/G) written and read, the level-1 sort when groups exceed 0.8 of
    # the rows, the result) against the sort path's passes, over each path's
    # measured bandwidth.  Nearly unique keys that spill pick the sort path; low
    # cardinality, small inputs and an unknown G pick the hash path.
    from paper_1311_0059_gb300 import groupby as gb, _abi
    auto = lambda g: gb.make_spec(ops=15, value_type=_abi.AGG_I64, path=_abi.AGG_PATH_AUTO, expected_groups=g)
    p = gb.plan(128 << 20, 3_000_000, auto(3_000_000))
    assert p["chosen_path"] == _abi.AGG_PATH_SORT and p["sort_seconds"] < p["hash_seconds"]
    assert p["hash_bytes"] > 16 * 3_000_000 + 2 * 16 * 1_900_000          # input and the spill both ways
    p = gb.plan(128 << 20, 3_000_000, auto(300_000))
    assert p["chosen_path"] == _abi.AGG_PATH_HASH and p["hash_seconds"] < p["sort_seconds"]
    assert gb.plan(128 << 20, 3_000_000, auto(0))["chosen_path"] == _abi.AGG_PATH_HASH   # G unknown
    assert gb.plan(128 << 20, 50_000, auto(50_000))["chosen_path"] == _abi.AGG_PATH_HASH  # fits the table
    assert gb.plan(256 << 20, 200_000_000, auto(49_000_000))["chosen_path"] == _abi.AGG_PATH_HASH
    assert gb.plan(256 << 20, 50_000_000, auto(50_000_000))["chosen_path"] == _abi.AGG_PATH_SORT
    # the fixed paths report themselves
    assert gb.plan(128 << 20, 3_000_000, gb.make_spec(path=_abi.AGG_PATH_HASH, expected_groups=3_000_000)
                   )["chosen_path"] == _abi.AGG_PATH_HASH
    assert gb.plan(128 << 20, 100, gb.make_spec(path=_abi.AGG_PATH_SORT))["chosen_path"] == _abi.AGG_PATH_SORT
