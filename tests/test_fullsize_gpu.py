"""Bit-exact parity with the CPU oracle at the full sizes of the benchmark
workloads: every group of the spilling (200M rows) and skewed (500M rows)
runs, every one of the 4,096 batched instances, and the queries of the 60 s
served stream (each query of at most 1e6 rows and a seeded 2% sample of the
larger ones against the oracle; ΣCOUNT, ΣSUM, global MIN/MAX and the group count
bound on every query).  The oracle work is spread over the host's cores
(tests/_fullsize.py)."""
import numpy as np
import pytest

import datagen as dg
from _fullsize import Shared, oracle_part, oracle_workload, part_of, pool, workload_params
from _gpu import FIELDS, OPS_BITS, check_invariants, device_workload

pytestmark = pytest.mark.gpu

PLOG = 4  # 16 key-disjoint parts


def _compare(got: dict, exp: dict, ops: int, what: str):
    gk, ek = got["keys"], exp["keys"]
    assert gk.size == ek.size, f"{what}: {gk.size} groups, oracle has {ek.size}"
    assert np.array_equal(gk, ek), f"{what}: group keys differ"
    for f, bit in OPS_BITS.items():
        if ops & bit:
            g = np.asarray(got[f]).astype(np.int64)
            e = np.asarray(exp[f]).astype(np.uint64).view(np.int64) if f == "count" else np.asarray(exp[f])
            bad = np.flatnonzero(g != e)
            assert bad.size == 0, f"{what}: {f} differs at {bad.size} groups, first key {gk[bad[0]]}"


def _full_size(w: dg.Workload):
    import torch
    from paper_1311_0059_gb300 import AGG_I32, AGG_I64
    from paper_1311_0059_gb300.groupby import GroupBy
    keys, vals, _ = device_workload(w)
    # inputs into shared memory for the oracle workers
    sk, sv = Shared(w.n, np.int64), Shared(w.n, np.int32 if vals.dtype == torch.int32 else np.int64)
    try:
        torch.from_numpy(sk.array).copy_(keys)
        torch.from_numpy(sv.array).copy_(vals)
        with pool() as p:
            pending = p.map_async(oracle_part, [(sk.ref(), sv.ref(), q, PLOG, w.budget) for q in range(1 << PLOG)])
            vt = AGG_I32 if w.vtype == "i32_1000" else AGG_I64
            with GroupBy(w.budget, ops=w.ops, value_type=vt) as g:
                res = g.run(keys, vals)
                got = {k: t.cpu().numpy() for k, t in res.items()}
                st = g.stats()
            del keys, vals, res
            torch.cuda.empty_cache()
            v64 = sv.array.astype(np.int64) if sv.dtype == np.int32 else sv.array
            vsum = v64.view(np.uint64).sum(dtype=np.uint64) if w.ops & 2 else None
            gmin, gmax = int(v64.min()), int(v64.max())
            del v64
            parts = dict(pending.get())
    finally:
        sk.close()
        sv.close()
    assert st["n_groups"] == got["keys"].size
    gp = part_of(got["keys"], PLOG)
    total = 0
    for q in range(1 << PLOG):
        m = gp == q
        o = np.argsort(got["keys"][m], kind="stable")
        sub = {f: got[f][m][o] for f in got}
        _compare(sub, parts[q], w.ops, f"{w.name}, part {q}")
        total += sub["keys"].size
    assert total == got["keys"].size
    c = {f: got[f] for f in got}
    check_invariants({**c, "keys": np.sort(c["keys"])}, w.n, vsum, global_min=gmin if w.ops & 4 else None,
                     global_max=gmax if w.ops & 8 else None)
    return st


def test_spilling_200m_rows_every_group():
    st = _full_size(dg.SPILL_200M_50M)
    assert st["levels"] >= 2 and st["spill_records"][0] > 0


def test_skewed_500m_rows_every_group():
    # the 10M groups would fit the 1 GB table, but the level-0 table stops at
    # 2^22 slots: the groups that fill it first stay resident (the hot keys
    # among them) and the tail's rows spill once
    st = _full_size(dg.ZIPF_500M_10M)
    assert st["levels"] == 2 and st["spill_records"][0] > 0


def test_plain_1m_rows_every_group():
    st = _full_size(dg.PLAIN_1M_10K)
    assert st["levels"] == 1


def test_batched_4096_instances_every_instance():
    import torch
    from paper_1311_0059_gb300 import AGG_I64, autotune
    from paper_1311_0059_gb300.groupby import Batch
    ws = dg.batch_workloads(4096, seed=0)
    with pool() as p:
        pending = p.imap_unordered(oracle_workload, [(i, workload_params(w)) for i, w in enumerate(ws)],
                                   chunksize=4)
        inst = []
        stream = torch.cuda.current_stream()
        for w in ws:
            k = torch.empty(w.n, dtype=torch.int64, device="cuda")
            v = torch.empty(w.n, dtype=torch.int64, device="cuda")
            cdf = torch.from_numpy(w.cdf()).cuda() if w.dist == "zipf" else None
            w.device(k.data_ptr(), v.data_ptr(), cdf_ptr=cdf.data_ptr() if cdf is not None else 0,
                     stream_handle=stream.cuda_stream)
            inst.append((k, v, w.budget, 0))
        torch.cuda.synchronize()
        b = Batch(inst, ops=15, value_type=AGG_I64, tuning=autotune.lookup("batched-4096"),
                  capacities=[min(w.n, w.domain) for w in ws])
        res = b.run()
        counts = [int(r["keys"].numel()) for r in res]
        del inst
        checked = 0
        for i, exp in pending:
            got = {f: t.cpu().numpy() for f, t in res[i].items()}
            o = np.argsort(got["keys"], kind="stable")
            _compare({f: a[o] for f, a in got.items()}, exp, 15, f"batched instance {i} ({ws[i].n} rows)")
            assert counts[i] == exp["keys"].size
            checked += 1
        b.close()
    assert checked == len(ws)


def test_served_60s_stream_sampled_against_the_oracle():
    import torch
    from paper_1311_0059_gb300 import AGG_I64
    from paper_1311_0059_gb300.groupby import Output, Server
    qs = dg.served_workloads(duration=60.0, rate=200.0, seed=0)
    rng = np.random.default_rng(2024)
    checked = {i for i, (_, w) in enumerate(qs) if w.n <= 1_000_000 or rng.random() < 0.02}
    zd = [w.domain for _, w in qs if w.dist == "zipf"]
    hdev = torch.from_numpy(dg.harmonic(max(zd)).copy()).cuda()
    srv = Server(64 << 30, max_active=64, ops=15, value_type=AGG_I64)
    gen = torch.cuda.Stream()
    live, got_results, inv = {}, {}, 0
    with pool() as p:
        pending = p.imap_unordered(oracle_workload, [(i, workload_params(qs[i][1])) for i in sorted(checked)],
                                   chunksize=8)

        def finish(t):
            nonlocal inv
            i, k, v, out = live.pop(t)
            info = srv.poll(t)
            assert info.state == 2 and info.status == 0, f"query {i}: state {info.state} status {info.status}"
            w = qs[i][1]
            ng = int(info.n_groups)
            assert 1 <= ng <= min(w.n, w.domain), f"query {i}: {ng} groups"
            r = out.result(ng)
            # invariants on every query, on the device
            assert int(r["count"].sum().item()) == w.n, f"query {i}: COUNTs do not add up to n"
            assert int(r["sum"].sum().item()) == int(v.sum().item()), f"query {i}: SUMs"
            assert int(r["min"].min().item()) == int(v.min().item()), f"query {i}: global MIN"
            assert int(r["max"].max().item()) == int(v.max().item()), f"query {i}: global MAX"
            inv += 1
            if i in checked:
                got_results[i] = {f: t.cpu().numpy() for f, t in r.items()}
            srv.release(t)

        for i, (_, w) in enumerate(qs):
            while len(live) >= 128:
                if srv.progress():
                    for t in [t for t in live if srv.poll(t).state >= 2]:
                        finish(t)
            with torch.cuda.stream(gen):  # inputs made on a side stream; the query waits on its event
                k = torch.empty(w.n, dtype=torch.int64, device="cuda")
                v = torch.empty(w.n, dtype=torch.int64, device="cuda")
                cdf = None
                if w.dist == "zipf":
                    cdf = hdev[:w.domain] / hdev[w.domain - 1]
                    cdf[-1] = 2.0
                w.device(k.data_ptr(), v.data_ptr(), cdf_ptr=cdf.data_ptr() if cdf is not None else 0,
                         stream_handle=gen.cuda_stream)
                ev = torch.cuda.Event()
                ev.record(gen)
            out = Output(min(w.n, w.domain), 15, "cuda")
            t = srv.submit(k, v, w.budget, out, ready_event=ev)
            live[t] = (i, k, v, out)
            if srv.progress():
                for t in [t for t in live if srv.poll(t).state >= 2]:
                    finish(t)
        while live:
            srv.progress()
            for t in [t for t in live if srv.poll(t).state >= 2]:
                finish(t)
        st = srv.stats()
        srv.close()
        assert inv == len(qs) and st["max_concurrent"] >= 2
        n_checked = 0
        for i, exp in pending:
            got = got_results.pop(i)
            o = np.argsort(got["keys"], kind="stable")
            _compare({f: a[o] for f, a in got.items()}, exp, 15, f"served query {i} ({qs[i][1].n} rows)")
            n_checked += 1
    assert n_checked == len(checked) and n_checked > len(qs) // 3
