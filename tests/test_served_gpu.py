"""The served form: queries arriving over time, admitted against a device
memory pool by their declared budgets, running concurrently.  Each query's
result must be the same in the mix as alone (and as the oracle's), exactly;
admission must never let the admitted budgets exceed the pool."""
import time

import numpy as np
import pytest

import datagen as dg
from _gpu import assert_parity, canon, oracle_expected, to_dev

pytestmark = pytest.mark.gpu
MB = 1 << 20


def test_served_results_equal_alone_and_pool_respected(oracle):
    import torch
    from paper_1311_0059_gb300 import _abi
    from paper_1311_0059_gb300.groupby import GroupBy, Output, Server
    qs = dg.served_workloads(duration=0.25, rate=160.0, seed=7, rows=(10_000, 400_000), card=(0.001, 0.5),
                             budget=(MB, 6 * MB))
    assert len(qs) >= 20
    pool = 16 * MB
    srv = Server(pool, max_active=8)
    data, tickets = [], []
    t0 = time.perf_counter()
    for arrival, w in qs:
        while time.perf_counter() - t0 < arrival:
            srv.progress()
        k, v = w.host()
        dk, dv = to_dev(k), to_dev(v)
        out = Output(w.n, 15, "cuda")
        tickets.append(srv.submit(dk, dv, w.budget, out))
        data.append((k, v, w.budget, out))
        srv.progress()
    deadline = time.perf_counter() + 60
    while srv.stats()["completed"] < len(qs) and time.perf_counter() < deadline:
        srv.progress()
    st = srv.stats()
    assert st["completed"] == len(qs)
    assert st["pool_peak"] <= pool
    assert st["max_concurrent"] >= 2, "queries should overlap on the device"
    for (k, v, b, out), t in zip(data, tickets):
        info = srv.poll(t)
        assert info.state == _abi.AGG_QUERY_DONE and info.status == 0
        assert info.t_done >= info.t_start >= info.t_submit
        got = canon({f: x.cpu().numpy() for f, x in out.result(info.n_groups).items()})
        exp = oracle_expected(oracle, k, v)
        assert_parity(got, exp, what=f"ticket {t} in the mix")
    # the same queries alone, one at a time
    for (k, v, b, out), t in list(zip(data, tickets))[:8]:
        with GroupBy(b) as g:
            alone = canon({f: x.cpu().numpy() for f, x in g.run(to_dev(k), to_dev(v)).items()})
        got = canon({f: x.cpu().numpy() for f, x in out.result(srv.poll(t).n_groups).items()})
        assert_parity(got, alone, what=f"ticket {t}: alone vs in the mix")
    srv.close()


def test_served_admission_waits_for_memory():
    # three queries whose budgets each take most of the pool: they must run one by one
    from paper_1311_0059_gb300 import _abi
    from paper_1311_0059_gb300.groupby import Output, Server
    pool = 8 * MB
    srv = Server(pool, max_active=4)
    ws = [dg.Workload(f"q{i}", n=200_000, domain=50_000, seed=i, budget=6 * MB) for i in range(3)]
    outs, ts = [], []
    for w in ws:
        k, v = w.host()
        o = Output(w.n, 15, "cuda")
        ts.append(srv.submit(to_dev(k), to_dev(v), w.budget, o))
        outs.append(o)
    srv.progress()
    st = srv.stats()
    assert st["running"] == 1 and st["queued"] == 2
    while srv.stats()["completed"] < 3:
        srv.progress()
    assert srv.stats()["max_concurrent"] == 1 and srv.stats()["pool_peak"] <= pool
    assert all(srv.poll(t).state == _abi.AGG_QUERY_DONE for t in ts)
    srv.close()


def test_served_rejects_budget_larger_than_pool():
    import torch
    from paper_1311_0059_gb300 import _abi
    from paper_1311_0059_gb300.groupby import Output, Server
    srv = Server(4 * MB, max_active=2)
    k = torch.zeros(10, dtype=torch.int64, device="cuda")
    with pytest.raises(_abi.AggError):
        srv.submit(k, k, 64 * MB, Output(10, 15, "cuda"))
    srv.close()


def test_served_rejects_pointers_the_kernel_cannot_use():
    # host memory, missing values, misaligned keys: argument errors at submit,
    # before anything is queued; a valid query on the same server still runs
    import torch
    from paper_1311_0059_gb300 import _abi
    from paper_1311_0059_gb300.groupby import Output, Server
    srv = Server(16 * MB, max_active=2)
    k = torch.arange(1000, dtype=torch.int64, device="cuda")
    v = torch.ones(1000, dtype=torch.int64, device="cuda")
    raw = torch.zeros(1001, dtype=torch.int64, device="cuda")
    out = Output(1000, 15, "cuda")

    class _Shifted:  # device keys 4 bytes off their 8-byte alignment
        def data_ptr(self):
            return raw.data_ptr() + 4

        def numel(self):
            return 1000

    for kk, vv, oo in ((k.cpu(), v, out), (k, None, out), (k, v.cpu(), out), (k, v, Output(1000, 15, "cpu")),
                       (_Shifted(), v, out)):
        with pytest.raises(_abi.AggError) as e:
            srv.submit(kk, vv, 4 * MB, oo)
        assert e.value.status == _abi.AGG_ERR_INVALID_ARG
    assert srv.stats()["submitted"] == 0
    t = srv.submit(k, v, 4 * MB, out)
    deadline = time.perf_counter() + 60
    while srv.stats()["completed"] < 1 and time.perf_counter() < deadline:
        srv.progress()
    info = srv.poll(t)
    assert info.state == _abi.AGG_QUERY_DONE and info.status == 0 and info.n_groups == 1000
    srv.close()


def test_served_failed_launch_frees_its_ranges_only_after_its_stream(oracle, monkeypatch):
    # The server's test hook AGG_INJECT_LAUNCH_FAILURE=k makes the k-th launch
    # fail on the host after its control-block clear and table set-up were
    # queued on the slot's stream.  The failed query must free its pool ranges
    # only once that queued work is done, and the queries admitted after it
    # (into the same ranges) must still give the oracle's result.
    from paper_1311_0059_gb300 import _abi
    from paper_1311_0059_gb300.groupby import Output, Server
    monkeypatch.setenv("AGG_INJECT_LAUNCH_FAILURE", "2")
    srv = Server(8 * MB, max_active=1)
    ws = [dg.Workload(f"q{i}", n=150_000, domain=40_000, seed=20 + i, budget=6 * MB) for i in range(4)]
    data, ts = [], []
    for w in ws:
        k, v = w.host()
        o = Output(w.n, 15, "cuda")
        ts.append(srv.submit(to_dev(k), to_dev(v), w.budget, o))
        data.append((k, v, o))
    deadline = time.perf_counter() + 60
    while srv.stats()["completed"] < len(ws) and time.perf_counter() < deadline:
        srv.progress()
    st = srv.stats()
    assert st["completed"] == len(ws) and st["pool_in_use"] == 0 and st["staging_in_use"] == 0
    assert st["blocks_in_use"] == 0
    infos = [srv.poll(t) for t in ts]
    assert infos[1].state == _abi.AGG_QUERY_FAILED and infos[1].status == _abi.AGG_ERR_CUDA
    for i in (0, 2, 3):
        assert infos[i].state == _abi.AGG_QUERY_DONE and infos[i].status == 0
        k, v, o = data[i]
        got = canon({f: x.cpu().numpy() for f, x in o.result(infos[i].n_groups).items()})
        assert_parity(got, oracle_expected(oracle, k, v), what=f"query {i} after an injected launch failure")
    srv.close()


def test_served_teams_never_exceed_the_resident_blocks(oracle):
    # Many concurrent queries whose wanted teams add up to several times the
    # blocks the GPU holds at once: admission must keep the running teams within
    # one co-resident wave (no cooperative grid waits on another, so no bounded
    # wait runs out), and every result must equal the oracle's.
    from paper_1311_0059_gb300 import _abi
    from paper_1311_0059_gb300.groupby import Output, Server
    srv = Server(512 * MB, max_active=32)
    ws = [dg.Workload(f"t{i}", n=n, domain=max(n // 8, 1), seed=40 + i, budget=8 * MB)
          for i, n in enumerate([3_000_000, 2_500_000, 4_000_000, 50_000, 3_500_000, 20_000, 2_000_000,
                                 60_000, 3_000_000, 10_000, 2_200_000, 80_000])]
    data, ts = [], []
    for w in ws:
        k, v = w.host()
        o = Output(w.n, 15, "cuda")
        ts.append(srv.submit(to_dev(k), to_dev(v), w.budget, o))
        data.append((k, v, o))
    peak_blocks = 0
    deadline = time.perf_counter() + 120
    while srv.stats()["completed"] < len(ws) and time.perf_counter() < deadline:
        srv.progress()
        st = srv.stats()
        peak_blocks = max(peak_blocks, st["blocks_in_use"])
        assert st["blocks_in_use"] <= st["blocks"]
    st = srv.stats()
    assert st["completed"] == len(ws) and st["max_concurrent"] >= 2
    assert peak_blocks <= st["blocks"]
    for t, (k, v, o) in zip(ts, data):
        info = srv.poll(t)
        assert info.state == _abi.AGG_QUERY_DONE and info.status == 0, f"ticket {t}: status {info.status}"
        got = canon({f: x.cpu().numpy() for f, x in o.result(info.n_groups).items()})
        assert_parity(got, oracle_expected(oracle, k, v), what=f"ticket {t} among concurrent big teams")
    srv.close()
