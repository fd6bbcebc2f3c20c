"""Benchmark of the budgeted group-by on GB300 (one JSON line on stdout).

A step is one agg_run of the hash path over one batch of synthetic rows already
resident in HBM.  The headline workload is the spilling hybrid-hash group-by:
200M rows, int64 keys uniform over a 50M-key domain, int64 values in
[0, 2^20), COUNT+SUM+MIN+MAX, 256 MB working-memory budget, so groups overflow
the table, spill, and recurse.  The same input also runs through the radix-sort
path for comparison.  Inputs (3.2 GB) exceed the 129 MB L2, so no flush is needed
between steps.  The same JSON line carries, under "configs", one record per
other workload: the plain in-budget group-by (1M rows, 10k keys), the skewed one
(500M Zipf rows), the batched form (4,096 instances in one launch against the
plain per-instance loop) and the served form (a 60 s Poisson stream against the
same queries one at a time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload spill|plain|zipf|batched|served] [--no-sub]
                  [--rows R --domain D --budget B]

Under torchrun (N > 1) every rank runs an independent instance of the workload
(its own seed) on its own GPU: the work shards with no data-path collective,
scaling is weak, and `value` is the total rows of all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import datagen as dg  # noqa: E402

WORKLOADS = {"spill": dg.SPILL_200M_50M, "plain": dg.PLAIN_1M_10K, "zipf": dg.ZIPF_500M_10M}
# the headline metric, printed identically by both arms
METRIC = "rows/s & HBM GB/s vs peak, budgeted group-by; batched/served vs plain, p99 latency"
CPU_SAMPLE_ROWS = 2_000_000  # rows of the oracle sample, the same in both arms
L2_BYTES = 129 << 20
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, about 8 TB/s nominal (the measured copy peak is the roofline)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="spill", choices=sorted(WORKLOADS) + ["sorted", "batched", "served"])
    ap.add_argument("--duration", type=float, default=60.0, help="served: seconds of Poisson arrivals")
    ap.add_argument("--rate", type=float, default=200.0, help="served: queries per second")
    ap.add_argument("--max-active", type=int, default=64, help="served: queries running at once")
    ap.add_argument("--instances", type=int, default=4096, help="instances of the batched workload")
    ap.add_argument("--tune", action="store_true", help="batched: run the autotuner and store its winner")
    ap.add_argument("--rows", type=int, default=0)
    ap.add_argument("--domain", type=int, default=0)
    ap.add_argument("--budget", type=int, default=0)
    ap.add_argument("--no-sort", action="store_true", help="skip the sort-path comparison leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=0, help="rows of the oracle sample (default 2M)")
    ap.add_argument("--no-sub", action="store_true", help="headline workload only (no per-config records)")
    return ap.parse_args(argv)


def workload(args, rank=0) -> dg.Workload:
    base = WORKLOADS["spill" if args.workload == "sorted" else args.workload]
    w = dg.Workload(base.name, n=args.rows or base.n, domain=args.domain or base.domain, dist=base.dist,
                    zipf_s=base.zipf_s, vtype=base.vtype, seed=base.seed + rank, budget=args.budget or base.budget,
                    ops=base.ops)
    if args.workload == "sorted":
        w.name = "sorted input: " + base.name + " (rows reordered by key before timing)"
    if args.rows or args.domain or args.budget:
        w.name = f"{w.dist} {w.n} rows over {w.domain} keys, budget {w.budget >> 20} MiB"
    return w


def config_of(w: dg.Workload, n_gpus: int) -> dict:
    return {"workload": w.name, "rows": w.n, "key_domain": w.domain, "distribution": w.dist,
            "zipf_s": w.zipf_s if w.dist == "zipf" else None, "value_type": w.vtype, "budget_bytes": w.budget,
            "ops": "COUNT,SUM,MIN,MAX" if w.ops == 15 else ("COUNT,SUM" if w.ops == 3 else str(w.ops)),
            "global_batch": w.n * n_gpus, "parallelism": f"independent instance per GPU x{n_gpus}",
            "l2": "inputs larger than L2, no flush" if w.n * 16 > 2 * L2_BYTES else "input copies rotated to defeat L2"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, interval_ms: int = 50):
        self.cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-i",
                    str(device_index), "-lms", str(interval_ms)]
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1311_0059_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None).  An entry lists the source hashes it
    holds for: the one it was captured on, plus later ones whose changes leave
    the captured kernel's code and its launch unchanged (each named in _note)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    ent = rec.get(workload_name)
    if not ent or kernel_source_hash() not in ent.get("kernel_source_hashes", []):
        return None
    return ent.get("dram_bytes_per_launch")


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def host_info() -> dict:
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu": model}


def oracle_sample(w: dg.Workload, rows: int):
    """Times the CPU oracle (single thread) on the first `rows` rows of w."""
    import oracle
    keys, vals = w.host(0, rows)
    o = oracle.default()
    t0 = time.perf_counter()
    res, runs = o.groupby(keys, vals, budget_bytes=w.budget)
    dt = time.perf_counter() - t0
    return dt, res["keys"].size, runs


def cpu_sample_rows(w: dg.Workload, args) -> int:
    return min(w.n, args.cpu_rows or CPU_SAMPLE_ROWS)


def cpu_sample_text(w: dg.Workload, rows: int) -> str:
    return (f"first {rows} rows of the headline workload ({w.name}), same distribution and budget, "
            "plain single-threaded C++ oracle")


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    w = workload(args)
    rows = cpu_sample_rows(w, args)
    for _ in range(args.warmup):
        oracle_sample(w, rows)
    times = []
    for _ in range(args.steps):
        dt, _, _ = oracle_sample(w, rows)
        times.append(dt)
    total = sum(times)
    v = rows * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "rows/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": config_of(w, world),
            "cpu_baseline": {"value": v, "unit": "rows/s", "cores": 1, "kind": "oracle",
                             "sample": cpu_sample_text(w, rows), "host": host_info()},
            "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def make_inputs(w: dg.Workload, vt: int, dev, stream, sort_keys: bool = False):
    """Device inputs of w; a small input is copied enough times that rotating
    through the copies streams more than twice the L2 per pass.  sort_keys
    reorders the rows by key (input preparation, before any timing)."""
    import torch
    from paper_1311_0059_gb300 import AGG_I32
    copies = 1 if w.n * 16 > 2 * L2_BYTES else max(2, (4 * L2_BYTES) // max(w.n * 12, 1) + 1)
    keys, vals, cdf = [], [], None
    for _ in range(copies):
        k = torch.empty(w.n, dtype=torch.int64, device=dev)
        v = torch.empty(w.n, dtype=torch.int32 if vt == AGG_I32 else torch.int64, device=dev)
        if w.dist == "zipf" and cdf is None:
            cdf = torch.from_numpy(w.cdf()).to(dev)
        w.device(k.data_ptr(), v.data_ptr(), cdf_ptr=cdf.data_ptr() if cdf is not None else 0,
                 stream_handle=stream.cuda_stream)
        if sort_keys:
            k, order = torch.sort(k)
            v = v[order]
            del order
        keys.append(k)
        vals.append(v)
    torch.cuda.synchronize()
    return keys, vals


PATH_KERNELS = {0: "hash_groupby_kernel", 1: "part_scatter_kernel + part_agg_kernel",
                2: "fast_agg_kernel + fast_emit_kernel"}


def measure_hash(w: dg.Workload, steps: int, warmup: int, world: int, local: int, dev, stream,
                 sort_keys: bool = False) -> dict:
    """One agg_run per step over w's rows, resident in HBM, timed with CUDA
    events on the launching stream; the roofline counts input, spill written,
    spill read and result bytes.  Returns the record and the live objects."""
    import torch
    from paper_1311_0059_gb300 import AGG_I32, AGG_I64, AGG_PATH_HASH, _abi
    from paper_1311_0059_gb300.costmodel import predicted_spill_records
    from paper_1311_0059_gb300.groupby import GroupBy, make_spec, plan

    vt = AGG_I32 if w.vtype == "i32_1000" else AGG_I64
    keys, vals = make_inputs(w, vt, dev, stream, sort_keys)
    copies = len(keys)
    g = GroupBy(w.budget, ops=w.ops, value_type=vt, path=AGG_PATH_HASH)
    g.reserve(w.n)
    out = g.output(w.n, dev)
    path = plan(w.budget, w.n, make_spec(ops=w.ops, value_type=vt))["in_budget_path"]

    def step(i):
        st = g.run_async(keys[i % copies], vals[i % copies], out, w.n, stream)
        if st != 0:
            raise RuntimeError(f"agg_run failed with status {st}")

    for i in range(max(warmup, 1)):
        step(i)
    n_groups = g.sync()
    launches0 = g.stats()["kernel_launches"]
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for i in range(steps):
            step(i)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms_total = ev0.elapsed_time(ev1)
    g.sync()
    stats = g.stats()
    gpu_launches = stats["kernel_launches"] - launches0
    ms_max = max_over_ranks(ms_total, world, dev)
    rows_total = sum_over_ranks(float(w.n * steps), world, dev)

    in_b = w.n * (8 + (4 if vt == AGG_I32 else 8))
    spill_b = stats["spill_bytes_written"] + stats["spill_bytes_read"]
    nagg = bin(w.ops).count("1")
    out_b = n_groups * 8 * (1 + nagg)
    alg_bytes = in_b + spill_b + out_b
    run_ms = ms_total / steps  # one run per step
    peak, peak_kind = measured_peak_gbs()
    achieved = alg_bytes / (run_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": recorded_traffic(w.name), "kernel": PATH_KERNELS[path], "peak_kind": peak_kind,
            "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
            "algorithmic_bytes_per_launch": alg_bytes, "launches_per_run": gpu_launches / steps,
            "bytes_breakdown": {"input": in_b, "spill_write": stats["spill_bytes_written"],
                                "spill_read": stats["spill_bytes_read"], "result": out_b}}
    rec = {"workload": w.name, "rows_per_s": rows_total / (ms_max / 1e3), "ms_per_run": ms_max / steps,
           "steps": steps, "roofline": roof, "gpu_launches": gpu_launches, "n_groups": n_groups,
           "in_budget_path": path, "levels": stats["levels"], "sorted_input_path": stats["sorted_input"],
           "fallback_records": stats["fallback_records"], "clocks": clocks.summary(),
           "l2": "inputs larger than L2, no flush" if copies == 1 else f"{copies} input copies rotated to defeat L2"}
    if spill_b:
        # planned level-0 groups: the table's capacity, within the level-0 cap
        k_cap = min(stats["table_capacity"],
                    stats["table_capacity"] * _abi.AGG_LEVEL0_SLOTS // max(stats["table_slots"], 1))
        k_res = stats["resident_groups"][0]
        pred = predicted_spill_records(w.n, k_cap, n_groups)
        rec["spill"] = {"measured_records_level0": stats["spill_records"][0], "measured_bytes_total": spill_b,
                        "model_records_level0": pred, "model_bytes_level0": pred * 16, "K": k_cap, "G_t": n_groups,
                        "K_resident_level0": k_res,
                        "model_records_level0_K_resident": predicted_spill_records(w.n, k_res, n_groups),
                        "levels": stats["levels"], "rounds": stats["rounds"], "fan_out": stats["fan_out"]}
    return rec, {"g": g, "keys": keys, "vals": vals, "out": out, "vt": vt, "in_b": in_b, "nagg": nagg}


def sort_leg(w, live, steps, dev, stream) -> dict:
    import torch
    from paper_1311_0059_gb300 import AGG_PATH_SORT
    from paper_1311_0059_gb300.groupby import GroupBy
    keys, vals, vt = live["keys"], live["vals"], live["vt"]
    copies = len(keys)
    gs = GroupBy(w.budget, ops=w.ops, value_type=vt, path=AGG_PATH_SORT)
    gs.reserve(w.n)
    outs = gs.output(w.n, dev)
    for _ in range(2):
        assert gs.run_async(keys[0], vals[0], outs, w.n, stream) == 0
    ng_sort = gs.sync()
    sk = max(3, min(10, steps))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(sk):
        assert gs.run_async(keys[i % copies], vals[i % copies], outs, w.n, stream) == 0
    ev1.record(stream)
    torch.cuda.synchronize()
    gs.sync()
    sms = ev0.elapsed_time(ev1) / sk
    gs.close()
    return {"rows_per_s": w.n / (sms / 1e3), "ms_per_run": sms, "n_groups": ng_sort, "steps": sk}


def e2e_leg(w, live, n_groups, steps, world, dev, stream) -> dict:
    """The same metric through agg_run_host on pinned host buffers: every step
    moves its input host->device and its result device->host."""
    import ctypes

    import torch
    from paper_1311_0059_gb300._abi import agg_output, check
    g, keys, vals, in_b, nagg = live["g"], live["keys"], live["vals"], live["in_b"], live["nagg"]
    hk = torch.empty(w.n, dtype=torch.int64, pin_memory=True)
    hv = torch.empty(w.n, dtype=vals[0].dtype, pin_memory=True)
    hk.copy_(keys[0])
    hv.copy_(vals[0])
    cap = max(n_groups, 1)
    hout = {f: torch.empty(cap, dtype=torch.int64, pin_memory=True) for f in ("keys", "count", "sum", "min", "max")}
    ho = agg_output(keys=hout["keys"].data_ptr(), count=hout["count"].data_ptr(), sum=hout["sum"].data_ptr(),
                    min=hout["min"].data_ptr(), max=hout["max"].data_ptr(), capacity=cap, d_n_groups=None)
    ng = ctypes.c_uint64()
    sp = ctypes.c_void_p(stream.cuda_stream)

    def once():
        check(g.lib.agg_run_host(g.h, ctypes.c_void_p(hk.data_ptr()), ctypes.c_void_p(hv.data_ptr()), w.n,
                                 ctypes.byref(ho), ctypes.byref(ng), sp), "agg_run_host")

    for _ in range(2):
        once()
    ek = max(3, min(10, steps))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(ek):
        once()
    dt = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_rows = sum_over_ranks(float(w.n * ek), world, dev)
    return {"value": e2e_rows / dt, "unit": "rows/s", "h2d_bytes_per_step": in_b,
            "d2h_bytes_per_step": int(ng.value) * 8 * (1 + nagg) + 8, "steps": ek,
            "api": "agg_run_host on pinned host buffers: the kernel reads the input from and writes the result "
                   "rows into host memory over the host link, inside the timed region"}


def release(live):
    import torch
    live["g"].close()
    live.clear()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args, rank)
    stream = torch.cuda.current_stream()

    rec, live = measure_hash(w, args.steps, args.warmup, world, local, dev, stream,
                             sort_keys=args.workload == "sorted")
    line = {"metric": METRIC, "value": rec["rows_per_s"], "unit": "rows/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rec["ms_per_run"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded SplitMix64 generator, generated on the device)",
            "config": config_of(w, world), "roofline": rec["roofline"], "gpu_launches": rec["gpu_launches"],
            "n_groups": rec["n_groups"], "in_budget_path": rec["in_budget_path"], "clocks": rec["clocks"]}
    line["config"]["l2"] = rec["l2"]
    if "spill" in rec:
        line["spill"] = rec["spill"]
    if not args.no_sort:
        try:
            sl = sort_leg(w, live, args.steps, dev, stream)
            sl["same_group_count"] = sl["n_groups"] == rec["n_groups"]
            line["sort_path"] = sl
        except Exception as e:  # the comparison leg must not hide the main number
            line["sort_path"] = {"error": str(e)}
    if not args.no_e2e:
        line["e2e"] = e2e_leg(w, live, rec["n_groups"], args.steps, world, dev, stream)
    release(live)

    if not args.no_cpu and rank == 0:
        rows = cpu_sample_rows(w, args)
        times = []
        for _ in range(3):
            dt, ng_s, runs = oracle_sample(w, rows)
            times.append(dt)
        dt = statistics.median(times)
        line["cpu_baseline"] = {"value": rows / dt, "unit": "rows/s", "cores": 1, "kind": "oracle",
                                "sample": cpu_sample_text(w, rows) + f" ({ng_s} groups, {runs} sorted runs), "
                                                                    "median of 3", "seconds": dt,
                                "host": host_info()}

    # one record per other workload, in the same line
    if not args.no_sub and args.workload == "spill" and not (args.rows or args.domain or args.budget):
        configs = {}
        for name, wl, steps, srt in (("plain", dg.PLAIN_1M_10K, max(args.steps, 200), False),
                                     ("skewed", dg.ZIPF_500M_10M, args.steps, False),
                                     ("sorted", dg.SPILL_200M_50M, args.steps, True)):
            wr = dg.Workload(wl.name, n=wl.n, domain=wl.domain, dist=wl.dist, zipf_s=wl.zipf_s, vtype=wl.vtype,
                             seed=wl.seed + rank, budget=wl.budget, ops=wl.ops)
            if srt:
                wr.name = "sorted input: " + wl.name + " (rows reordered by key before timing)"
            try:
                r, lv = measure_hash(wr, steps, args.warmup, world, local, dev, stream, sort_keys=srt)
                release(lv)
                configs[name] = r
            except Exception as e:
                configs[name] = {"error": str(e)}
        try:
            configs["batched"] = batched_record(args, world, rank, local, dev, stream)
        except Exception as e:
            configs["batched"] = {"error": str(e)}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        try:
            configs["served"] = served_record(args, world, rank, local, dev)
        except Exception as e:
            configs["served"] = {"error": str(e)}
        line["configs"] = configs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ batched workload

def batched_record(args, world, rank, local, dev, stream) -> dict:
    """4,096 independent instances in one persistent launch (CUDA graph replay)
    against the plain loop of one agg_run per instance, at identical output."""
    import torch
    from paper_1311_0059_gb300 import AGG_I64, agg_tuning, autotune
    from paper_1311_0059_gb300.groupby import Batch, GroupBy

    ws = dg.batch_workloads(args.instances, seed=rank)
    inst = []
    for w in ws:
        k = torch.empty(w.n, dtype=torch.int64, device=dev)
        v = torch.empty(w.n, dtype=torch.int64, device=dev)
        cdf = torch.from_numpy(w.cdf()).to(dev) if w.dist == "zipf" else None
        w.device(k.data_ptr(), v.data_ptr(), cdf_ptr=cdf.data_ptr() if cdf is not None else 0,
                 stream_handle=stream.cuda_stream)
        inst.append((k, v, w.budget, 0))
    torch.cuda.synchronize()
    caps = [min(w.n, w.domain) for w in ws]  # a group per distinct key at most
    rows = sum(w.n for w in ws)
    wclass = f"batched-{args.instances}"

    def make(t):
        return Batch(inst, ops=15, value_type=AGG_I64, tuning=t, capacities=caps)

    tuning = None if args.tune else autotune.lookup(wclass)
    tune_info = None
    if tuning is None:
        best, trials = autotune.tune_batch(make, reps=2, log=lambda m: print(m, file=sys.stderr))
        autotune.store(wclass, best, trials)
        tuning = autotune.lookup(wclass)
        tune_info = {"trials": len(trials), "best": best}
    b = make(tuning)
    for _ in range(max(args.warmup, 1)):
        assert b.run_async(stream) == 0
    counts_b = b.sync()
    steps = max(3, min(args.steps, 20))
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(steps):
            assert b.run_async(stream) == 0
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms_batch = max_over_ranks(ev0.elapsed_time(ev1) / steps, world, dev)
    b.sync()

    # plain loop: one agg_run per instance on handles whose budget is the
    # instance's budget rounded up to a power of two MiB (never less memory)
    handles = {}

    def handle_for(budget):
        mb = 4
        while (mb << 20) < budget:
            mb *= 2
        if mb not in handles:
            h = GroupBy(mb << 20, ops=15, value_type=AGG_I64)
            h.reserve(max(w.n for w in ws))
            handles[mb] = h
        return handles[mb]

    outs = b.outs

    def plain_pass():
        for (k, v, bud, _), o, w in zip(inst, outs, ws):
            assert handle_for(bud).run_async(k, v, o, w.n, stream) == 0

    plain_pass()
    torch.cuda.synchronize()
    counts_p = [int(o.n_groups.item()) for o in outs]
    reps_plain = max(1, min(3, steps))
    ev0.record(stream)
    for _ in range(reps_plain):
        plain_pass()
    ev1.record(stream)
    torch.cuda.synchronize()
    for h in handles.values():
        h.sync()
    ms_plain = max_over_ranks(ev0.elapsed_time(ev1) / reps_plain, world, dev)
    rows_all = sum_over_ranks(float(rows), world, dev)
    rec = {"workload": f"batched: {args.instances} instances, rows log-uniform [1e3, 4e6], distinct 1-50% of rows, "
                       "uniform or Zipf(s in [0.5,1.2]), budgets log-uniform [4, 64] MiB, COUNT+SUM+MIN+MAX",
           "rows": rows, "rows_per_s": rows_all / (ms_batch / 1e3), "ms_per_batch": ms_batch, "steps": steps,
           "team_blocks": tuning.team_blocks, "smem_entries": tuning.smem_entries,
           "max_load_factor": tuning.max_load_factor,
           "plain_loop": {"rows_per_s": rows_all / (ms_plain / 1e3), "ms_per_pass": ms_plain,
                          "launches_per_pass": len(ws)},
           "speedup_vs_plain": ms_plain / ms_batch, "identical_group_counts": counts_b == counts_p,
           "gpu_launches": steps, "clocks": clocks.summary()}
    if tune_info:
        rec["autotune"] = tune_info
    b.close()
    for h in handles.values():
        h.close()
    del inst, outs
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec


def run_batched(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    rec = batched_record(args, world, rank, local, dev, stream)
    line = {"metric": "batched group-by rows/s (4,096 instances, one persistent launch)",
            "value": rec["rows_per_s"], "unit": "rows/s", "n_gpus": world, "steps": rec["steps"],
            "warmup": args.warmup, "ms_per_step": rec["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic (seeded, generated on the device)",
            "config": {"workload": rec["workload"], "rows": rec["rows"], "team_blocks": rec["team_blocks"],
                       "smem_entries": rec["smem_entries"], "max_load_factor": rec["max_load_factor"]},
            **{k: rec[k] for k in ("plain_loop", "speedup_vs_plain", "identical_group_counts", "gpu_launches",
                                   "clocks")}}
    if "autotune" in rec:
        line["autotune"] = rec["autotune"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ served workload

def served_record(args, world, rank, local, dev) -> dict:
    """Poisson arrivals of group-by queries admitted against a 64 GB device pool
    by their declared budgets.  The same arrivals go through the same request
    loop twice: with continuous admission (up to --max-active queries running
    at once, on teams of blocks that never exceed one co-resident wave) and one
    query at a time (each alone on the whole GPU).  Latency is arrival -> result
    ready; rows/s is the capacity measured by submitting the same queries as fast
    as the loop accepts them (at most 2 x max-active in flight)."""
    import torch
    from paper_1311_0059_gb300 import AGG_I64
    from paper_1311_0059_gb300.groupby import Output, Server

    qs = dg.served_workloads(duration=args.duration, rate=args.rate, seed=rank)
    zd = [w.domain for _, w in qs if w.dist == "zipf"]
    hdev = torch.from_numpy(dg.harmonic(max(zd) if zd else 1).copy()).to(dev)
    gen = torch.cuda.Stream(device=dev)

    def make_input(w):
        with torch.cuda.stream(gen):
            k = torch.empty(w.n, dtype=torch.int64, device=dev)
            v = torch.empty(w.n, dtype=torch.int64, device=dev)
            cdf = None
            if w.dist == "zipf":
                cdf = hdev[:w.domain] / hdev[w.domain - 1]
                cdf[-1] = 2.0
            w.device(k.data_ptr(), v.data_ptr(), cdf_ptr=cdf.data_ptr() if cdf is not None else 0,
                     stream_handle=gen.cuda_stream)
            ev = torch.cuda.Event()
            ev.record(gen)
        return k, v, ev

    def serve(max_active, paced):
        srv = Server(64 << 30, max_active=max_active, ops=15, value_type=AGG_I64)
        tickets, live = [], {}

        def reap():
            for tt in list(live):
                if srv.poll(tt).state >= 2:
                    srv.release(tt)
                    del live[tt]

        t0 = time.perf_counter()
        for arr, w in qs:
            if paced:
                while time.perf_counter() - t0 < arr:
                    srv.progress()
            else:
                while len(live) >= 2 * max_active:
                    if srv.progress():
                        reap()
            k, v, ev = make_input(w)
            out = Output(min(w.n, w.domain), 15, dev)
            t = srv.submit(k, v, w.budget, out, ready_event=ev)
            tickets.append(t)
            live[t] = True
            if srv.progress():
                reap()
        while srv.stats()["completed"] < len(qs):
            if srv.progress():
                reap()
        infos = [srv.poll(t) for t in tickets]
        st = srv.stats()
        srv.close()
        lat = np.array([i.t_done - i.t_submit for i in infos])
        span = max(i.t_done for i in infos) - min(i.t_submit for i in infos)
        return {"lat": lat, "span": span, "ng": [i.n_groups for i in infos], "stats": st,
                "failed": sum(1 for i in infos if i.state != 2), "status": [i.status for i in infos]}

    rows = sum(w.n for _, w in qs)
    with ClockSampler(local, interval_ms=200) as clocks:
        cont = serve(args.max_active, paced=True)
    one = serve(1, paced=True)
    cont_cap = serve(args.max_active, paced=False)
    one_cap = serve(1, paced=False)

    def pct(r):
        return {"p50_ms": float(np.percentile(r["lat"], 50) * 1e3), "p99_ms": float(np.percentile(r["lat"], 99) * 1e3),
                "max_ms": float(r["lat"].max() * 1e3)}

    runs = (cont, one, cont_cap, one_cap)
    return {"workload": f"served: Poisson {args.rate:g} queries/s for {args.duration:g} s, rows log-uniform "
                        "[1e4, 1e8], distinct 0.1-50% of rows, uniform or Zipf(1.0), budgets log-uniform "
                        "[16 MiB, 2 GiB], 64 GiB pool", "queries": len(qs), "rows": rows,
            "max_active": args.max_active,
            "rows_per_s": sum_over_ranks(rows / cont_cap["span"], world, dev), "span_s": cont_cap["span"],
            "latency": pct(cont),
            "one_at_a_time": dict(pct(one), rows_per_s=rows / one_cap["span"]),
            "speedup_vs_one_at_a_time": one_cap["span"] / cont_cap["span"],
            "identical_group_counts": cont["ng"] == one["ng"] == cont_cap["ng"] == one_cap["ng"],
            "failed_queries": sum(r["failed"] for r in runs),
            "timeouts": sum(1 for r in runs for s_ in r["status"] if s_ == 6),
            "pool_peak_bytes": cont["stats"]["pool_peak"], "staging_peak_bytes": cont["stats"]["staging_peak"],
            "max_concurrent": cont["stats"]["max_concurrent"], "paced_rows_per_s": rows / cont["span"],
            "clocks": clocks.summary()}


def run_served(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rec = served_record(args, world, rank, local, dev)
    line = {"metric": "served group-by rows/s with p50/p99 latency (continuous admission against a 64 GB pool)",
            "value": rec["rows_per_s"], "unit": "rows/s", "n_gpus": world, "steps": rec["queries"], "warmup": 0,
            "ms_per_step": 1e3 * rec["span_s"] / rec["queries"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded; each input generated on the device at its arrival)",
            "config": {"workload": rec["workload"], "queries": rec["queries"], "rows": rec["rows"],
                       "max_active": rec["max_active"]},
            **{k: v for k, v in rec.items() if k not in ("workload", "queries", "rows", "max_active", "rows_per_s")}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
