"""The N>1 path of bench.py, on CPU with the gloo backend (world size 2).

The group-by shards by independent problems: every rank runs its own instance
of the workload (its own seed) and the ranks exchange nothing but the timing
reductions.  These tests check those reductions, the per-rank inputs and the
rank-0-only output of the reference arm, without a GPU."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        args = bench.parse_args(["--workload", "plain", "--rows", "4096"])
        w = bench.workload(args, rank)
        k, _ = w.host(0, 64)
        res = {
            "max": bench.max_over_ranks(10.0 * (rank + 1), world),
            "sum": bench.sum_over_ranks(1.5 * (rank + 1), world),
            "seed": w.seed,
            "keys": k.tolist(),
        }
        bench.barrier(world)
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_timing_reductions_and_per_rank_instances_gloo():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert got[r]["max"] == 20.0          # the slowest rank's time is the job's time
        assert got[r]["sum"] == 4.5           # units processed add up over ranks
    assert got[0]["seed"] != got[1]["seed"]   # weak scaling: an independent instance per rank
    assert not np.array_equal(got[0]["keys"], got[1]["keys"])


def test_reference_arm_prints_one_line_from_rank_0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--workload", "plain",
           "--gpus", "2", "--steps", "2", "--warmup", "1", "--cpu-rows", "20000"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_single_rank_helpers_need_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.sum_over_ranks(3.0, 1) == 3.0
    bench.barrier(1)
