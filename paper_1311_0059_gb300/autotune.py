"""Autotuner of the batched form.

Runs a batch under each candidate setting of the knobs the planner cannot
derive from the data alone - the team shape (thread blocks per instance), the
shared-memory table size and the table load factor - and keeps the fastest.
Results do not depend on these knobs (they change only speed), so any setting
is safe; the table of winners is stored in tuning_table.json beside this file,
keyed by workload class, and read by callers that do not tune themselves.
"""
from __future__ import annotations

import itertools
import json
import os
import time

from ._abi import agg_batch_tuning

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning_table.json")

CANDIDATES = {
    "team_blocks": (1, 2, 4, 8, 16),
    "smem_entries": (1024, 2048),
    "max_load_factor": (0.5, 0.7),
}


def load_table() -> dict:
    try:
        with open(TABLE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(workload_class: str) -> agg_batch_tuning | None:
    ent = load_table().get(workload_class)
    if not ent:
        return None
    return agg_batch_tuning(team_blocks=ent["team_blocks"], smem_entries=ent["smem_entries"],
                            max_load_factor=ent["max_load_factor"], fan_out=0, use_graph=0)


def tune_batch(make_batch, reps: int = 3, candidates: dict | None = None, log=print) -> tuple[dict, list]:
    """make_batch(tuning) -> object with run_async()/sync(); returns (best, trials)."""
    import torch
    cand = candidates or CANDIDATES
    trials = []
    for tb, ns, lf in itertools.product(cand["team_blocks"], cand["smem_entries"], cand["max_load_factor"]):
        t = agg_batch_tuning(team_blocks=tb, smem_entries=ns, max_load_factor=lf, fan_out=0, use_graph=0)
        b = make_batch(t)
        b.run_async()
        b.sync()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.run_async()
        e1.record()
        torch.cuda.synchronize()
        b.sync()
        ms = e0.elapsed_time(e1) / reps
        b.close()
        rec = {"team_blocks": tb, "smem_entries": ns, "max_load_factor": lf, "ms": ms}
        trials.append(rec)
        if log:
            log(json.dumps(rec))
    best = min(trials, key=lambda r: r["ms"])
    return best, trials


def store(workload_class: str, best: dict, trials: list) -> None:
    table = load_table()
    table[workload_class] = dict(best, trials=len(trials), when=time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()))
    with open(TABLE, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
