"""The plain-C example (paper_1311_0059_gb300/examples/groupby_host.c) builds
against include/agg.h and libagg.so alone.  Without a GPU it prints the
host-only plan, which must equal agg_plan's through the Python binding, and
exits 2; on a GPU its run must satisfy the invariants of any correct group-by
(sum of COUNT = rows, sum of SUM = sum of values, groups = distinct keys,
result keys distinct), checked by the program itself."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1311_0059_gb300", "examples", "groupby_host.c")
MB = 1 << 20


def _build(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1311_0059_gb300 import _abi
    if not os.path.exists(_abi.LIB_PATH):
        from paper_1311_0059_gb300 import build
        build.build()
    pkg = os.path.dirname(_abi.LIB_PATH)
    exe = str(tmp_path / "groupby_host")
    subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-I", os.path.join(ROOT, "include"), SRC,
                    "-L", pkg, "-lagg", f"-Wl,-rpath,{pkg}", "-o", exe], check=True)
    return exe


def test_c_example_plans_without_a_gpu(tmp_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the GPU test runs the example end to end")
    from paper_1311_0059_gb300 import _abi
    from paper_1311_0059_gb300 import groupby as gb
    exe = _build(tmp_path)
    r = subprocess.run([exe, "100000", "1000", str(16 * MB)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 2, r.stdout + r.stderr
    line = next(x for x in r.stdout.splitlines() if x.startswith("plan:"))
    words = line.split()[1:]
    got = {words[i]: int(words[i + 1]) for i in range(0, len(words), 2)}
    exp = gb.plan(16 * MB, 100000, gb.make_spec(ops=15, value_type=_abi.AGG_I64))
    assert got == {k: exp[k] for k in got}


@pytest.mark.gpu
@pytest.mark.parametrize("rows,domain,budget", [(300_000, 5_000, 16 * MB), (2_000_000, 1_000_000, 4 * MB)])
def test_c_example_runs_on_the_gpu(tmp_path, rows, domain, budget):
    exe = _build(tmp_path)
    r = subprocess.run([exe, str(rows), str(domain), str(budget)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "invariants hold" in r.stdout
