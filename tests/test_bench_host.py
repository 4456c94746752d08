"""Host-side checks of bench.py and __graft_entry__.py that need no GPU: every name
they load is bound somewhere in the module (a name dropped by an edit only fails
when its line runs, which may be minutes into a GPU run), and the JSON keys the
measurement line promises are spelled in the source."""
import ast
import builtins
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def unbound_names(path):
    tree = ast.parse(open(path).read())
    bound = set(dir(builtins)) | {"__file__", "__name__"}
    for n in ast.walk(tree):
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            bound.add(n.name)
        elif isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            bound.add(n.id)
        elif isinstance(n, ast.arg):
            bound.add(n.arg)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            for a in n.names:
                bound.add((a.asname or a.name).split(".")[0])
        elif isinstance(n, ast.ExceptHandler) and n.name:
            bound.add(n.name)
    loaded = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
    return sorted(loaded - bound)


@pytest.mark.parametrize("name", ["bench.py", "__graft_entry__.py"])
def test_every_loaded_name_is_bound(name):
    assert unbound_names(os.path.join(ROOT, name)) == []


def test_bench_line_keys_present():
    src = open(os.path.join(ROOT, "bench.py")).read()
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "h2d_bytes_per_step",
                "d2h_bytes_per_step", "gpu_launches", "roofline", "cpu_baseline", "clocks", "impl"):
        assert f'"{key}"' in src, key


def test_bench_constants():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert mod.UNIT == "trials/s" and "trials/s" in mod.METRIC
    assert mod.C3["N"] == 1024 and mod.C3["replicas"] == 1024 and mod.C3["steps"] == 200_000


def test_tts99_closed_form():
    """TTS99 = tau R99 with R99 = log(0.01) / log(1 - theta), theta the Jeffreys
    posterior mean (y + 1/2) / (r + 1), at least one run."""
    import math
    import numpy as np
    import bench
    E = np.array([-10.0, -10.0, -9.0, -8.0, -10.0 + 1e-9])       # 3 hits within the tolerance
    t = bench.tts99(E, tau_run=2.0)
    theta = 3.5 / 6.0
    assert t["hits"] == 3 and t["runs"] == 5 and abs(t["theta"] - theta) < 1e-15
    assert abs(t["R99"] - math.log(0.01) / math.log(1 - theta)) < 1e-12
    assert abs(t["tts99_s"] - 2.0 * t["R99"]) < 1e-12
    # every run a hit: theta = (r + 1/2) / (r + 1) > 0.99 for r >= 50, R99 clamps to one run
    t = bench.tts99(np.full(100, -3.0), tau_run=0.5)
    assert t["R99"] == 1.0 and t["tts99_s"] == 0.5


def test_recorded_step_counts_match_the_kernel_source():
    """The instruction count and DRAM traffic bench.py reports for the step kernel come from an ncu
    capture of one kernel source; a change to that source must come with a new capture (this
    test fails until the recorded hash is updated with the new counts)."""
    import bench
    assert bench.step_source_sha() == bench.STEP_TRAFFIC["source_sha256_16"], (
        "the step kernel changed since its ncu counts were recorded: capture it again and update "
        "STEP_INST_PER_REPLICA_STEP and STEP_TRAFFIC")
