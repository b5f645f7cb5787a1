"""bench.py's measurement contract, checked on the CPU.

* The reference arm (the FP64 oracle timed on a bounded sample of the large
  workload) prints one JSON line with the keys the contract names.
* The committed DRAM-traffic figure is reported only for the kernel source it
  was captured on.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e")


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--cpu-sample", "2000"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    d = json.loads(lines[0])
    for k in KEYS:
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is False and d["unit"] == "ms" and d["value"] > 0
    assert d["vs_baseline"] is None
    assert "workload" in d["config"]
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == d["value"] and cpu["cores"] >= 1
    assert "2000" in cpu["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_traffic_figure_is_tied_to_the_kernel_source():
    sys.path.insert(0, ROOT)
    import bench

    with open(os.path.join(ROOT, "profiles", "dual_eval_large_traffic.json")) as f:
        rec = json.load(f)
    t = bench.ncu_traffic()
    if rec["kernel_hash"] == bench.kernel_hash():
        assert t == rec["dram_bytes_per_launch"]
        # one launch streams n (4m + 9) = 1.37 GB; re-reads would show up here
        assert 1.0 <= t / 1.37e9 < 1.05
    else:
        assert t is None


def test_every_mode_of_main_is_defined():
    """main() dispatches to one function per mode (--sweep, --profile, the
    reference arm, the sharded and the single-GPU runs); each must exist."""
    sys.path.insert(0, ROOT)
    import ast
    import bench

    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    main = next(n for n in tree.body if isinstance(n, ast.FunctionDef) and n.name == "main")
    called = {c.func.id for c in ast.walk(main)
              if isinstance(c, ast.Call) and isinstance(c.func, ast.Name) and c.func.id.startswith("run_")}
    assert {"run_sweep", "run_profile", "run_reference", "run_sharded", "run_gpu"} <= called
    for name in called:
        assert callable(getattr(bench, name, None)), name
