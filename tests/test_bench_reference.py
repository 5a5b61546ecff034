"""The bench's reference arm (the CPU oracle timed on the host) on the small
chain: it runs without a GPU, prints one JSON line with the fields the bench
contract names, and its step estimate covers every op of the step."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line_on_chain10():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "chain10_chi256", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == "gate_applications_per_sec"
    assert line["unit"] == "gate-applications/s" and line["higher_is_better"] is True
    assert np.isfinite(line["value"]) and line["value"] > 0.0
    # value = ops per step / estimated step time (ms_per_step)
    import workloads as W
    from oracle import schedule
    n_ops = sum(len(layer) for layer in schedule.step_layers(10, W.chain_bonds(10)))
    assert abs(line["value"] - n_ops / (line["ms_per_step"] / 1e3)) <= 1e-9 * line["value"]
    assert f"one step of {n_ops} ops" in line["config"]["oracle"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
