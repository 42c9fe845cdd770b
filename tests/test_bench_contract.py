"""The JSON line of `bench.py --impl reference` (the CPU oracle on its bounded
sample), run end to end on the host: one line, the benchmark's metric, unit
and workload, the oracle described as the CPU baseline, and an end-to-end
figure with no host/device copies."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    env.pop("WORLD_SIZE", None)
    env.pop("RANK", None)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("SDIRK2 step throughput at fixed Newton tolerance (DOF-steps/s)")
    assert "TGV 16^3 hexes P=3" in d["metric"]
    assert d["unit"] == "DOF*step/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == "tgv16^3_P3_Q6_sdirk2_dt10xexplicit"
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # value x time per step = the sample's DOF (3^3 elements of 5 x 64 modes)
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - 27 * 5 * 64) < 1e-6 * 27 * 5 * 64
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert isinstance(cb["cores"], int) and cb["cores"] >= 1 and "3^3" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
