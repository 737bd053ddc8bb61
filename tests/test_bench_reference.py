"""`bench.py --impl reference` (the FP64 oracle on the host cores) prints one
JSON line with the keys of the benchmark contract: the same metric, unit and
workload as the GPU arm, the oracle's own cpu_baseline and a host-only e2e."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--no-cpu-baseline"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "cell-direction updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "channel_td_1024x1024_S16"
    assert d["config"]["nsteps"] == 100 and d["config"]["tol"] == 1e-8
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_clock_samples_are_matched_by_uuid():
    """nvidia-smi numbers GPUs physically while CUDA_VISIBLE_DEVICES renumbers
    them per process: the bench keeps the samples of its own GPU's UUID."""
    sys.path.insert(0, ROOT)
    import bench
    rows = ["GPU-aaaa, 0, 1200, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "GPU-bbbb, 3, 2070, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
            "GPU-bbbb, 3, 2050, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
            "GPU-aaaa, 0, 1210, 2070, 900.0, 0x0, Active, Not Active, Not Active, Not Active"]
    c = bench.parse_clock_samples(rows, uuid="bbbb")
    assert c["samples"] == 2 and c["sm_mhz"] == 2060.0 and c["reasons"] == ["sw_power_cap"]
    assert c["matched_by"] == "uuid"
    c = bench.parse_clock_samples(rows, index=0)
    assert c["samples"] == 2 and c["reasons"] == ["hw_slowdown"] and c["matched_by"] == "index"
    assert bench.parse_clock_samples(rows, uuid="cccc") is None


def test_sweep_traffic_table_is_one_capture():
    """bench.py imports, and its table of captured sweep traffic holds one
    entry per workload, all from one capture of one set of sources."""
    import bench
    t = bench.SWEEP_TRAFFIC
    assert set(t) == {"timedep_fp64", "channel", "batch"}
    assert len({d for d, _ in t.values()}) == 1
    assert all(isinstance(b, int) and b > 0 for _, b in t.values())
    assert len(bench.sweep_sources_digest()) == 16
