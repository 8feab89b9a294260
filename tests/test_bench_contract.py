"""The benchmark's reference arm (the oracle on the host cores) keeps the
one-JSON-line contract, and a non-zero rank of a multi-rank launch prints
nothing (CPU only)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--num-lps", "300", "--cpu-sample", "100", *args],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    return r.stdout


def test_reference_arm_prints_one_json_line():
    out = [l for l in _run().splitlines() if l.strip()]
    assert len(out) == 1
    d = json.loads(out[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "LPs/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "dense50x50_phase1_100k" and d["config"]["num_lps_per_gpu"] == 300
    # the same config object as the GPU arm's line (bench.bench_config of the same batch)
    sys.path.insert(0, ROOT)
    import bench
    from paper_1802_08557_gb300 import workloads as W
    assert d["config"] == bench.bench_config("dense50x50_phase1_100k", W.mixed_sign_dense(300, 50, 50))
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "LPs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    out = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.strip() == ""
