"""The reference arm's JSON line on CPU: `bench.py --impl reference` times the
FP64 oracle on a small row sample and prints one line with the keys and types
of the bench contract (the GPU arm's line is checked on the GPU by running it)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--workload", "power_fp32_4096x256", "--cpu-rows", "1024"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and "unavailable" not in j
    for key, typ in [("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                     ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                     ("dtype", str), ("data", str), ("config", dict), ("cpu_baseline", dict), ("e2e", dict)]:
        assert isinstance(j[key], typ), key
    assert j["vs_baseline"] is None
    assert (j["n_gpus"], j["steps"], j["warmup"]) == (1, 2, 1)
    assert j["value"] > 0 and j["ms_per_step"] > 0
    assert j["config"]["workload"] == "power_fp32_4096x256"
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["unit"] == j["unit"]
    assert cb["cores"] >= 1 and "1024-row" in cb["sample"]
    assert j["e2e"] == {"value": j["value"], "unit": j["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_pass_labels_of_the_power_workloads():
    sys.path.insert(0, ROOT)
    import bench
    main = bench.pass_labels("bf16", 1000000 * 4096 * 2)
    assert main == {"prime_precision": "bf16 (fast)", "finalize_precision": "bf16x3 (split)",
                    "kernel": "fused single-read X-pass (xpass_fused_kernel + zreduce + split_v), algorithmic "
                              "bytes n*d*2 per pass",
                    "l2": "inputs (8.2 GB) larger than L2, no flush"}
    small = bench.pass_labels("f32", 4096 * 256 * 4)          # 4.2 MB: L2-resident
    assert small["prime_precision"] == "3xtf32 (fast)" and "xv_f32_kernel" in small["kernel"]
    assert small["l2"].startswith("inputs (4.2 MB) fit in L2") and "not meaningful" in small["l2"]
    assert bench.pass_labels("f32", 100000 * 1024 * 4)["l2"] == "inputs (0.4 GB) larger than L2, no flush"


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "power_fp32_4096x256", "--cpu-rows", "512"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_probe_and_batch_options_parse():
    """The profiler probe and the batch switches parse, and the default run uses neither."""
    sys.path.insert(0, ROOT)
    import bench
    a = bench.parse_args(["--probe", "projected_gram", "--rows", "131072", "--steps", "5"])
    assert a.probe == "projected_gram" and a.rows == 131072 and a.steps == 5
    d = bench.parse_args([])
    assert d.probe is None and not d.batch_no_lockstep and d.batch_priming == "bf16"
    assert bench.parse_args(["--batch-no-lockstep"]).batch_no_lockstep
