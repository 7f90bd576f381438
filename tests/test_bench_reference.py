"""bench.py --impl reference (the FP64 oracle on the host cores) prints one
JSON line with the contract's keys; CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "builds/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "builds/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "stored_n200_m16"


def test_traffic_record_matches_workload_and_source():
    """The DRAM traffic the bench reports comes from the committed ncu record
    of the same kernel, workload and precision, and only while the kernel's
    source is the one that was captured; the committed records are current."""
    sys.path.insert(0, ROOT)
    import bench
    recs = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    for kernel, rec in recs.items():
        workload, prec = rec["workload"].rsplit(" ", 1)
        assert bench.ncu_traffic(kernel, prec, workload) == rec["traffic_bytes_per_launch"], kernel
        assert bench.ncu_traffic(kernel, prec, "precision_n400_m64") is None
        assert bench.ncu_traffic(kernel, "bf16x2" if prec != "bf16x2" else "fp64", workload) is None
