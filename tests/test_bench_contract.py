"""The bench's JSON line (the measurement contract) on the CPU: the reference
arm (the oracle timed on the host cores) on a small workload prints one line
with the keys the contract names, and the argument defaults select the
documented configurations."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "20000",
         "--queries", "512", "--filters", "10", "--leaf-cap", "1000", "--steps", "1",
         "--warmup", "3", "--cpu-sample", "8"],
        cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_argument_defaults():
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    try:
        for cfg, (n, wave) in {"batched": (1_000_000, 64), "precision": (10_000_000, 4096),
                               "mixed": (25_000_000, 65536), "serving": (50_000_000, 16384),
                               "ablation": (1_000_000, 64)}.items():
            sys.argv = ["bench.py", "--config", cfg]
            a = bench.parse()
            assert (a.n, a.wave, a.gpus, a.warmup >= 3) == (n, wave, 1, True), cfg
    finally:
        sys.argv = old
