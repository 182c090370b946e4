"""The benchmark on the GPU (a short run): one JSON line with the keys of the benchmark
contract -- throughput, the dominant kernel's roofline, the oracle as CPU baseline, the
end-to-end figure with the bytes it copies, the clocks seen during the timed region and the
number of kernel launches."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--steps", "5", "--warmup", "3", "--no-plain", "--serve-kf", "0",
                        "--no-dense", "--no-forward", "--cpu-seconds", "0.2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout[-3000:]
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks",
              "gpu_launches"):
        assert k in d, k
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (5, 3, 1)
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["unit"] == "keyframes/s"
    assert "workload" in d["config"] and "model" not in d["config"]
    rf = d["roofline"]
    assert rf["bound"] in ("hbm", "tensor", "alu") and rf["unit"] in ("GB/s", "TFLOP/s")
    assert rf["achieved"] > 0 and rf["peak"] > 0 and rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert rf["traffic"] is None or rf["traffic"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["sample"]
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"] and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    c = d["clocks"]
    assert "sm_mhz" in c and "sm_max_mhz" in c and isinstance(c["reasons"], list)
    assert d["gpu_launches"] >= 5
    cf = d["configs"]
    for name in ("cfg0", "cfg1", "cfg3"):
        for form in ("batched", "plain"):
            r = cf[name][form]
            assert r["keyframes_per_s"] > 0 and r["p99_ms"] >= r["p50_ms"] > 0
            assert r["parity"] == "oracle, bit-exact"
        assert cf[name]["oracle_1_core"]["keyframes_per_s"] > 0
        assert cf[name]["oracle_all_cores"]["cores"] >= 1
    assert d["e2e"]["serial"]["value"] > 0 and d["e2e"]["serial"]["unit"] == d["unit"]
    assert d["e2e"]["one_thread"]["value"] > 0 and d["e2e"]["one_thread"]["unit"] == d["unit"]
