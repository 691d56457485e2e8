"""Host-side checks of bench.py's output contract (no GPU).

* The reference arm (`--impl reference`, the FP64 oracle on the host cores) prints one JSON
  line with the keys the benchmark contract names, on the same metric and workload as the
  GPU arm.
* A recorded ncu DRAM-traffic figure is reported only for the kernel variant and source
  files it was captured on.
"""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.strip().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["metric"] == "heat3d_256_fp64_mcell_updates_per_s" and d["unit"] == "Mcell-updates/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0
    assert d["config"]["workload"].startswith("heat3d_r3_256^3_fp64")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_traffic_record_is_tied_to_variant_and_sources():
    b = _bench_module()
    for case in b.NCU_TRAFFIC:
        recs = b._traffic_records(case)
        keys = {(r["variant"], r["zmode"]) for r in recs}
        assert len(keys) == len(recs), case  # one record per variant and z-chunk mode
        for rec in recs:
            # sources unchanged since the capture
            assert b._traffic(case, rec["variant"], rec["zmode"]) == rec["bytes"], (case, rec["variant"])
            assert b._traffic(case, rec["variant"] + "_other", rec["zmode"]) is None
            if (rec["variant"], rec["zmode"] + 1) not in keys:
                assert b._traffic(case, rec["variant"], rec["zmode"] + 1) is None  # another z-chunk length
    assert b._traffic("no_such_case", "x") is None


def test_weak_scaling_value_counts_all_ranks():
    b = _bench_module()
    # units per rank x ranks / seconds, in millions
    assert abs(b.weak_scaling_value(4, 1e6, 0.5) - 8.0) < 1e-12
