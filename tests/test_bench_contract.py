"""The bench's reference arm (the oracle on the host, no GPU): one JSON line with the contract's keys,
labelled with the sample of the headline workload that actually ran."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "heat3d_q2_dg2_16cubed_jitter0.15_rho4blocks"
    assert d["config"]["sample_of"] == "heat3d_q2_dg2_32cubed_jitter0.15_rho4blocks"
    assert d["cpu_baseline"]["value_1_thread"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_traffic_records_match_the_current_sources_and_go_null_on_change(monkeypatch):
    """profiles/traffic.json holds the DRAM bytes of the ncu captures; a record counts only while the
    kernel's sources hash to the recorded value."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for key in ("asm_bf16", "apply_df32", "apply_fp32"):
        assert bench.read_traffic(key) is not None and bench.read_traffic(key) > 1e7, key
    monkeypatch.setattr(bench, "source_sha", lambda paths: "0" * 16)
    assert bench.read_traffic("asm_bf16") is None
