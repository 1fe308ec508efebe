"""bench.py's reference arm (the oracle on the host cores) runs without a
GPU and prints one JSON line with the keys of the measurement contract."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                        "--cpu-seconds", "0.3", "--nodes", "2"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600, env=dict(os.environ, OMP_NUM_THREADS="4"))
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]


def _load_bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_record_scales_by_subdomains_and_expires_with_the_sources(tmp_path, monkeypatch):
    """roofline.traffic: the committed ncu bytes per subdomain scaled to the
    launch, reported only while the kernel's sources hash to the profiled
    ones (a changed kernel reports null until it is profiled again)"""
    b = _load_bench()
    (tmp_path / "profiles").mkdir()
    rec = {"segmented": {"dram_bytes_per_subdomain": 1000.5, "kernel_sha256": "abc"}}
    (tmp_path / "profiles" / "bound_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "kernel_sha", lambda which: "abc")
    assert b.traffic_for(1 << 24, "segmented") == 1000.5 * (1 << 24)
    assert b.traffic_for(4, "segmented") == 4002.0
    assert b.traffic_for(1 << 24, "interpreter") is None
    monkeypatch.setattr(b, "kernel_sha", lambda which: "abd")
    assert b.traffic_for(1 << 24, "segmented") is None


def test_committed_traffic_records_name_existing_sources():
    """every committed record lists the sources its hash covers, and those
    are the files bench.py hashes for that kernel"""
    b = _load_bench()
    with open(os.path.join(ROOT, "profiles", "bound_traffic.json")) as fh:
        recs = json.load(fh)
    for which, rec in recs.items():
        assert which in b.KERNEL_SOURCES, which
        assert tuple(rec["sources"]) == tuple(b.KERNEL_SOURCES[which]), which
        for name in rec["sources"]:
            assert os.path.exists(os.path.join(ROOT, "paper_2507_20769_gb300", "csrc", name)), name
        assert rec["dram_bytes_per_subdomain"] > 0 and rec["subdomains"] > 0
        per = (rec["dram_bytes_read"] + rec["dram_bytes_write"]) / rec["subdomains"]
        assert abs(per - rec["dram_bytes_per_subdomain"]) <= 1e-9 * per


def test_roofline_fraction_is_algorithmic_endpoint_operations_over_the_fp64_peak(monkeypatch):
    """roofline.frac = endpoint operations per subdomain (the static counts) x
    subdomains of a step / step time / (2 FP64 lanes per clock per SM x SMs x
    the sampled SM clock); independent of how fast the primitives run"""
    import types
    import torch
    b = _load_bench()
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev: types.SimpleNamespace(multi_processor_count=152))
    monkeypatch.setattr(b, "traffic_for", lambda subs, which: None)
    counts = {"addsub": 14188, "mul": 31542, "div": 1844, "rcp": 2730, "sqrt": 1892, "exp": 1872, "log": 1724, "rn": 48}

    class FakeProblem:
        def op_counts(self):
            return dict(counts)

        def get_segmentation(self):
            return {"recomputed": 0}

        def get_tuning(self):
            return {"kernel": 2}

    subs, step_s = 1 << 24, 3.7
    rf = b.roofline_block(FakeProblem(), subs, step_s, {"sm_mhz": 2070.0}, 0)
    peak = 2.0 * 152 * 2070e6
    assert rf["bound"] == "alu" and rf["kernel"] == "segmented"
    assert rf["work_per_subdomain"]["endpoint_ops"] == 55840
    assert abs(rf["frac"] - 55840 * subs / step_s / peak) <= 1e-12
    assert abs(rf["achieved"] - 55840 * subs / step_s / 1e9) <= 1e-9 * rf["achieved"]
    assert abs(rf["peak"] - peak / 1e9) <= 1e-9
    rf2 = b.roofline_block(FakeProblem(), subs, step_s, {"sm_mhz": None}, 0)   # no clock sample: maximum clock
    assert abs(rf2["peak"] - peak / 1e9) <= 1e-9
