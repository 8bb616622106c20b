"""bench.py's reference arm (the oracle, one full-size user step timed over
worker processes, one pole solve per task; two workers here to bound memory)
prints the contract's JSON line."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-workers", "2"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 0
    assert d["unit"] == "REXI steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1000.0 / d["value"]) < 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "REXI steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "2d_wells_512x512_K32_dt0.5"


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_roofline_picks_the_nearer_roof_per_arithmetic():
    # double-float path: HBM against the FP32 pipe (kernel-counted FP32-pipe
    # instructions); FP64 path: HBM against the FP64 unit; mixed: HBM
    import argparse
    b = _bench_module()
    ms = 1.0
    for prec, flops, ops32, want in (("df64", 1.6e7, 4.0e9, "hbm"), ("df64", 1.6e7, 4.0e10, "alu"),
                                     ("fp64", 3.0e8, 0.0, "hbm"), ("fp64", 1.0e9, 0.0, "alu"),
                                     ("mixed", 1.0e9, 0.0, "hbm")):
        args = argparse.Namespace(precision=prec, ortho="lanczos", window=0)
        r = b.roofline(args, 2000.0, 6784.5, "measured", None, 2.0e9, 4.6e11, flops, ms, 2, ops32)
        assert r["bound"] == want, (prec, r["bound"])
        assert r["other"]["bound"] == ("alu" if want == "hbm" else "hbm")
        alu = r if r["bound"] == "alu" else r["other"]
        if prec == "df64":
            assert alu["unit"] == "TOP/s" and alu["peak"] == b.NOMINAL_FP32_TOPS
            assert abs(alu["achieved"] - ops32 / (ms * 1e-3) / 1e12) < 1e-9 * alu["achieved"]
        else:
            assert alu["unit"] == "TFLOP/s" and alu["peak"] == b.NOMINAL_FP64_TFLOPS
        for d in (r, r["other"]):
            assert abs(d["frac"] - d["achieved"] / d["peak"]) < 1e-12


def test_traffic_record_lookup(tmp_path, monkeypatch):
    # a record applies only to its source hash, workload and path; both the
    # list form and the single-record form are read
    b = _bench_module()
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    rec = {"engine_cu_sha256": "abc", "workload": b.WORKLOAD, "path": "df64|lanczos", "dram_bytes_per_launch": 5.0}
    (tmp_path / "profiles" / "lanczos_traffic.json").write_text(json.dumps({"records": [rec]}))
    assert b.engine_traffic("abc", "df64|lanczos") == 5.0
    assert b.engine_traffic("abd", "df64|lanczos") is None
    assert b.engine_traffic("abc", "fp64|lanczos") is None
    rec2 = dict(rec, path="fp64|window=2", dram_bytes_per_launch=7.0)
    (tmp_path / "profiles" / "engine_traffic.json").write_text(json.dumps(rec2))
    assert b.engine_traffic("abc", "fp64|window=2") == 7.0
