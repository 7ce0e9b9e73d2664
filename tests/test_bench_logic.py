"""Host logic of bench.py that needs no GPU: the DRAM-traffic figure is reported only while the
kernel source it was measured on is unchanged, and the one-thread oracle sample runs in a child
process."""
import hashlib
import os

import bench


def test_traffic_reported_only_for_the_measured_source(monkeypatch):
    key = ("mode_product", "fp64", "cavity32", "per-direction")
    entry = dict(bench.TRAFFIC[key])
    src = os.path.join(bench.ROOT, "paper_2311_06926_gb300", "csrc", entry["source"])
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    monkeypatch.setitem(bench.TRAFFIC, key, dict(entry, sha256=digest))
    traffic, profile = bench.traffic_for(*key)
    assert traffic == entry["bytes_per_launch"] and profile.startswith("profiles/")
    assert os.path.exists(os.path.join(bench.ROOT, profile))
    monkeypatch.setitem(bench.TRAFFIC, key, dict(entry, sha256="0" * 64))
    assert bench.traffic_for(*key) == (None, None)
    assert bench.traffic_for("band_pass", "fp64", "cavity32") == (None, None)
    assert bench.traffic_for(*key[:3], bench.fd_form(2)) == (None, None)   # no capture of that form


def test_one_thread_oracle_sample():
    out = bench.oracle_sample_one_thread(2, 1, 2, 1, 1)
    assert out is not None
    seconds, iterations = out
    assert seconds > 0 and iterations > 0


def test_class_rooflines():
    prof = {"mode_product": dict(launches=10, ms=2.0, flops=1.0e9, bytes=4.0e6),
            "vector": dict(launches=4, ms=1.0, flops=0.0, bytes=6.678e9),
            "line_solve": dict(launches=0, ms=0.0, flops=0.0, bytes=0.0)}
    out = bench.class_rooflines(prof, 4.0, "fp64", {"hbm_gbs": 6678.0})
    assert out["mode_product"]["bound"] == "fp64"
    assert abs(out["mode_product"]["achieved_tflops"] - 0.5) < 1e-9
    assert abs(out["mode_product"]["frac"] - 0.5 / bench.FP64_PEAK_TFLOPS) < 1e-4
    assert out["vector"]["bound"] == "hbm" and abs(out["vector"]["frac"] - 1.0) < 1e-6
    assert out["mode_product"]["share"] == 0.5 and "frac" not in out["line_solve"]
    # reduced precision: every class against HBM
    assert bench.class_rooflines(prof, 4.0, "tf32", {})["mode_product"]["bound"] == "hbm"
