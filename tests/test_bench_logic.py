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
    assert bench.traffic_for(*key[:3], bench.fd_form(4)) == (None, None)


def test_one_thread_oracle_sample():
    out = bench.oracle_sample_one_thread(2, 1, 2, 1, 1)
    assert out is not None
    seconds, iterations = out
    assert seconds > 0 and iterations > 0
