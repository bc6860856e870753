"""The bench's measurement records on the CPU: every DRAM-traffic entry the
bench can put in its roofline names a profile summary that exists, records
the same kernel-source digest and the same bytes per sample, and the
staleness check reports a missing or changed capture as `traffic: null`
instead of a number."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_name_their_profiles():
    assert set(bench.TRAFFIC_FOR.values()) <= set(bench.TRAFFIC)
    for key, rec in bench.TRAFFIC.items():
        path = os.path.join(ROOT, rec["capture"])
        assert os.path.isfile(path), (key, rec["capture"])
        text = open(path).read()
        # the summary states the digest of the sources it was captured on
        assert rec["source"] in text, (key, rec["source"])
        assert re.fullmatch(r"[0-9a-f]{16}", rec["source"])
        # and the bytes per sample the table holds (two decimals)
        assert "%.2f" % rec["bytes_per_sample"] in text or "%.1f" % rec["bytes_per_sample"] in text, key
        assert 0.0 < rec["bytes_per_sample"] < 200.0


def test_stale_capture_reports_null(monkeypatch):
    n = 1.0e9
    key = ("large_bf16", "march_bwd")
    rec = bench.TRAFFIC[bench.TRAFFIC_FOR[key]]
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: rec["source"])
    b, _, _, info = bench.traffic_for(key[0], key[1], n)
    assert b == rec["bytes_per_sample"] * n and info["capture"] == rec["capture"]
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "0" * 16)
    b, _, _, info = bench.traffic_for(key[0], key[1], n)
    assert b is None and info == {"capture": rec["capture"], "stale": True}
    # a workload without a capture has no traffic and no record
    assert bench.traffic_for("small", "march", n) == (None, None, None, None)
