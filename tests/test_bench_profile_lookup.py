"""bench.py reads a kernel's DRAM traffic and utilisation from its ncu summary
only while the kernel's sources still hash to the value recorded there (CPU)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SUMMARY = """# fake summary

| counter | value |
|---|---|
| smsp__issue_active (% of active) | 61.5 |
| gpu__dram_throughput (% of peak) | 21.0 |

traffic_bytes_per_launch: 123456789
kernel_sources: {srcs}
kernel_source_sha256: {sha}
"""


def _with_summary(tmp_path, monkeypatch, sha):
    srcs = bench.PROFILE_OF["pef"][1]
    md = tmp_path / "pef.md"
    md.write_text(SUMMARY.format(srcs=",".join(srcs), sha=sha))
    monkeypatch.setitem(bench.PROFILE_OF, "pef", (str(md), srcs))
    return srcs


def test_summary_used_while_sources_match(tmp_path, monkeypatch):
    srcs = bench.PROFILE_OF["pef"][1]
    _with_summary(tmp_path, monkeypatch, bench.kernel_source_sha256(srcs))
    assert bench.measured_traffic("pef") == 123456789
    lim = bench.measured_limiter("pef")
    assert lim["issue_active_pct"] == 61.5 and lim["dram_throughput_pct"] == 21.0


def test_summary_ignored_after_a_source_change(tmp_path, monkeypatch):
    _with_summary(tmp_path, monkeypatch, "0" * 64)
    assert bench.measured_traffic("pef") is None
    assert bench.measured_limiter("pef") is None


def test_missing_summary(tmp_path, monkeypatch):
    monkeypatch.setitem(bench.PROFILE_OF, "pef", (str(tmp_path / "absent.md"), ["k_pef.cu"]))
    assert bench.measured_traffic("pef") is None
