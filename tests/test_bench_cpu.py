"""bench.py's reading of the committed ncu summaries (the `traffic` of its roofline object):
every persistent-kernel summary carries a source digest, the DRAM traffic of the captured
launch and its algorithmic bytes, and the traffic is within a few percent of the algorithmic
bytes (no re-reads)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.mark.parametrize("precision", ["fp64", "double_float"])
def test_profile_summary_fields(precision, monkeypatch):
    path = bench.PROFILE_SUMMARY[precision]
    assert os.path.exists(path)
    txt = open(path).read()
    digest = next(l.split("`")[1] for l in txt.splitlines() if l.strip().startswith("- csrc_sha256"))
    monkeypatch.setattr(bench, "csrc_digest", lambda: digest)  # read the fields whatever the sources
    traffic, alg = bench.profiled_traffic(precision)
    assert traffic is not None and alg is not None
    assert 0.95 <= traffic / alg <= 1.05


def test_profile_summary_stale_digest_gives_none(monkeypatch):
    monkeypatch.setattr(bench, "csrc_digest", lambda: "0000000000000000")
    assert bench.profiled_traffic("fp64") == (None, None)
