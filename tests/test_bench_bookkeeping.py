"""The benchmark's per-launch DRAM traffic figures are tied to a digest of the
kernel sources they were captured from: a figure is reported only while those
sources are unchanged, and as None once they differ (no GPU needed)."""
import re

import bench


def test_source_digest_is_stable_and_short():
    for group in bench.TRAFFIC_SOURCES:
        d = bench.source_digest(group)
        assert re.fullmatch(r"[0-9a-f]{12}", d), (group, d)
        assert bench.source_digest(group) == d


def test_traffic_is_reported_only_for_matching_sources(monkeypatch):
    group = "ae_decode"
    digest = bench.source_digest(group)
    monkeypatch.setitem(bench.TRAFFIC, group, (123456, digest))
    assert bench.current_traffic(group) == 123456
    stale = "0" * 12 if digest != "0" * 12 else "1" * 12
    monkeypatch.setitem(bench.TRAFFIC, group, (123456, stale))
    assert bench.current_traffic(group) is None
    monkeypatch.delitem(bench.TRAFFIC, group)
    assert bench.current_traffic(group) is None


def test_every_recorded_group_names_its_sources():
    assert set(bench.TRAFFIC) <= set(bench.TRAFFIC_SOURCES)
    for group, (nbytes, digest) in bench.TRAFFIC.items():
        assert nbytes > 0 and re.fullmatch(r"[0-9a-f]{12}", digest), group
