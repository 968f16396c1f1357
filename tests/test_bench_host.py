"""Host-side pieces of bench.py that need no GPU: the kernel-source hash
and the committed DRAM-traffic figure it validates."""
import bench


def test_source_hash_is_stable_and_short():
    h = bench.kernel_source_hash()
    assert h == bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0


def test_traffic_only_for_matching_sources(tmp_path, monkeypatch):
    f = tmp_path / "launches.md"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    f.write_text(f"# summary\n\ntraffic: source={bench.kernel_source_hash()} bytes_per_launch=12345\n")
    assert bench.committed_traffic() == 12345.0
    f.write_text("traffic: source=0000000000000000 bytes_per_launch=12345\n")  # another kernel version
    assert bench.committed_traffic() is None
    f.write_text("no traffic line\n")
    assert bench.committed_traffic() is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.md"))
    assert bench.committed_traffic() is None
