"""bench.py's host-side bookkeeping (CPU): the sources each measured
kernel's DRAM record is tied to, and the record lookup."""
import json
import os

import bench


def test_kernel_sources_exist_and_cover_the_includes():
    csrc = os.path.join(bench.ROOT, "paper_2002_11529_gb300", "csrc")
    for kernel, files in bench.KERNEL_SOURCES.items():
        paths = [os.path.normpath(os.path.join(csrc, f)) for f in files]
        assert all(os.path.exists(p) for p in paths), kernel
        # every local header that a listed file includes is listed too
        names = {os.path.basename(p) for p in paths}
        for p in paths:
            for line in open(p):
                if line.startswith("#include \""):
                    inc = os.path.basename(line.split('"')[1])
                    assert inc in names, (kernel, p, inc)


def test_digest_is_per_kernel():
    d0 = bench.source_digest("ut_decode")
    assert d0 == bench.source_digest("ut_decode") and d0 != bench.source_digest("compass_find")


def test_traffic_record_lookup(tmp_path, monkeypatch):
    """A record counts only for its kernel's current sources."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"ut_decode|plain": {"dram_bytes_per_launch": 123, "source_sha256": "current"},
           "compass_find|plain": {"dram_bytes_per_launch": 456, "source_sha256": "stale"}}
    (prof / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_digest", lambda kernel: "current")
    assert bench.measured_traffic("ut_decode", "plain") == 123
    assert bench.measured_traffic("compass_find", "plain") is None    # taken on other sources
    assert bench.measured_traffic("ut_run_batched", "plain") is None  # no record
    assert bench.measured_traffic("unknown_kernel", "plain") is None
