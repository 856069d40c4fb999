"""The committed DRAM-traffic records (``profiles/traffic.json``) that ``bench.py`` reports
as ``roofline.traffic``: every entry must name a known workload and stage, carry the
hash of the kernel sources it was captured on (a record of an older kernel would be
ignored by the bench and only mislead a reader, so it is removed instead), and hold a
positive per-launch byte count with the capture it came from."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_traffic_records_match_the_kernel_sources():
    import bench
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    assert d, "no traffic records"
    for workload, stages in d.items():
        assert workload in bench.WORKLOADS, workload
        for stage, e in stages.items():
            assert stage in bench.KERNEL_SOURCES, (workload, stage)
            assert e["source_sha"] == bench.source_hash(stage, workload), (
                f"{workload}/{stage}: captured on other kernel sources; capture it again or "
                "remove the record")
            assert isinstance(e["dram_bytes_per_launch"], int) and e["dram_bytes_per_launch"] > 0
            assert e["how"] and e["kernel"]
            assert bench.captured_traffic(stage, workload) == e["dram_bytes_per_launch"]


def test_profile_summaries_are_text_with_their_command():
    pdir = os.path.join(ROOT, "profiles")
    for name in os.listdir(pdir):
        p = os.path.join(pdir, name)
        assert name.endswith((".md", ".txt", ".json")), name   # nothing that runs
        assert os.path.getsize(p) < 16 * 1024, name             # short summaries only
        if name.endswith(".md"):
            text = open(p).read()
            assert "ncu " in text and "--clock-control none" in text, name
