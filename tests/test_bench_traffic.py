"""The benchmark's guard on the captured splat traffic (CPU only): the hashed text is the binning rule
followed by the splat kernel, found in the current source, and the captured bytes are reported only
while that text is the captured one (scaled to a run by its records)."""
import hashlib
import os
from types import SimpleNamespace

import bench

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0811_2055_gb300", "csrc",
                   "render.cu")


def test_hashed_text_is_the_binning_rule_and_the_splat_kernel():
    src = open(SRC, "rb").read()
    t = bench.splat_source(src)
    assert t.startswith(b"constexpr int DIRECT_BOX")
    assert b"bool direct_box(" in t and b"struct SplatSmem {" in t and b"k_splat_tiles(" in t
    assert t.endswith(b"}\n") and t.count(b"k_splat_tiles(") == 1
    # both parts are taken whole: the rule ends before the splat kernel starts
    assert t.index(b"bool direct_box(") < t.index(b"struct SplatSmem {")


def test_traffic_is_reported_only_for_the_captured_text_and_scaled_by_records(monkeypatch):
    src = open(SRC, "rb").read()
    a = SimpleNamespace(workload="mid", particles=0)
    counts = {"pairs": 3_000, "pairs_captured": 100}
    captured = bench.SPLAT_CAPTURE["dram_read_bytes"] + bench.SPLAT_CAPTURE["dram_write_bytes"]
    cur = hashlib.sha256(bench.splat_source(src)).hexdigest()
    monkeypatch.setitem(bench.SPLAT_CAPTURE, "source_sha256", cur)
    assert abs(bench.splat_traffic(a, counts, 20) - captured * 1.5) < 1e-6 * captured
    assert bench.splat_traffic(SimpleNamespace(workload="paper", particles=0), counts, 20) is None
    assert bench.splat_traffic(a, dict(counts, pairs_captured=0), 20) is None
    monkeypatch.setitem(bench.SPLAT_CAPTURE, "source_sha256", "0" * 64)
    assert bench.splat_traffic(a, counts, 20) is None
