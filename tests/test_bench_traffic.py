"""The benchmark's bookkeeping on CPU: the guard on the captured splat traffic (the hashed text is
the binning rule followed by the splat kernel, and captured bytes are reported only while that text
is the captured one, scaled per record), and the reference arm's band cameras (a band of a frame is
exactly those rows of the full frame, so timing bands times frames)."""
import hashlib
import os

import numpy as np

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
    captured = bench.SPLAT_CAPTURE["dram_read_bytes"] + bench.SPLAT_CAPTURE["dram_write_bytes"]
    cur = hashlib.sha256(bench.splat_source(src)).hexdigest()
    monkeypatch.setitem(bench.SPLAT_CAPTURE, "source_sha256", cur)
    monkeypatch.setitem(bench.SPLAT_CAPTURE, "records", 1000)
    assert abs(bench.splat_traffic(2500.0) - captured * 2.5) < 1e-6 * captured
    assert bench.splat_traffic(0.0) is None
    monkeypatch.setitem(bench.SPLAT_CAPTURE, "records", 0)
    assert bench.splat_traffic(2500.0) is None
    monkeypatch.setitem(bench.SPLAT_CAPTURE, "records", 1000)
    monkeypatch.setitem(bench.SPLAT_CAPTURE, "source_sha256", "0" * 64)
    assert bench.splat_traffic(2500.0) is None


def test_band_cameras_draw_the_rows_of_the_full_frame():
    from oracle import oracle as O
    from paper_0811_2055_gb300 import synth
    p = synth.tiny(20000, seed=25)
    T = O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=400)
    cam = synth.look_at((0.5, 0.55, -0.5), (0.5, 0.5, 0.5), width=96, height=72)
    rp = O.rparams(lambda_px=10.0)
    full, st, nd, npts, nu = O.render_lod_counted(T, cam, rp)
    nb = 6
    bands = [O.render_lod_rows(T, cam, rp, *bench.band_rows(cam["height"], b, nb)) for b in range(nb)]
    assert full.sum() > 0 and st == 0
    assert np.array_equal(np.concatenate([b[0] for b in bands], 0), full)
    assert sum(b[4] for b in bands) == nu  # the bands' pixel updates add up to the frame's
