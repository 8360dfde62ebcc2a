"""The paper-scale timestep (150M particles, the size the paper renders per timestep) at full size:
properties that hold at any size (node invariants of the octree paragraph; a full-depth LOD frame equal
to the brute-force frame, bit for bit) and the brute-force image checked pixel by pixel against the
oracle's direct sum over all 150M particles at a fixed sample of pixels."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

N_MAX = 16000


@pytest.fixture(scope="module")
def scene():
    from paper_0811_2055_gb300 import gblod
    torch.cuda.set_device(0)
    p = synth.paper_scale()
    d = to_dev(p.xyz, p.mass, p.h)
    t = gblod.build_lod(*d, n_max=N_MAX, seed=1)
    yield gblod, p, d, t
    t.free()


def test_octree_invariants_at_full_size(scene):
    G, p, d, t = scene
    info = t.info()
    assert info.n_particles == p.n
    ex = t.export()
    nodes = ex["nodes"]
    internal = (nodes["flags"] & G.NODE_INTERNAL) != 0
    assert np.all(nodes["point_count"] <= N_MAX)
    assert np.all(nodes["point_count"][internal] == N_MAX)
    assert np.all(nodes["point_count"][~internal] == nodes["seg_count"][~internal])
    # children partition their parent's particles and carry its exact mass
    mass = [int(hi) << 64 | int(lo) for lo, hi in zip(nodes["mass_lo"], nodes["mass_hi"])]
    for i in np.nonzero(internal)[0]:
        c0, cn = int(nodes[i]["child_first"]), int(nodes[i]["child_count"])
        assert int(nodes["seg_count"][c0:c0 + cn].sum()) == int(nodes[i]["seg_count"])
        assert sum(mass[c0:c0 + cn]) == mass[i]
    # every particle sits in exactly one leaf, stored verbatim
    leaves = ~internal
    assert int(nodes["seg_count"][leaves].sum()) == p.n
    assert mass[0] == int(round(float(p.mass.astype(np.float64).sum()) * 2 ** 47))


def test_full_depth_lod_equals_bruteforce_at_full_size(scene):
    G, p, d, t = scene
    nodes = t.export()["nodes"]
    assert not np.any(nodes["flags"] & G.NODE_LOSSY)  # no depth-21 node holds more than n_max particles
    r = G.Renderer()
    cam = synth.paper_view(3)
    _, a = r.render(t, cam, G.make_params(lambda_px=0.0))
    _, b = r.render_bruteforce(*d, cam, G.make_params())
    assert r.status() == G.OK
    assert torch.equal(a, b) and int(G.u64(a).max()) > 0
    r.close()


def test_bruteforce_pixels_match_the_oracle_sum_at_full_size(scene):
    G, p, d, t = scene
    r = G.Renderer()
    cam = synth.paper_view(3)
    _, acc = r.render_bruteforce(*d, cam, G.make_params())
    img = G.u64(acc)
    pts4 = np.empty((p.n, 4), np.float32)
    pts4[:, :3] = p.xyz
    pts4[:, 3] = p.mass
    rp = O.rparams(lambda_px=0.0)
    for px, py in [(960, 540), (955, 536), (1010, 580), (700, 540), (1300, 300), (40, 1060)]:
        assert img[py, px] == O.pixel_value(pts4, p.h, cam, rp, px, py), (px, py)
    assert img[540, 960] > 0
    r.close()
