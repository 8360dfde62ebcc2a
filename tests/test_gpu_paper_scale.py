"""The paper-scale timestep (150M particles, the size the paper renders per timestep) at full size:
the device octree equals the oracle's (every node field, the sorted keys and permutation, every
representative and stored point, bit for bit); the default-detail frames of the whole-box view and of
the next view in equal the oracle's frames (selection, 64-bit image, 8-bit image within 1), also when
the frame is split into record-budget passes; properties that hold at any size (node invariants of
the octree paragraph; a full-depth LOD frame equal to the brute-force frame, bit for bit); and the
brute-force image checked pixel by pixel against the oracle's direct sum over all 150M particles at a
fixed sample of pixels."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

from gpu_helpers import compare_trees, to_dev

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


@pytest.fixture(scope="module")
def oracle_tree(scene):
    G, p, d, t = scene
    O.set_threads(0)
    return O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=N_MAX)


def test_octree_equals_the_oracle_at_full_size(scene, oracle_tree):
    G, p, d, t = scene
    compare_trees(t.export(), oracle_tree)


@pytest.mark.parametrize("view", [7, 6])
def test_default_detail_frames_equal_the_oracle_at_full_size(scene, oracle_tree, view):
    G, p, d, t = scene
    cam = synth.paper_view(view)
    lam = float(np.sqrt(N_MAX))
    r = G.Renderer()
    img, acc = r.render(t, cam, G.make_params(lambda_px=lam))
    assert r.status() == G.OK
    sel = r.last_selection()
    rp = O.rparams(lambda_px=lam)
    want, st, nd, npts = O.render_lod(oracle_tree, cam, rp)
    assert st == 0 and nd > 1_000_000
    assert np.array_equal(sel, O.select(oracle_tree, cam, rp))
    assert np.array_equal(G.u64(acc), want)
    assert int(np.abs(img.cpu().numpy().astype(np.int32) - O.tonemap(want, rp).astype(np.int32)).max()) <= 1
    # the same frame split into passes whose (tile, splat) records fit a small record budget
    img2, acc2 = r.render(t, cam, G.make_params(lambda_px=lam, record_budget=1 << 23))
    assert r.status() == G.OK
    assert torch.equal(acc2, acc) and torch.equal(img2, img)
    r.close()


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
