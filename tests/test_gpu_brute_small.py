"""All-particle frames of unordered particles through the partitioned binning, against the oracle
bit for bit: mostly tiny splats (the small-box record stream and its shared-memory tile images),
points stacked on one pixel, points on tile edges and image corners, large blobs centred off the
image with a small visible sliver, a frame split into record-budget passes, and a frame with more
tiles than the partitioned path takes (the ordered binning is used there)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

from gpu_helpers import to_dev, u8_close

pytestmark = pytest.mark.gpu


def _points(n=300000, seed=81):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
    h = np.full(n, 3e-4, np.float32)                       # sigma well below a pixel: tiny boxes
    h[: n // 10] = rng.uniform(0.002, 0.02, n // 10).astype(np.float32)  # some binned blobs
    xyz[n // 10: n // 10 + 2000] = (0.5, 0.5, 0.5)         # 2,000 points on one spot
    mass = rng.uniform(0.5, 2.0, n).astype(np.float32)
    return xyz, mass, h


@pytest.mark.parametrize("W,H,budget", [(1920, 1080, 0), (1920, 1080, 1 << 16), (640, 360, 0), (4000, 2000, 0)])
def test_unordered_all_particle_frames_equal_the_oracle(W, H, budget):
    from paper_0811_2055_gb300 import gblod
    torch.cuda.set_device(0)
    xyz, mass, h = _points()
    cam = synth.look_at((0.5, 0.5, -1.2), (0.5, 0.5, 0.5), width=W, height=H)
    # a few points exactly on tile edges and image corners
    F, D = cam["f_px"], 1.7
    for k, (u, v) in enumerate([(64.0, 16.0), (0.0, 0.0), (W - 1e-3, H - 1e-3), (128.0, 32.0)]):
        xyz[300 + k] = (0.5 - (u - cam["cx"]) * D / F, 0.5 - (v - cam["cy"]) * D / F, 0.5)
    # large blobs centred off the image: slivers along an edge, and blobs off a corner whose clipped
    # box is a few pixels square although its pixels lie hundreds of pixels from the centre (their
    # disc does not reach the image; a squared distance that wrapped in 32 bits would add spurious
    # contributions)
    for k, (u, v, sig) in enumerate([(-296.0, 300.0, 100.0), (W + 296.0, 200.0, 100.0), (500.0, -116.0, 40.0),
                                     (700.0, H + 116.0, 40.0), (-294.0, -294.0, 100.0), (W + 294.0, -294.0, 100.0),
                                     (-294.0, H + 294.0, 100.0), (W + 294.0, H + 294.0, 100.0)]):
        xyz[400 + k] = (0.5 - (u - cam["cx"]) * D / F, 0.5 - (v - cam["cy"]) * D / F, 0.5)
        h[400 + k] = sig * D / F
    r = gblod.Renderer()
    par = gblod.make_params(record_budget=budget)
    img, acc = r.render_bruteforce(*to_dev(xyz, mass, h), cam, par)
    assert r.status() == gblod.OK
    rp = O.rparams()
    want, st, nd = O.splat_particles(xyz, mass, h, cam, rp)
    assert st == 0 and nd > 200000
    assert np.array_equal(gblod.u64(acc), want)
    assert u8_close(img.cpu().numpy(), O.tonemap(want, rp)) <= 1
    # counted frame: the kernels' pixel updates equal the oracle's count
    r.render_bruteforce(*to_dev(xyz, mass, h), cam, gblod.make_params(record_budget=budget, count_updates=True))
    pts4 = np.concatenate([xyz, mass[:, None]], 1).astype(np.float32)
    assert r.stats()["pixel_updates"] == O.count_updates(pts4, h, cam, rp)
    r.close()
