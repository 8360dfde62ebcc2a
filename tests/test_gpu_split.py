"""Split frame on one GPU, through the C ABI: the parts of a frame (gblod_render_part) sum to the
whole frame bit for bit, each part equals the oracle's part, and gblod_tonemap of the sum is the
frame's 8-bit image."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_parts_sum_to_the_frame_and_match_the_oracle():
    from oracle import oracle as O
    from paper_0811_2055_gb300 import gblod, split, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    p = synth.tiny(120000, seed=52)
    xyz, mass, h = (torch.from_numpy(a).to(dev) for a in (p.xyz, p.mass, p.h))
    tree = gblod.build_lod(xyz, mass, h, n_max=500, seed=1)
    T = O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=500)
    r = gblod.Renderer()
    for cam in (synth.look_at((0.45, 0.55, -0.6), (0.5, 0.5, 0.5), width=320, height=240),
                synth.look_at((0.5, 0.48, 0.45), (0.9, 0.5, 0.6), width=301, height=199, z_near=1e-3)):
        par = gblod.make_params(lambda_px=8.0)
        img, acc = r.render(tree, cam, par)
        rp = O.rparams(lambda_px=8.0)
        for n_parts in (2, 3):
            total = torch.zeros_like(acc)
            for k in range(n_parts):
                part = r.render_part(tree, cam, k, n_parts, par)
                want, st, _, _ = O.render_lod_part(T, cam, rp, k, n_parts)
                assert st == 0 and np.array_equal(gblod.u64(part), want), (n_parts, k)
                total += part
            assert torch.equal(total, acc)
            assert torch.equal(r.tonemap(total, par), img)
        # one rank: the host helper is the plain frame
        simg, sacc = split.render_split(r, tree, cam, par, 0, 1)
        assert torch.equal(sacc, acc) and torch.equal(simg, img)
    with pytest.raises(gblod.GblodError):
        r.render_part(tree, cam, 2, 2, par)
    r.close()
    tree.free()
