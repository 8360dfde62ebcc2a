"""Fitted representatives written back into the octree (abstract: an LOD image indistinguishable
from a full rendering), through the C ABI: node points and member ids read back exactly; points
written into several nodes (values generated on the host) give a node table, stored points and LOD
frames equal to the oracle's tree after the same write, bit for bit; and fitting a node's
representatives to its particles' images by the adjoint splat raises the LOD frame's PSNR against
the all-particle frame."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

from gpu_helpers import compare_trees, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    from paper_0811_2055_gb300 import gblod
    torch.cuda.set_device(0)
    p = synth.tiny(120000, seed=71)
    d = to_dev(p.xyz, p.mass, p.h)
    return gblod, p, d


def test_written_points_match_the_oracle(scene):
    G, p, d = scene
    t = G.build_lod(*d, n_max=1000, seed=1)
    T = O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=1000)
    nodes = t.export_nodes()
    internal = np.nonzero(nodes["flags"] & G.NODE_INTERNAL)[0]
    leaves = np.nonzero(~(nodes["flags"] & G.NODE_INTERNAL).astype(bool))[0]
    rng = np.random.default_rng(3)
    for node in [int(internal[0]), int(internal[len(internal) // 2]), int(leaves[3]), int(leaves[-1])]:
        p4, hs = t.node_points(node)
        ids = t.node_members(node).cpu().numpy()
        nd = T.nodes[node]
        pf, n = int(nd["point_first"]), int(nd["point_count"])
        assert np.array_equal(p4.cpu().numpy(), T.pts4[pf:pf + n]) and np.array_equal(hs.cpu().numpy(), T.hs[pf:pf + n])
        sf = int(nd["seg_first"])
        assert np.array_equal(ids, T.sidx[sf:sf + int(nd["seg_count"])])
        new = T.pts4[pf:pf + n].copy()
        new[:, :3] += rng.normal(0, 0.03, (n, 3)).astype(np.float32)
        new[:, 3] *= rng.uniform(0.6, 1.4, n).astype(np.float32)
        nh = (T.hs[pf:pf + n] * rng.uniform(0.7, 2.0, n)).astype(np.float32)
        t.set_points(node, torch.from_numpy(new).cuda(), torch.from_numpy(nh).cuda())
        T.set_points(node, new, nh)
    compare_trees(t.export(), T)
    r = G.Renderer()
    for cam in (synth.look_at((0.5, 0.5, -0.8), (0.5, 0.5, 0.5), width=320, height=240),
                synth.look_at((0.1, 0.9, 0.2), (0.5, 0.45, 0.5), width=256, height=200)):
        for lam in (4.0, 30.0):
            _, acc = r.render(t, cam, G.make_params(lambda_px=lam))
            want, st, _, _ = O.render_lod(T, cam, O.rparams(lambda_px=lam))
            assert st == 0 and np.array_equal(G.u64(acc), want)
    with pytest.raises(G.GblodError):
        t.set_points(0, torch.zeros((3, 4), device="cuda"), torch.zeros(3, device="cuda"))
    r.close()
    t.free()


def test_fitting_a_node_brings_its_image_closer_to_its_particles(scene):
    from paper_0811_2055_gb300 import fit
    G, p, d = scene
    t = G.build_lod(*d, n_max=2000, seed=1)
    nodes = t.export_nodes()
    # the internal node with the most particles below the root: its 2,000 points stand for many
    internal = [i for i in np.nonzero(nodes["flags"] & G.NODE_INTERNAL)[0] if nodes[i]["depth"] >= 1]
    node = int(max(internal, key=lambda i: int(nodes[i]["seg_count"])))
    lam = 24.0
    cams = fit.node_views(t, node, lam, n_views=8, size=128)
    test_cams = fit.node_views(t, node, lam, n_views=5, size=128, margin=1.4)
    r = G.Renderer()
    par = G.make_params(lambda_px=lam)
    for cam in test_cams:  # the views draw this node, not its children
        r.render(t, cam, par)
        assert node in set(r.last_selection().tolist())
    ids = t.node_members(node).long()
    sub = [x[ids].contiguous() for x in d]
    full = [G.u64(r.render_bruteforce(*sub, cam, par)[1]).astype(np.float64) for cam in test_cams]

    def error():
        """relative L2 difference of the exact integer images: the node's points vs its particles"""
        p4, hs = t.node_points(node)
        num = den = 0.0
        for cam, f in zip(test_cams, full):
            a = G.u64(r.render_bruteforce(p4[:, :3].contiguous(), p4[:, 3].contiguous(), hs, cam, par)[1])
            num += float(((a.astype(np.float64) - f) ** 2).sum())
            den += float((f ** 2).sum())
        return math.sqrt(num / den)

    before = error()
    res = fit.fit_node(t, node, *d, cams, steps=80, renderer=r)
    after = error()
    assert res["loss_last"] < 0.7 * res["loss_first"], res
    assert after < 0.8 * before, (before, after)
    # the written points are the fitted ones and the octree still draws the node in these views
    p4, hs = t.node_points(node)
    assert torch.equal(p4, res["pts4"]) and torch.equal(hs, res["hs"])
    for cam in test_cams:
        r.render(t, cam, par)
        assert node in set(r.last_selection().tolist())
    assert r.status() == G.OK
    r.close()
    t.free()
