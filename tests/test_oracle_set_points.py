"""Pins of the oracle's write-back of fitted points (orc_tree_set_points, CPU only): the written
points are stored; the node's and every ancestor's particle bounds and h_cull grow to cover them and
no other node changes; writing the node's own points back changes nothing drawn; and a point moved
into a view that culled its node before makes the node visible and drawn (culling stays
conservative)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0811_2055_gb300 import synth


def _tree():
    p = synth.tiny(30000, seed=61)
    return p, O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=500)


def _ancestors(T, i):
    out = []
    while i >= 0:
        out.append(i)
        i = int(T.nodes[i]["parent"])
    return out


def test_written_points_are_covered_by_the_bounds_of_the_node_and_its_ancestors():
    p, T = _tree()
    internal = np.nonzero(T.nodes["flags"] & O.INTERNAL)[0]
    node = int(internal[-1])
    nd = T.nodes[node]
    pf, n = int(nd["point_first"]), int(nd["point_count"])
    rng = np.random.default_rng(0)
    new = T.pts4[pf:pf + n].copy()
    new[:5, :3] += rng.normal(0, 0.2, (5, 3)).astype(np.float32)  # some far outside the cell
    new[:, 3] *= rng.uniform(0.5, 1.5, n).astype(np.float32)
    hs = T.hs[pf:pf + n] * np.float32(3.0)
    before = T.nodes.copy()
    T.set_points(node, new, hs)
    assert np.array_equal(T.pts4[pf:pf + n], new) and np.array_equal(T.hs[pf:pf + n], hs)
    assert np.all(T.pt_src[pf:pf + n] == 0xFFFFFFFF)
    path = set(_ancestors(T, node))
    for i in range(len(T.nodes)):
        a, b = T.nodes[i], before[i]
        if i in path:
            assert np.all(a["bmin"] <= new[:, :3].min(0)) and np.all(a["bmax"] >= new[:, :3].max(0))
            assert a["h_cull"] >= hs.max()
            assert np.all(a["bmin"] <= b["bmin"]) and np.all(a["bmax"] >= b["bmax"]) and a["h_cull"] >= b["h_cull"]
        else:
            assert a.tobytes() == b.tobytes(), i
    with pytest.raises(O.OracleError):
        T.set_points(node, new[:-1], hs[:-1])


def test_writing_the_same_points_changes_no_frame():
    p, T = _tree()
    cam = synth.look_at((0.5, 0.55, -0.7), (0.5, 0.5, 0.5), width=160, height=120)
    rp = O.rparams(lambda_px=10.0)
    a = O.render_lod(T, cam, rp)[0]
    for node in range(0, len(T.nodes), 7):
        nd = T.nodes[node]
        pf, n = int(nd["point_first"]), int(nd["point_count"])
        T.set_points(node, T.pts4[pf:pf + n].copy(), T.hs[pf:pf + n].copy())
    assert np.array_equal(O.render_lod(T, cam, rp)[0], a)


def test_a_point_moved_into_view_keeps_its_node_drawn():
    p, T = _tree()
    # a narrow view of the corner region near (0.02, 0.02, 0.02)
    cam = synth.look_at((0.02, 0.02, -0.3), (0.02, 0.02, 0.02), vfov_deg=4.0, width=64, height=64)
    rp = O.rparams(lambda_px=0.0)  # full depth: every visible leaf
    leaves = np.nonzero(~(T.nodes["flags"] & O.INTERNAL).astype(bool))[0]
    sel0 = set(O.select(T, cam, rp).tolist())
    far = [int(i) for i in leaves if int(i) not in sel0]
    node = far[-1]
    nd = T.nodes[node]
    pf, n = int(nd["point_first"]), int(nd["point_count"])
    new = T.pts4[pf:pf + n].copy()
    new[0, :3] = (0.02, 0.02, 0.02)
    before = O.render_lod(T, cam, rp)[0]
    T.set_points(node, new, T.hs[pf:pf + n].copy())
    assert node in set(O.select(T, cam, rp).tolist())
    after = O.render_lod(T, cam, rp)[0]
    single = O.splat_points(new[:1], T.hs[pf:pf + 1], cam, rp)[0]
    assert single.sum() > 0 and np.array_equal(after, before + single + O.splat_points(
        new[1:], T.hs[pf + 1:pf + n], cam, rp)[0])
