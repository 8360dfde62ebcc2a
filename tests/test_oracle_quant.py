"""Pins of the oracle's 16-bit block codes (CPU only).

The paper stores each coordinate in 2 bytes spanning the block that holds the point, so that
deeper (smaller) blocks are more accurate and nothing is lost, and codes the other properties
the same way.  Pins below: hand-worked codes, the half-step error bound, the lossless decode
once the step is below half an fp32 spacing, decode -> encode round trips over every code,
linear codes of the weights and smoothing lengths, the decoded tree's bounds covering every
decoded point of each subtree, and a full-depth render of the quantised tree equal to the
brute-force splat of the decoded points.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "block16_hand.json")


def test_hand_worked_codes():
    d = json.load(open(GOLDEN))
    for e in d["position"]:
        x = np.float32(float(e["x"]))
        step = math.ldexp(1.0, e["qstep_log2"])
        c = O.block_code_pos([x], e["qlo"], step)[0]
        assert int(c) == e["code"], e
        dec = O.block_decode_pos([c], e["qlo"], step)[0]
        assert dec == np.float32(e["decoded"]), e


def _ulp(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


@pytest.mark.parametrize("depth", [0, 1, 3, 6, 9, 14, 21])
def test_half_step_error_bound(depth):
    rng = np.random.default_rng(depth)
    edge = math.ldexp(1.0, -depth)
    corner = math.floor(rng.uniform(0, 1) / edge) * edge
    x = (corner + rng.uniform(0, edge, 20000)).astype(np.float32)
    x = x[(x >= corner) & (x < corner + edge)]
    step = math.ldexp(edge, -16)
    c = O.block_code_pos(x, corner, step)
    xd = O.block_decode_pos(c, corner, step).astype(np.float64)
    err = np.abs(xd - x.astype(np.float64))
    bound = edge * 2.0 ** -17 + 0.5 * _ulp(xd)
    assert np.all(err <= bound), (depth, float(np.max(err / bound)))
    # decoded points stay in the block (the decode is the centre of a sub-cell)
    assert np.all(xd >= corner) and np.all(xd <= corner + edge)


@pytest.mark.parametrize("depth", [9, 12, 16, 21])
def test_lossless_when_step_is_below_half_an_ulp(depth):
    # in [1/2, 1) the fp32 spacing is 2^-24; the step edge 2^-16 = 2^-(depth+16) is at most
    # 2^-25 from depth 9 on, so the decoded value is the input itself
    rng = np.random.default_rng(100 + depth)
    edge = math.ldexp(1.0, -depth)
    corner = 0.5 + math.floor(rng.uniform(0, 0.5) / edge) * edge
    x = (corner + rng.uniform(0, edge, 5000)).astype(np.float32)
    x = x[(x >= corner) & (x < corner + edge)]
    step = math.ldexp(edge, -16)
    xd = O.block_decode_pos(O.block_code_pos(x, corner, step), corner, step)
    assert np.array_equal(xd, x)


@pytest.mark.parametrize("lo,step", [(0.0, 2.0 ** -16), (0.25, 2.0 ** -20), (0.703125, 2.0 ** -37),
                                     (-3.0, 2.0 ** -10)])
def test_every_position_code_round_trips(lo, step):
    c = np.arange(65536, dtype=np.uint16)
    xd = O.block_decode_pos(c, lo, step)
    c2 = O.block_code_pos(xd, lo, step)
    # a decoded value that fp32 rounding moved onto a neighbour's cell can only happen when the
    # sub-cell is finer than fp32; there several codes decode to one float and the code that
    # comes back decodes to the same float
    same = c2 == c
    assert np.array_equal(O.block_decode_pos(c2, lo, step), xd)
    if step * 2 >= np.spacing(np.float32(abs(lo) + 65536 * step)):
        assert np.all(same)


def test_linear_codes():
    rng = np.random.default_rng(5)
    v = rng.uniform(0.01, 0.2, 4000).astype(np.float32)
    lo, hi = float(v.min()), float(v.max())
    step = float(np.float32((hi - lo) / 65535.0))
    c = O.block_code_lin(v, lo, step)
    vd = O.block_decode_lin(c, lo, step).astype(np.float64)
    assert np.all(np.abs(vd - v) <= 0.5 * step + _ulp(vd) + 1e-12)
    assert c.min() == 0 and c.max() >= 65534
    # equal values: zero step, exact decode
    w = np.full(10, 0.37, np.float32)
    assert np.all(O.block_code_lin(w, 0.37, 0.0) == 0)
    assert np.all(O.block_decode_lin(np.zeros(10, np.uint16), np.float32(0.37), 0.0) == w)
    # every code round-trips for a non-degenerate step
    cc = np.arange(65536, dtype=np.uint16)
    assert np.array_equal(O.block_code_lin(O.block_decode_lin(cc, 0.01, 3e-6), 0.01, 3e-6), cc)
    # non-finite values take code 0
    assert list(O.block_code_lin(np.array([np.nan, np.inf, -np.inf], np.float32), 0.0, 1.0)) == [0, 0, 0]


def _tree(n=30000, n_max=200, seed=21, unequal=False):
    p = synth.tiny(n, seed=seed)
    xyz = p.xyz.copy()
    xyz[:3] = np.array([[1.2, 0.5, 0.5], [-0.3, 0.2, 0.1], [0.5, 1.5, 0.5]])
    mass = p.mass.copy()
    if unequal:
        mass = (mass * np.random.default_rng(1).uniform(0.5, 2.0, n)).astype(np.float32)
    return p, xyz, mass, O.build_tree(xyz, mass, p.h, seed=3, n_max=n_max)


def test_quantised_tree_codes_and_bounds():
    p, xyz, mass, T = _tree(unequal=True)
    codes, qa, D = O.block_quantize(T)
    assert codes.shape == (len(T.pts4), 5) and codes.dtype == np.uint16
    assert codes.nbytes == 10 * len(T.pts4)          # half of the 20 bytes of (x, y, z, w, h) in fp32
    nodes = T.nodes
    internal = (nodes["flags"] & O.INTERNAL) != 0
    # a node's block is its cell: corner at qlo, step edge 2^-16
    assert np.all(qa[:, 3] == np.ldexp(1.0, -(nodes["depth"] + 16)).astype(np.float32))
    for i in range(len(nodes)):
        f, m = int(nodes[i]["point_first"]), int(nodes[i]["point_count"])
        pts = D.pts4[f:f + m]
        # representatives of an internal node share one weight: coded exactly
        if internal[i]:
            assert np.all(pts[:, 3] == nodes[i]["w_rep"])
        # decoded positions lie in the node's cell
        for a in range(3):
            assert np.all(pts[:, a] >= qa[i, a]) and np.all(pts[:, a] <= qa[i, a] + 65536 * qa[i, 3])
    # subtree bounds and h_cull cover every decoded point below, and are attained
    dn = D.nodes
    for i in range(len(dn)):
        sub = [i]
        k = 0
        while k < len(sub):
            nd = dn[sub[k]]
            if int(nd["flags"]) & O.INTERNAL:
                sub.extend(range(int(nd["child_first"]), int(nd["child_first"]) + int(nd["child_count"])))
            k += 1
        idx = np.concatenate([np.arange(int(dn[j]["point_first"]), int(dn[j]["point_first"]) + int(dn[j]["point_count"]))
                              for j in sub])
        P = D.pts4[idx]
        assert np.array_equal(dn[i]["bmin"], P[:, :3].min(axis=0))
        assert np.array_equal(dn[i]["bmax"], P[:, :3].max(axis=0))
        assert dn[i]["h_cull"] == D.hs[idx].max()
    # everything except the point data and the cull fields is the tree's own
    for f in ("code", "point_first", "point_count", "child_first", "child_count", "depth", "flags", "w_rep"):
        assert np.array_equal(dn[f], nodes[f])


@pytest.mark.parametrize("kernel", [0, 1])
def test_full_depth_quantised_render_equals_brute_force_of_decoded_points(kernel):
    p, xyz, mass, T = _tree(unequal=True)
    codes, qa, D = O.block_quantize(T)
    cam = synth.look_at((0.45, 0.55, -0.6), (0.5, 0.5, 0.5), width=160, height=120)
    rp0 = O.rparams(lambda_px=0.0, kernel=kernel)
    lod, st, nd, npts = O.render_lod(D, cam, rp0)
    leaves = (D.nodes["flags"] & O.INTERNAL) == 0
    idx = np.concatenate([np.arange(int(x["point_first"]), int(x["point_first"]) + int(x["point_count"]))
                          for x in D.nodes[leaves]])
    brute, st2, nd2 = O.splat_points(D.pts4[idx], D.hs[idx], cam, rp0)
    assert st == 0 and st2 == 0 and nd == nd2
    assert np.array_equal(lod, brute)
    # and the quantised image is close to the unquantised one (relative L1 of the accumulators)
    ref, _, _ = O.splat_particles(xyz, mass, p.h, cam, rp0)
    rel = np.abs(lod.astype(np.float64) - ref.astype(np.float64)).sum() / ref.astype(np.float64).sum()
    assert rel < 2e-3, rel


def test_default_lod_render_of_quantised_tree_is_close():
    # every particle inside the root cube (one outside it is clamped into its boundary block)
    p = synth.tiny(30000, seed=21)
    T = O.build_tree(p.xyz, p.mass, p.h, seed=3, n_max=200)
    codes, qa, D = O.block_quantize(T)
    cam = synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=200, height=150)
    rp = O.rparams(n_max=200)
    a, _, _, _ = O.render_lod(T, cam, rp)
    b, st, _, _ = O.render_lod(D, cam, rp)
    assert st == 0
    ia, ib = O.tonemap(a, rp).astype(int), O.tonemap(b, rp).astype(int)
    assert np.abs(ia - ib).max() <= 2 and np.abs(ia - ib).mean() < 0.01
