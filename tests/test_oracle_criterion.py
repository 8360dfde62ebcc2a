"""Pins of the oracle's detail criterion on both sides of its threshold (CPU only).

Depth paragraph: nodes close to the viewer are drawn deep, far ones shallow.  Reading R-13 makes
this exact: an internal node is refined iff (F * edge)^2 > lambda^2 * max(D^2, z_near^2), with
`edge` the node's cell edge (root side * 2^-depth) and D the distance from the eye to the node's
cell (0 inside).  Each case below puts the eye (or lambda, or F) a relative 1e-9 to either side
of the threshold worked out by hand, so any other reading -- lambda instead of lambda^2, the cell
diagonal instead of its edge, the distance to the cell centre or along one axis only, D instead
of max(D, z_near) -- lands on the wrong side of at least one case.
"""
import math

import numpy as np

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

EPS = 1e-9


def _tree(z_lo=0.0, z_hi=1.0, n=600, n_max=4, seed=5):
    rng = np.random.default_rng(seed)
    xyz = np.stack([rng.uniform(0.02, 0.98, n), rng.uniform(0.02, 0.98, n), rng.uniform(z_lo, z_hi, n)], 1)
    xyz = xyz.astype(np.float32)
    mass = np.ones(n, np.float32)
    h = np.full(n, 1e-4, np.float32)
    T = O.build_tree(xyz, mass, h, seed=1, n_max=n_max)
    assert int(T.nodes[0]["flags"]) & O.INTERNAL
    return T


def _cam(eye, target, F, W=64, H=64, z_near=1e-3):
    cam = synth.look_at(eye, target, width=W, height=H, z_near=z_near)
    cam["f_px"] = float(F)
    return cam


def _sel(T, cam, lam):
    return set(O.select(T, cam, O.rparams(lambda_px=lam)).tolist())


def _children(T, i):
    nd = T.nodes[i]
    return list(range(int(nd["child_first"]), int(nd["child_first"]) + int(nd["child_count"])))


def test_root_threshold_on_axis():
    # eye on the cube's axis, D = distance to the face z = 0; (F * 1)^2 = lambda^2 D^2 at D = F / lambda
    T = _tree()
    F, lam = 1000.0, 10.0
    for s, refined in ((1.0 - EPS, True), (1.0 + EPS, False)):
        D = (F / lam) * s
        sel = _sel(T, _cam((0.5, 0.5, -D), (0.5, 0.5, 0.5), F), lam)
        assert (0 not in sel) == refined, (s, sorted(sel)[:8])
        if refined:
            assert set(_children(T, 0)) <= sel  # the children (edge 1/2, D >= 100) are emitted
        else:
            assert sel == {0}


def test_root_threshold_off_axis_corner_distance():
    # eye beyond the x = 1 face and in front of z = 0: D^2 = 30^2 + 40^2 = 50^2 (distance to the
    # cell's edge line, not to its centre and not along one axis)
    T = _tree()
    F, lam = 1000.0, 20.0
    for s, refined in ((1.0 - EPS, True), (1.0 + EPS, False)):
        eye = (1.0 + 30.0 * s, 0.5, -40.0 * s)
        sel = _sel(T, _cam(eye, (0.5, 0.5, 0.5), F), lam)
        assert (0 not in sel) == refined, s


def test_child_threshold_uses_the_child_edge():
    # lambda scanned instead of the eye: at D = 100 the front children (cells z in [0, 1/2),
    # edge 1/2) meet the threshold at lambda = F * 0.5 / D = 5; the back ones are 100.5 away
    T = _tree()
    F, D = 1000.0, 100.0
    cam = _cam((0.5, 0.5, -D), (0.5, 0.5, 0.5), F)
    front = [c for c in _children(T, 0) if (int(T.nodes[c]["code"]) & 1) == 0]
    back = [c for c in _children(T, 0) if (int(T.nodes[c]["code"]) & 1) == 1]
    front_int = [c for c in front if int(T.nodes[c]["flags"]) & O.INTERNAL]
    assert front_int and back
    lo = _sel(T, cam, 5.0 * (1.0 - EPS))
    hi = _sel(T, cam, 5.0 * (1.0 + EPS))
    for c in front_int:
        assert c not in lo and c in hi
    for c in back:
        assert c in lo and c in hi
    assert 0 not in lo and 0 not in hi


def test_near_plane_replaces_a_smaller_distance():
    # eye 0.3 in front of the root cell, particles only at z in [0.9, 1) (so nothing is behind
    # z_near = 0.5): D = 0.3 < z_near, and the root is refined iff F > lambda * z_near = 5
    T = _tree(z_lo=0.9, z_hi=0.999)
    lam, zn = 10.0, 0.5
    for s, refined in ((1.0 + EPS, True), (1.0 - EPS, False)):
        F = lam * zn * s
        cam = _cam((0.5, 0.5, -0.3), (0.5, 0.5, 0.5), F, z_near=zn)
        sel = _sel(T, cam, lam)
        assert (0 not in sel) == refined, s
    # with D = 0.3 alone the threshold would be F = 3: F = 4 must still emit the root
    cam = _cam((0.5, 0.5, -0.3), (0.5, 0.5, 0.5), 4.0, z_near=zn)
    assert _sel(T, cam, lam) == {0}


def test_threshold_scales_with_lambda_squared():
    # lambda and D scaled together leave the decision unchanged; lambda alone moves it as 1/D
    T = _tree()
    F = 1000.0
    for lam in (2.0, 10.0, 50.0):
        D = F / lam
        assert 0 not in _sel(T, _cam((0.5, 0.5, -D * (1 - EPS)), (0.5, 0.5, 0.5), F), lam)
        assert _sel(T, _cam((0.5, 0.5, -D * (1 + EPS)), (0.5, 0.5, 0.5), F), lam) == {0}
    assert math.isclose(F / 10.0, 100.0)
