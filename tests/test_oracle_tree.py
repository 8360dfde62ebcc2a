"""Pins of the oracle's octree build (CPU only).

Octree paragraph of the paper: a spatial octree whose every node is represented by at most
n points (n = 16000 there); over-full nodes are reduced by a density-weighted random
subselection, and the children of a node hold the same data as the parent at 8x the detail.
These tests check the oracle against: keys derived by repeated halving of the box in exact
rational arithmetic, a second tree construction that never forms a key, hand-derived trees,
and the invariants the paragraph fixes.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def halving_key(x, y, z, lo=(0.0, 0.0, 0.0), side=1.0):
    """Octant path by repeated halving of the root cube, with exact rationals (valid when
    lo and side are dyadic, so that the specified FP64 quantisation is exact)."""
    p = [Fraction(float(v)) if not math.isnan(v) else None for v in (x, y, z)]
    blo = [Fraction(v) for v in lo]
    edge = Fraction(side)
    key = 0
    for _ in range(21):
        edge /= 2
        o = 0
        for a in range(3):
            if p[a] is None:
                bit = 0
            else:
                bit = 1 if p[a] >= blo[a] + edge else 0
            if bit:
                blo[a] += edge
            o |= bit << (2 - a)
        key = key * 8 + o
    return key


def test_morton_against_halving():
    rng = np.random.default_rng(1)
    pts = rng.uniform(-0.1, 1.1, (400, 3)).astype(np.float32)
    special = np.array([[0, 0, 0], [0.5, 0.5, 0.5], [0.75, 0.25, 0.25], [1.0, 1.0, 1.0],
                        [np.nextafter(np.float32(1), np.float32(0))] * 3, [-1e-30, 2.0, 0.999],
                        [1e-30, 1e-38, 0.125]], np.float32)
    pts = np.concatenate([pts, special])
    keys = O.morton_keys(pts)
    for (x, y, z), k in zip(pts.tolist(), keys.tolist()):
        assert k == halving_key(x, y, z), (x, y, z)
    assert int(O.morton_key(0.75, 0.25, 0.25)) >> 60 == 4
    assert (int(O.morton_key(0.75, 0.25, 0.25)) >> 57) & 7 == 7


def test_morton_nondefault_root_and_nan():
    rng = np.random.default_rng(2)
    lo, side = (-0.5, 0.25, -2.0), 4.0
    pts = (np.array(lo) + rng.uniform(-0.2, 4.2, (300, 3))).astype(np.float32)
    keys = O.morton_keys(pts, lo=lo, side=side)
    for (x, y, z), k in zip(pts.tolist(), keys.tolist()):
        assert k == halving_key(x, y, z, lo, side)
    nan = float("nan")
    assert O.morton_key(nan, nan, nan) == 0
    assert O.morton_key(nan, 0.75, 0.0) == halving_key(0.0, 0.75, 0.0)


def _members(T, i, ids=None):
    nd = T.nodes[i]
    sl = T.sidx[int(nd["seg_first"]): int(nd["seg_first"]) + int(nd["seg_count"])]
    return np.sort(sl if ids is None else ids[sl])


def _clustered_small(n=20000, seed=3):
    return synth.clustered(n, 32, 0.1, 0.2, seed=seed)


INPUTS = {
    "tiny_nmax1000": lambda: (synth.tiny(40000, seed=11), 1000),
    "clustered_nmax64": lambda: (_clustered_small(), 64),
    "uniform_nmax8": lambda: (synth.uniform(3000, seed=4), 8),
}


@pytest.mark.parametrize("name", sorted(INPUTS))
def test_two_constructions_agree(name):
    p, n_max = INPUTS[name]()
    T = O.build_tree(p.xyz, p.mass, p.h, seed=5, n_max=n_max)
    td = O.build_topdown(p.xyz, n_max=n_max)
    assert np.array_equal(td["code"], T.nodes["code"])
    assert np.array_equal(td["depth"], T.nodes["depth"])
    assert np.array_equal(td["count"], T.nodes["seg_count"])
    assert np.array_equal(td["flags"], T.nodes["flags"])
    off = 0
    for i in range(len(T.nodes)):
        c = int(T.nodes[i]["seg_count"])
        assert np.array_equal(td["members"][off:off + c], _members(T, i))
        off += c


def test_hand_worked_trees():
    g = json.load(open(os.path.join(GOLDEN, "hand_tree_5pts.json")))
    xyz = np.asarray(g["points"], np.float32)
    mass = np.asarray(g["mass"], np.float32)
    h = np.full(len(xyz), 0.01, np.float32)
    kinds = {"leaf": O.LEAF, "internal": O.INTERNAL | O.REPS}
    for tree in g["trees"]:
        T = O.build_tree(xyz, mass, h, seed=1, n_max=tree["n_max"])
        assert len(T.nodes) == len(tree["nodes"])
        M = T.masses()
        for i, want in enumerate(tree["nodes"]):
            nd = T.nodes[i]
            assert int(nd["code"]) == want["code"] and int(nd["depth"]) == want["depth"]
            assert _members(T, i).tolist() == want["members"]
            assert int(nd["flags"]) == kinds[want["kind"]]
            assert M[i] == int(want["mass"] * 2**47)
            if want["kind"] == "internal":
                n_sel = tree["n_max"]
                assert nd["w_rep"] == np.float32(want["mass"] / n_sel)
                assert nd["s_rep"] == np.float32(len(want["members"]) / n_sel) ** np.float32(1 / 3) or \
                    abs(float(nd["s_rep"]) - (len(want["members"]) / n_sel) ** (1 / 3)) <= 1e-6


def check_invariants(T, xyz, mass, h, n_max):
    nodes = T.nodes
    n = T.n
    M = T.masses()
    Mtot = sum(int(round(float(m) * 2**47)) for m in mass.astype(np.float64))
    if n == 0:
        assert len(nodes) == 0
        return
    assert M[0] == Mtot
    leaf_cover = np.zeros(n, np.int64)
    for i, nd in enumerate(nodes):
        f, c, d = int(nd["flags"]), int(nd["seg_count"]), int(nd["depth"])
        b = int(nd["seg_first"])
        # I1: at most n points stored per node
        assert int(nd["point_count"]) <= n_max
        if f & O.LEAF:
            assert c <= n_max and int(nd["point_count"]) == c
            leaf_cover[b:b + c] += 1
            # I4: leaves keep their particles verbatim
            p0 = int(nd["point_first"])
            src = T.sidx[b:b + c]
            assert np.array_equal(T.pts4[p0:p0 + c, :3], xyz[src])
            assert np.array_equal(T.pts4[p0:p0 + c, 3], mass[src])
            assert np.array_equal(T.hs[p0:p0 + c], h[src])
        else:
            assert c > n_max and int(nd["point_count"]) == n_max
            assert bool(f & O.INTERNAL) == (d < O.MAX_DEPTH)
            # I5: representatives are distinct members of the node
            p0 = int(nd["point_first"])
            srcpos = T.pt_src[p0:p0 + n_max].astype(np.int64)
            assert np.all(np.diff(srcpos) > 0) and srcpos[0] >= b and srcpos[-1] < b + c
            src = T.sidx[srcpos]
            assert np.array_equal(T.pts4[p0:p0 + n_max, :3], xyz[src])
            w = np.float32(nd["w_rep"])
            assert np.all(T.pts4[p0:p0 + n_max, 3] == w)
            # weights carry the node's mass: n_sel * w == M_node to fp32 rounding
            assert abs(float(w) * n_max - M[i] / 2**47) <= n_max * float(np.spacing(w)) / 2
            ratio = T.hs[p0:p0 + n_max].astype(np.float64) / h[src].astype(np.float64)
            assert np.allclose(ratio, (c / n_max) ** (1 / 3), rtol=3e-7)
        if f & O.INTERNAL:
            # I2: children are the non-empty octants, in octant order, partitioning the parent
            k0, kc = int(nd["child_first"]), int(nd["child_count"])
            assert 1 <= kc <= 8
            ch = nodes[k0:k0 + kc]
            octs = [int(x) - 8 * int(nd["code"]) for x in ch["code"]]
            assert octs == sorted(octs) and all(0 <= o < 8 for o in octs)
            assert np.all(ch["depth"] == d + 1)
            assert int(ch[0]["seg_first"]) == b
            assert np.all(ch["seg_first"][1:] == ch["seg_first"][:-1] + ch["seg_count"][:-1])
            assert int(ch["seg_count"].sum()) == c
            assert sum(M[k0:k0 + kc]) == M[i]
            assert float(nd["h_cull"]) >= float(ch["h_cull"].max())
        # particle bounds contain the members; cull radius covers every stored h
        mem = xyz[T.sidx[b:b + c]]
        assert np.all(mem >= nd["bmin"]) and np.all(mem <= nd["bmax"])
        p0, pc = int(nd["point_first"]), int(nd["point_count"])
        assert float(nd["h_cull"]) >= float(T.hs[p0:p0 + pc].max())
        # cell box: in-cube members sit in the node's octant cell
        qs = np.stack([np.floor(mem.astype(np.float64) * 2**21)], 0)[0]
        inside = np.all((mem >= 0) & (mem < 1), axis=1)
        cell = int(nd["code"]) ^ (1 << (3 * d))
        if d > 0 and inside.any():
            qq = qs[inside].astype(np.int64) >> (21 - d)
            for a in range(3):
                want = 0
                for l in range(d):
                    want = (want << 1) | ((cell >> (3 * (d - 1 - l) + (2 - a))) & 1)
                assert np.all(qq[:, a] == want)
    # I4: every particle in exactly one leaf
    lossy = [i for i, nd in enumerate(nodes) if int(nd["flags"]) & O.LOSSY]
    for i in lossy:
        b, c = int(nodes[i]["seg_first"]), int(nodes[i]["seg_count"])
        leaf_cover[b:b + c] += 1
    assert np.all(leaf_cover == 1)
    # I3: mass conserved on every level cut (nodes at depth L plus shallower leaves)
    for L in range(T.depth_max + 1):
        tot = 0
        for i, nd in enumerate(nodes):
            d = int(nd["depth"])
            if d == L or (d < L and not int(nd["flags"]) & O.INTERNAL):
                tot += M[i]
        assert tot == Mtot, L


@pytest.mark.parametrize("name", sorted(INPUTS))
def test_invariants(name):
    p, n_max = INPUTS[name]()
    T = O.build_tree(p.xyz, p.mass, p.h, seed=5, n_max=n_max)
    check_invariants(T, p.xyz, p.mass, p.h, n_max)


def test_invariants_tiny_workload(tiny_particles):
    p = tiny_particles
    T = O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=16000)
    check_invariants(T, p.xyz, p.mass, p.h, 16000)


def test_unequal_masses_and_outside_points():
    rng = np.random.default_rng(8)
    n = 5000
    xyz = rng.uniform(-0.05, 1.05, (n, 3)).astype(np.float32)
    mass = np.exp(rng.uniform(-3, 3, n)).astype(np.float32)
    h = rng.uniform(0.001, 0.02, n).astype(np.float32)
    T = O.build_tree(xyz, mass, h, seed=2, n_max=50)
    assert not T.equal_mass
    check_invariants(T, xyz, mass, h, 50)


def test_coincident_points_make_a_lossy_leaf():
    n = 100
    xyz = np.full((n, 3), 0.3, np.float32)
    T = O.build_tree(xyz, np.ones(n, np.float32), np.full(n, 0.01, np.float32), seed=1, n_max=10)
    assert len(T.nodes) == 22 and T.depth_max == 21
    last = T.nodes[-1]
    assert int(last["flags"]) == O.LOSSY | O.REPS and int(last["point_count"]) == 10
    check_invariants(T, xyz, np.ones(n, np.float32), np.full(n, 0.01, np.float32), 10)


def test_degenerate_sizes():
    e = np.zeros((0, 3), np.float32)
    T = O.build_tree(e, np.zeros(0, np.float32), np.zeros(0, np.float32), n_max=4)
    assert len(T.nodes) == 0 and len(T.pts4) == 0
    T = O.build_tree(np.array([[0.2, 0.4, 0.6]], np.float32), np.ones(1, np.float32), np.ones(1, np.float32), n_max=1)
    assert len(T.nodes) == 1 and int(T.nodes[0]["flags"]) == O.LEAF
    p = synth.uniform(500, seed=1)
    T = O.build_tree(p.xyz, p.mass, p.h, n_max=500)  # n_max >= N: the root is a leaf
    assert len(T.nodes) == 1 and int(T.nodes[0]["flags"]) == O.LEAF


def test_mass_out_of_range_is_rejected():
    xyz = np.zeros((2, 3), np.float32)
    for bad in [0.0, -1.0, 2.0**25, float("nan"), float("inf"), 2.0**-25]:
        with pytest.raises(O.OracleError) as e:
            O.build_tree(xyz, np.array([1.0, bad], np.float32), np.ones(2, np.float32), n_max=1)
        assert e.value.code == O.ERR_RANGE


def test_order_free_under_permutation():
    p = _clustered_small(8000, seed=6)
    ids = np.arange(p.n, dtype=np.uint32) * 3 + 11
    T1 = O.build_tree(p.xyz, p.mass, p.h, ids=ids, seed=9, n_max=100)
    perm = np.random.default_rng(0).permutation(p.n)
    T2 = O.build_tree(p.xyz[perm], p.mass[perm], p.h[perm], ids=ids[perm], seed=9, n_max=100)
    for f in ("code", "seg_first", "seg_count", "point_first", "point_count", "mass_lo", "mass_hi", "flags",
              "w_rep", "s_rep", "h_cull", "bmin", "bmax"):
        assert np.array_equal(T1.nodes[f], T2.nodes[f]), f
    assert np.array_equal(T1.pts4, T2.pts4) and np.array_equal(T1.hs, T2.hs)
    assert np.array_equal(ids[T1.sidx], ids[perm][T2.sidx])
    # and without ids the ids are the input indices, so a permutation changes the draw
    T3 = O.build_tree(p.xyz[perm], p.mass[perm], p.h[perm], seed=9, n_max=100)
    assert not np.array_equal(T1.pts4, T3.pts4)
