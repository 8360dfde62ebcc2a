"""GPU parity of the octree build (A1-A5) against the oracle, through the C ABI.

Bit-exact: Morton keys, the (key, id) sort, the node table, exact node masses, representative
choice, weights and smoothing lengths (octree paragraph of the paper; readings R-1..R-9)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

from gpu_helpers import compare_trees, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_0811_2055_gb300 import gblod
    torch.cuda.set_device(0)
    return gblod


def test_morton_keys(G):
    rng = np.random.default_rng(1)
    pts = rng.uniform(-0.1, 1.1, (100_003, 3)).astype(np.float32)
    pts[:6] = [[0, 0, 0], [0.5, 0.5, 0.5], [1, 1, 1], [np.nan, 0.3, 0.2], [-1e-30, 2.0, 0.999], [1e-38, 0.5, 0.25]]
    (d,) = to_dev(pts)
    got = G.morton_keys(d).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, O.morton_keys(pts))
    lo, side = (-0.37, 0.25, -2.0), 3.3  # a root cube where the FP64 quantisation rounds
    got = G.morton_keys(d, root_lo=lo, root_side=side).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, O.morton_keys(pts, lo=lo, side=side))


CASES = {
    "tiny_cfg": lambda: (synth.tiny(), None, 16000),
    "tiny_nmax1000": lambda: (synth.tiny(40000, seed=11), None, 1000),
    "clustered_nmax64": lambda: (synth.clustered(20000, 32, 0.1, 0.2, seed=3), None, 64),
    "uniform_nmax8": lambda: (synth.uniform(3000, seed=4), None, 8),
    "nmax1": lambda: (synth.uniform(700, seed=9), None, 1),
    "mid_1M": lambda: (synth.mid(1 << 20, seed=12), None, 16000),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_tree_parity(G, name):
    p, ids, n_max = CASES[name]()
    xyz, mass, h = to_dev(p.xyz, p.mass, p.h)
    t = G.build_lod(xyz, mass, h, n_max=n_max, seed=7)
    compare_trees(t.export(), O.build_tree(p.xyz, p.mass, p.h, seed=7, n_max=n_max))


def test_unequal_masses_outside_points(G):
    rng = np.random.default_rng(8)
    n = 50000
    xyz = rng.uniform(-0.05, 1.05, (n, 3)).astype(np.float32)
    mass = np.exp(rng.uniform(-3, 3, n)).astype(np.float32)
    h = rng.uniform(0.001, 0.02, n).astype(np.float32)
    h[:10] = [0.0, -1.0, np.nan, np.inf, 1e-30, 0, 0, 0, 0, 0]
    t = G.build_lod(*to_dev(xyz, mass, h), n_max=300, seed=2)
    ot = O.build_tree(xyz, mass, h, seed=2, n_max=300)
    assert not ot.equal_mass
    compare_trees(t.export(), ot)


@pytest.mark.parametrize("m0", [0.3, 3000.0])
def test_equal_masses_other_than_one_with_and_without_ids(G, m0):
    # one mass for every particle: node masses are the count times m0's fixed-point value (no mass
    # prefix), and without caller ids the sorted ids are the sort permutation itself
    p = synth.clustered(50000, 60, 0.1, 0.3, seed=14)
    mass = np.full(p.n, m0, np.float32)
    ids = ((np.arange(p.n, dtype=np.uint64) * 2246822519 + 7) % (1 << 32)).astype(np.uint32)
    t = G.build_lod(*to_dev(p.xyz, mass, p.h), n_max=200, seed=5)
    ot = O.build_tree(p.xyz, mass, p.h, seed=5, n_max=200)
    assert ot.equal_mass
    compare_trees(t.export(), ot)
    t = G.build_lod(*to_dev(p.xyz, mass, p.h), ids=to_dev(ids.view(np.int32))[0], n_max=200, seed=5)
    compare_trees(t.export(), O.build_tree(p.xyz, mass, p.h, ids=ids, seed=5, n_max=200))


def test_ids_and_order_freeness(G):
    p = synth.clustered(30000, 40, 0.1, 0.2, seed=6)
    ids = ((np.arange(p.n, dtype=np.uint64) * 2654435761) % (1 << 32)).astype(np.uint32)
    assert len(np.unique(ids)) == p.n
    perm = np.random.default_rng(0).permutation(p.n)
    a = G.build_lod(*to_dev(p.xyz, p.mass, p.h), ids=to_dev(ids.view(np.int32))[0], n_max=100, seed=9).export()
    b = G.build_lod(*to_dev(p.xyz[perm], p.mass[perm], p.h[perm]), ids=to_dev(ids[perm].view(np.int32))[0],
                    n_max=100, seed=9).export()
    compare_trees(a, O.build_tree(p.xyz, p.mass, p.h, ids=ids, seed=9, n_max=100))
    for f in ("code", "seg_count", "mass_lo", "w_rep", "h_cull"):
        assert np.array_equal(a["nodes"][f], b["nodes"][f])
    assert np.array_equal(a["pts4"], b["pts4"]) and np.array_equal(a["hs"], b["hs"])


def test_coincident_points_lossy_leaf(G):
    n = 5000
    xyz = np.full((n, 3), 0.3, np.float32)
    xyz[:100] = 0.7
    mass, h = np.ones(n, np.float32), np.full(n, 0.01, np.float32)
    t = G.build_lod(*to_dev(xyz, mass, h), n_max=10, seed=1)
    ot = O.build_tree(xyz, mass, h, seed=1, n_max=10)
    ex = t.export()
    compare_trees(ex, ot)
    assert ex["depth_max"] == 21 and ((ex["nodes"]["flags"] & G.NODE_LOSSY) != 0).sum() == 2


def test_degenerate_sizes(G):
    e = np.zeros((0, 3), np.float32)
    t = G.build_lod(*to_dev(e, np.zeros(0, np.float32), np.zeros(0, np.float32)), n_max=4)
    assert t.info().n_nodes == 0
    one = np.array([[0.2, 0.4, 0.6]], np.float32)
    t = G.build_lod(*to_dev(one, np.ones(1, np.float32), np.ones(1, np.float32)), n_max=1)
    compare_trees(t.export(), O.build_tree(one, np.ones(1, np.float32), np.ones(1, np.float32), n_max=1))
    p = synth.uniform(5000, seed=1)
    t = G.build_lod(*to_dev(p.xyz, p.mass, p.h), n_max=5000)
    ex = t.export()
    assert len(ex["nodes"]) == 1 and ex["nodes"]["flags"][0] == G.NODE_LEAF
    compare_trees(ex, O.build_tree(p.xyz, p.mass, p.h, n_max=5000))


def test_bad_masses_are_rejected(G):
    xyz = np.random.default_rng(0).uniform(0, 1, (1000, 3)).astype(np.float32)
    for bad in [0.0, -1.0, 2.0**25, float("nan"), float("inf")]:
        mass = np.ones(1000, np.float32)
        mass[500] = bad
        with pytest.raises(G.GblodError) as e:
            G.build_lod(*to_dev(xyz, mass, np.ones(1000, np.float32)), n_max=10)
        assert e.value.code == G.ERR_RANGE
    with pytest.raises(G.GblodError) as e:
        G.build_lod(*to_dev(xyz, np.ones(1000, np.float32), np.ones(1000, np.float32)), n_max=0)
    assert e.value.code == G.ERR_INVALID_ARG


def test_mid_workload_full_size(G):
    """The 2^24-particle mid workload at full size, exactly as the benchmark builds it."""
    p = synth.mid()
    t = G.build_lod(*to_dev(p.xyz, p.mass, p.h), n_max=16000, seed=1)
    compare_trees(t.export(), O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=16000))
