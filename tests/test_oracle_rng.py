"""Pins of the oracle's random-number and special-function pieces (CPU only).

The octree paragraph of the paper reduces every over-full node by a "density-weighted
random subselection".  The oracle reads that as an exponential race driven by
Philox4x32-10; these tests pin each ingredient to something other than the oracle itself:
the generator's published known answers, high-precision logarithms and cube roots, and the
exact inclusion probabilities of successive sampling proportional to mass.
"""
import math
import os

import mpmath as mp
import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if ln.strip() and ln[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        ctr = [int(v, 16) for v in r[0:4]]
        key = [int(v, 16) for v in r[4:6]]
        want = [int(v, 16) for v in r[6:10]]
        assert O.philox4x32_10(ctr, key) == want


def test_node_draw_layout():
    # counter = (particle id, code low word, code high word, 0), key = (seed low, seed high),
    # and the 64-bit draw is (r0 << 32) | r1
    seed, code, pid = 0x0123456789ABCDEF, (1 << 60) | 12345, 777
    r = O.philox4x32_10([pid, code & 0xFFFFFFFF, code >> 32, 0], [seed & 0xFFFFFFFF, seed >> 32])
    assert O.node_draw(seed, code, pid) == (r[0] << 32) | r[1]


def _ulp(x):
    return math.ulp(abs(x))


@pytest.mark.parametrize("u", [0, 1, (1 << 12) - 1, 1 << 12, 0x8000000000000000, 0xFFFFFFFFFFFFFFFF,
                               0x5A5A5A5A5A5A5A5A, 0x0000000100000000, 0xB504F333F9DE6484])
def test_neglog_special(u):
    mp.mp.prec = 200
    U = (mp.mpf(u >> 12) + mp.mpf(0.5)) * mp.mpf(2) ** -52
    ref = float(-mp.log(U))
    got = O.neglog(u)
    assert abs(got - ref) <= 2 * _ulp(ref), (u, got, ref)


def test_neglog_random():
    mp.mp.prec = 120
    rng = np.random.default_rng(5)
    us = rng.integers(0, 2**64 - 1, 2000, dtype=np.uint64, endpoint=True)
    got = O.neglogs(us)
    for u, g in zip(us.tolist(), got.tolist()):
        U = (mp.mpf(u >> 12) + mp.mpf(0.5)) * mp.mpf(2) ** -52
        ref = float(-mp.log(U))
        assert abs(g - ref) <= 2 * _ulp(ref), (u, g, ref)


def test_cbrt():
    mp.mp.prec = 120
    for t in [1.0, 8.0, 27.0, 64.0, 1000.0, 9375.0, 1.0000001, 2.0, 3.0, 16000.0 / 16000.0 + 1e-9]:
        ref = float(mp.cbrt(mp.mpf(t)))
        assert abs(O.cbrt(t) - ref) <= 2 * _ulp(ref), t
    for t in [8.0, 27.0, 64.0, 125.0, 1000.0]:
        assert O.cbrt(t) == round(t ** (1 / 3))  # exact cubes come out exact
    rng = np.random.default_rng(9)
    for t in np.exp(rng.uniform(0.0, math.log(1e7), 3000)):
        ref = float(mp.cbrt(mp.mpf(float(t))))
        assert abs(O.cbrt(float(t)) - ref) <= 2 * _ulp(ref), t


def _inclusion_exact(m, n):
    """Inclusion probabilities of successive sampling without replacement, each step choosing
    an item with probability proportional to its mass (what the exponential race produces)."""
    from itertools import permutations
    m = [float(x) for x in m]
    K = len(m)
    pi = [0.0] * K
    for order in permutations(range(K), n):
        p, left = 1.0, sum(m)
        for i in order:
            p *= m[i] / left
            left -= m[i]
        for i in order:
            pi[i] += p
    return pi


@pytest.mark.parametrize("masses,n_sel", [([1.0, 2.0, 3.0, 4.0], 1), ([1.0, 2.0, 3.0, 4.0], 2),
                                          ([0.5, 0.5, 4.0, 1.0, 2.0], 3)])
def test_density_weighted_inclusion(masses, n_sel):
    K = len(masses)
    pos = np.arange(K, dtype=np.uint32)
    ids = np.arange(100, 100 + K, dtype=np.uint32)
    mass = np.asarray(masses, np.float32)
    S = 20000
    hits = np.zeros(K)
    for s in range(S):
        ch = O.select_node(pos, ids, mass, code=9, seed=s, n_sel=n_sel, equal_mass=False)
        assert len(ch) == n_sel and np.all(np.diff(ch.astype(np.int64)) > 0)
        hits[ch] += 1
    want = np.array(_inclusion_exact(masses, n_sel))
    freq = hits / S
    sd = np.sqrt(want * (1 - want) / S)
    assert np.all(np.abs(freq - want) <= 5 * sd + 1e-12), (freq, want)


def test_equal_mass_uniform_inclusion():
    K, n_sel, S = 12, 4, 20000
    pos = np.arange(K, dtype=np.uint32)
    ids = np.arange(K, dtype=np.uint32) * 7 + 3
    mass = np.ones(K, np.float32)
    hits = np.zeros(K)
    for s in range(S):
        hits[O.select_node(pos, ids, mass, code=1, seed=s, n_sel=n_sel, equal_mass=True)] += 1
    p = n_sel / K
    sd = math.sqrt(p * (1 - p) / S)
    assert np.all(np.abs(hits / S - p) <= 5 * sd)


def test_selection_depends_on_node_code_and_seed():
    K, n_sel = 200, 20
    pos = np.arange(K, dtype=np.uint32)
    ids = np.arange(K, dtype=np.uint32)
    mass = np.ones(K, np.float32)
    a = O.select_node(pos, ids, mass, code=8, seed=1, n_sel=n_sel, equal_mass=True)
    b = O.select_node(pos, ids, mass, code=9, seed=1, n_sel=n_sel, equal_mass=True)
    c = O.select_node(pos, ids, mass, code=8, seed=2, n_sel=n_sel, equal_mass=True)
    d = O.select_node(pos, ids, mass, code=8, seed=1, n_sel=n_sel, equal_mass=True)
    assert not np.array_equal(a, b) and not np.array_equal(a, c) and np.array_equal(a, d)


def test_selection_is_the_smallest_keys():
    # brute force on a tiny node: the kept set is the n smallest (draw, id) pairs
    K, n_sel, code, seed = 50, 7, 77, 3
    pos = np.arange(K, dtype=np.uint32)
    ids = (np.arange(K, dtype=np.uint32) * 31 + 5).astype(np.uint32)
    mass = np.ones(K, np.float32)
    ch = O.select_node(pos, ids, mass, code=code, seed=seed, n_sel=n_sel, equal_mass=True)
    draws = []
    for j in range(K):
        r = O.philox4x32_10([int(ids[j]), code & 0xFFFFFFFF, code >> 32, 0], [seed & 0xFFFFFFFF, seed >> 32])
        draws.append(((r[0] << 32) | r[1], int(ids[j]), j))
    want = sorted(j for _, _, j in sorted(draws)[:n_sel])
    assert ch.tolist() == want
