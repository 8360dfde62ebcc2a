"""Shared helpers of the GPU parity tests (inputs go to both sides from the same arrays)."""
import numpy as np
import torch

from oracle import oracle as O

NODE_FIELDS = ("code", "seg_first", "point_first", "mass_lo", "mass_hi", "seg_count", "point_count", "child_first",
               "child_count", "depth", "flags", "parent", "h_cull", "w_rep", "s_rep", "bmin", "bmax")


def dev():
    return torch.device("cuda", 0)


def to_dev(*arrays):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev()) for a in arrays)


def compare_trees(ex: dict, ot: "O.OracleTree"):
    """Bit-exact comparison of a GPU octree export with the oracle's tree."""
    gn, on = ex["nodes"], ot.nodes
    assert len(gn) == len(on), (len(gn), len(on))
    for f in NODE_FIELDS:
        a, b = gn[f], on[f]
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0][:5]
            raise AssertionError(f"node field {f} differs at {bad}: gpu {a[bad]} oracle {b[bad]}")
    assert ex["depth_max"] == ot.depth_max
    assert ex["equal_mass"] == ot.equal_mass
    assert np.array_equal(ex["skey"], ot.skey), "sorted keys differ"
    assert np.array_equal(ex["sidx"], ot.sidx), "sort permutation differs"
    assert np.array_equal(ex["pt_src"], ot.pt_src), "representative choice differs"
    assert same_floats(ex["pts4"], ot.pts4), "stored points differ"
    assert same_floats(ex["hs"], ot.hs), "stored smoothing lengths differ"


def same_floats(a, b) -> bool:
    """Bit-identical, except that any two NaNs count as equal (a NaN's payload is not part of the
    result: fp32 multiplies on the GPU return the canonical NaN, CPUs propagate the input's)."""
    a, b = np.asarray(a), np.asarray(b)
    if a.shape != b.shape:
        return False
    na, nb = np.isnan(a), np.isnan(b)
    return bool(np.array_equal(na, nb) and np.array_equal(a[~na].view(np.uint32), b[~nb].view(np.uint32)))


def u8_close(a, b, tol=1):
    d = np.abs(np.asarray(a).astype(np.int32) - np.asarray(b).astype(np.int32))
    return int(d.max()) if d.size else 0
