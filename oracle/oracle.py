"""ctypes wrapper of the C oracle in ``oracle.c``.

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the benchmark's
CPU-baseline leg are the only users.  The product library neither imports nor links this.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

LEAF, INTERNAL, LOSSY, REPS = 1, 2, 4, 8
MAX_DEPTH = 21
OK, ERR_INVALID, ERR_RANGE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c with every float operation rounded on its own (no FMA contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-lm", "-o", tmp]
        try:  # OpenMP only shares a frame's points out between threads (integer images, order-free)
            subprocess.check_call(base[:5] + ["-fopenmp"] + base[5:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, LIB)
    return LIB


class Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("right", C.c_double * 3), ("up", C.c_double * 3),
                ("fwd", C.c_double * 3), ("f_px", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("z_near", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class RParams(C.Structure):
    _fields_ = [("lambda_px", C.c_double), ("sigma_min_px", C.c_double), ("sigma_max_px", C.c_double),
                ("tone_lo", C.c_double), ("tone_hi", C.c_double), ("kernel", C.c_int32),
                ("tone_auto", C.c_int32)]


class Node(C.Structure):
    _fields_ = [("code", C.c_uint64), ("seg_first", C.c_uint64), ("point_first", C.c_uint64),
                ("mass_lo", C.c_uint64), ("mass_hi", C.c_uint64), ("seg_count", C.c_uint32),
                ("point_count", C.c_uint32), ("child_first", C.c_uint32), ("child_count", C.c_uint32),
                ("depth", C.c_int32), ("flags", C.c_int32), ("parent", C.c_int32), ("pad", C.c_int32),
                ("h_cull", C.c_float), ("w_rep", C.c_float), ("s_rep", C.c_float), ("pad2", C.c_float),
                ("bmin", C.c_float * 3), ("bmax", C.c_float * 3)]


class Tree(C.Structure):
    _fields_ = [("nodes", C.POINTER(Node)), ("n_nodes", C.c_uint64), ("pts4", C.POINTER(C.c_float)),
                ("hs", C.POINTER(C.c_float)), ("pt_src", C.POINTER(C.c_uint32)), ("n_pts", C.c_uint64),
                ("skey", C.POINTER(C.c_uint64)), ("sidx", C.POINTER(C.c_uint32)), ("n", C.c_uint64),
                ("depth_max", C.c_int32), ("equal_mass", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        f32p, u32p, u64p, i32p, f64p = (np.ctypeslib.ndpointer(np.float32, flags="C"),
                                          np.ctypeslib.ndpointer(np.uint32, flags="C"),
                                          np.ctypeslib.ndpointer(np.uint64, flags="C"),
                                          np.ctypeslib.ndpointer(np.int32, flags="C"),
                                          np.ctypeslib.ndpointer(np.float64, flags="C"))
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_node_draw.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32]
        L.orc_node_draw.restype = C.c_uint64
        L.orc_node_draws.argtypes = [C.c_uint64, C.c_uint64, u32p, C.c_uint64, u64p]
        L.orc_neglog.argtypes = [C.c_uint64]
        L.orc_neglog.restype = C.c_double
        L.orc_neglogs.argtypes = [u64p, C.c_uint64, f64p]
        L.orc_cbrt.argtypes = [C.c_double]
        L.orc_cbrt.restype = C.c_double
        L.orc_kernel_table.argtypes = [C.c_int, i32p]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        L.orc_morton_key.argtypes = [C.c_float, C.c_float, C.c_float, f64p, C.c_double]
        L.orc_morton_key.restype = C.c_uint64
        L.orc_morton_keys.argtypes = [f32p, C.c_uint64, f64p, C.c_double, u64p]
        L.orc_quantize.argtypes = [C.c_float, C.c_float, C.c_float, f64p, C.c_double, u32p]
        L.orc_build.argtypes = [f32p, f32p, f32p, C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint32, f64p,
                                C.c_double, P(P(Tree))]
        L.orc_build.restype = C.c_int
        L.orc_tree_free.argtypes = [P(Tree)]
        L.orc_build_topdown.argtypes = [f32p, C.c_void_p, C.c_uint64, C.c_uint32, f64p, C.c_double,
                                        P(C.c_uint64), P(C.c_uint64), C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
        L.orc_select_node.argtypes = [u32p, u32p, f32p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, C.c_int,
                                      u32p]
        L.orc_project.argtypes = [P(Camera), P(RParams), C.c_float, C.c_float, C.c_float, C.c_float, C.c_float,
                                  np.ctypeslib.ndpointer(np.int64, flags="C")]
        L.orc_project.restype = C.c_int
        L.orc_splat_points.argtypes = [f32p, f32p, C.c_uint64, P(Camera), P(RParams), u64p, P(C.c_uint64)]
        L.orc_splat_points.restype = C.c_int
        L.orc_count_updates.argtypes = [f32p, f32p, C.c_uint64, P(Camera), P(RParams)]
        L.orc_count_updates.restype = C.c_uint64
        L.orc_splat_particles.argtypes = [f32p, f32p, f32p, C.c_uint64, P(Camera), P(RParams), u64p,
                                          P(C.c_uint64)]
        L.orc_splat_particles.restype = C.c_int
        L.orc_pixel_value.argtypes = [f32p, f32p, C.c_uint64, P(Camera), P(RParams), C.c_int, C.c_int]
        L.orc_pixel_value.restype = C.c_uint64
        L.orc_select.argtypes = [P(Tree), f64p, C.c_double, P(Camera), P(RParams), u32p]
        L.orc_select.restype = C.c_int64
        L.orc_render_lod.argtypes = [P(Tree), f64p, C.c_double, P(Camera), P(RParams), u64p, P(C.c_uint64),
                                     P(C.c_uint64)]
        L.orc_render_lod_counted.argtypes = [P(Tree), f64p, C.c_double, P(Camera), P(RParams), u64p,
                                             P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
        L.orc_render_lod_counted.restype = C.c_int
        L.orc_render_lod_rows.argtypes = [P(Tree), f64p, C.c_double, P(Camera), P(RParams), C.c_int32, C.c_int32,
                                          u64p, P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
        L.orc_render_lod_rows.restype = C.c_int
        L.orc_render_lod_part.argtypes = [P(Tree), f64p, C.c_double, P(Camera), P(RParams), C.c_int32, C.c_int32,
                                          u64p, P(C.c_uint64), P(C.c_uint64)]
        L.orc_render_lod_part.restype = C.c_int
        L.orc_tree_set_points.argtypes = [P(Tree), C.c_uint32, f32p, f32p, C.c_uint64]
        L.orc_tree_set_points.restype = C.c_int
        L.orc_render_lod.restype = C.c_int
        L.orc_tonemap.argtypes = [u64p, C.c_uint64, P(RParams), np.ctypeslib.ndpointer(np.uint8, flags="C")]
        L.orc_constants.argtypes = [np.ctypeslib.ndpointer(np.float32, flags="C")]
        u16p = np.ctypeslib.ndpointer(np.uint16, flags="C")
        L.orc_block_quantize.argtypes = [P(Tree), f64p, C.c_double, u16p, f32p, P(P(Tree))]
        L.orc_block_quantize.restype = C.c_int
        for nm in ("orc_block_code_pos", "orc_block_code_lin"):
            getattr(L, nm).argtypes = [f32p, C.c_uint64, C.c_float, C.c_float, u16p]
        for nm in ("orc_block_decode_pos", "orc_block_decode_lin"):
            getattr(L, nm).argtypes = [u16p, C.c_uint64, C.c_float, C.c_float, f32p]
        _lib = L
    return _lib


def constants():
    out = np.zeros(4, np.float32)
    lib().orc_constants(out)
    return dict(A_gauss=out[0], A_cubic=out[1], B_gauss=out[2], B_cubic=out[3])


# ------------------------------------------------------------------ small functions

def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return [int(v) for v in out]


def node_draw(seed: int, code: int, pid: int) -> int:
    return int(lib().orc_node_draw(seed, code, pid))


def node_draws(seed: int, code: int, ids) -> np.ndarray:
    ids = np.ascontiguousarray(ids, np.uint32)
    out = np.zeros(ids.size, np.uint64)
    lib().orc_node_draws(seed, code, ids, ids.size, out)
    return out


def neglog(u: int) -> float:
    return float(lib().orc_neglog(u))


def neglogs(u) -> np.ndarray:
    u = np.ascontiguousarray(u, np.uint64)
    out = np.zeros(u.size, np.float64)
    lib().orc_neglogs(u, u.size, out)
    return out


def cbrt(t: float) -> float:
    return float(lib().orc_cbrt(t))


def set_threads(n: int):
    """Threads of the frame loops (0 = all that OpenMP offers); images do not depend on it."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def kernel_table(kernel: int = 0) -> np.ndarray:
    K = np.zeros(1024, np.int32)
    lib().orc_kernel_table(kernel, K)
    return K


def _lo(lo):
    return np.ascontiguousarray(lo if lo is not None else (0.0, 0.0, 0.0), np.float64)


def morton_key(x, y, z, lo=None, side=1.0) -> int:
    return int(lib().orc_morton_key(x, y, z, _lo(lo), side))


def morton_keys(xyz, lo=None, side=1.0) -> np.ndarray:
    xyz = np.ascontiguousarray(xyz, np.float32)
    out = np.zeros(xyz.shape[0], np.uint64)
    lib().orc_morton_keys(xyz, xyz.shape[0], _lo(lo), side, out)
    return out


def quantize(x, y, z, lo=None, side=1.0):
    q = np.zeros(3, np.uint32)
    lib().orc_quantize(x, y, z, _lo(lo), side, q)
    return [int(v) for v in q]


def camera(cam: dict) -> Camera:
    c = Camera()
    for k in ("eye", "right", "up", "fwd"):
        getattr(c, k)[:] = [float(v) for v in cam[k]]
    c.f_px, c.cx, c.cy, c.z_near = float(cam["f_px"]), float(cam["cx"]), float(cam["cy"]), float(cam["z_near"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


def rparams(lambda_px=None, n_max=16000, sigma_min_px=0.5, sigma_max_px=128.0, kernel=0, tone_auto=1,
            tone_lo=0.0, tone_hi=0.0) -> RParams:
    r = RParams()
    r.lambda_px = math.sqrt(n_max) if lambda_px is None else float(lambda_px)
    r.sigma_min_px, r.sigma_max_px = float(sigma_min_px), float(sigma_max_px)
    r.tone_lo, r.tone_hi = float(tone_lo), float(tone_hi)
    r.kernel, r.tone_auto = int(kernel), int(tone_auto)
    return r


def project(cam: dict, rp: RParams, x, y, z, w, h):
    out = np.zeros(5, np.int64)
    lib().orc_project(C.byref(camera(cam)), C.byref(rp), x, y, z, w, h, out)
    return tuple(int(v) for v in out)


# ------------------------------------------------------------------ octree

NODE_DTYPE = np.dtype([("code", "<u8"), ("seg_first", "<u8"), ("point_first", "<u8"), ("mass_lo", "<u8"),
                       ("mass_hi", "<u8"), ("seg_count", "<u4"), ("point_count", "<u4"),
                       ("child_first", "<u4"), ("child_count", "<u4"), ("depth", "<i4"), ("flags", "<i4"),
                       ("parent", "<i4"), ("pad", "<i4"), ("h_cull", "<f4"), ("w_rep", "<f4"),
                       ("s_rep", "<f4"), ("pad2", "<f4"), ("bmin", "<f4", (3,)), ("bmax", "<f4", (3,))])
assert NODE_DTYPE.itemsize == C.sizeof(Node)


class OracleTree:
    """Octree built by the oracle; numpy copies of everything plus the C handle."""

    def __init__(self, ptr, lo, side, n_max, seed):
        self._ptr = ptr
        T = ptr.contents
        self.lo, self.side, self.n_max, self.seed = np.asarray(lo, np.float64), float(side), n_max, seed
        self.n = int(T.n)
        nn, npt = int(T.n_nodes), int(T.n_pts)
        self.nodes = (np.frombuffer(C.string_at(T.nodes, nn * NODE_DTYPE.itemsize), NODE_DTYPE).copy()
                      if nn else np.zeros(0, NODE_DTYPE))
        self.pts4 = np.ctypeslib.as_array(T.pts4, (max(npt, 1) * 4,))[: npt * 4].reshape(npt, 4).copy()
        self.hs = np.ctypeslib.as_array(T.hs, (max(npt, 1),))[:npt].copy()
        self.pt_src = np.ctypeslib.as_array(T.pt_src, (max(npt, 1),))[:npt].copy() if T.pt_src else None
        n = self.n
        self.skey = np.ctypeslib.as_array(T.skey, (max(n, 1),))[:n].copy() if T.skey else None
        self.sidx = np.ctypeslib.as_array(T.sidx, (max(n, 1),))[:n].copy() if T.sidx else None
        self.depth_max = int(T.depth_max)
        self.equal_mass = bool(T.equal_mass)

    def __del__(self):
        if getattr(self, "_ptr", None) is not None and _lib is not None:
            _lib.orc_tree_free(self._ptr)
            self._ptr = None

    def set_points(self, node: int, pts4, hs):
        """Overwrites node `node`'s stored points (orc_tree_set_points) and refreshes these copies."""
        pts4 = np.ascontiguousarray(pts4, np.float32).reshape(-1, 4)
        hs = np.ascontiguousarray(hs, np.float32)
        st = lib().orc_tree_set_points(self._ptr, int(node), pts4.reshape(-1), hs, pts4.shape[0])
        if st != OK:
            raise OracleError(st)
        T = self._ptr.contents
        nn, npt = int(T.n_nodes), int(T.n_pts)
        self.nodes = np.frombuffer(C.string_at(T.nodes, nn * NODE_DTYPE.itemsize), NODE_DTYPE).copy()
        self.pts4 = np.ctypeslib.as_array(T.pts4, (max(npt, 1) * 4,))[: npt * 4].reshape(npt, 4).copy()
        self.hs = np.ctypeslib.as_array(T.hs, (max(npt, 1),))[:npt].copy()
        if T.pt_src:
            self.pt_src = np.ctypeslib.as_array(T.pt_src, (max(npt, 1),))[:npt].copy()

    def masses(self) -> np.ndarray:
        """Exact node masses as Python ints in units of 2^-47."""
        return [int(hi) << 64 | int(lo) for lo, hi in zip(self.nodes["mass_lo"], self.nodes["mass_hi"])]


def build_tree(xyz, mass, h, ids=None, seed=1, n_max=16000, lo=None, side=1.0):
    xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
    mass = np.ascontiguousarray(mass, np.float32)
    h = np.ascontiguousarray(h, np.float32)
    idp = None
    if ids is not None:
        ids = np.ascontiguousarray(ids, np.uint32)
        idp = ids.ctypes.data
    out = C.POINTER(Tree)()
    st = lib().orc_build(xyz, mass, h, idp, xyz.shape[0], seed, n_max, _lo(lo), side, C.byref(out))
    if st != OK:
        raise OracleError(st)
    return OracleTree(out, _lo(lo), side, n_max, seed)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle status {code}")
        self.code = code


def build_topdown(xyz, ids=None, n_max=16000, lo=None, side=1.0):
    xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
    idp = None
    if ids is not None:
        ids = np.ascontiguousarray(ids, np.uint32)
        idp = ids.ctypes.data
    nn, nm = C.c_uint64(), C.c_uint64()
    L = lib()
    L.orc_build_topdown(xyz, idp, xyz.shape[0], n_max, _lo(lo), side, C.byref(nn), C.byref(nm), None, None, None,
                        None, None)
    codes = np.zeros(nn.value, np.uint64)
    depths = np.zeros(nn.value, np.int32)
    counts = np.zeros(nn.value, np.uint32)
    flags = np.zeros(nn.value, np.int32)
    members = np.zeros(max(nm.value, 1), np.uint32)
    L.orc_build_topdown(xyz, idp, xyz.shape[0], n_max, _lo(lo), side, C.byref(nn), C.byref(nm), codes.ctypes.data,
                        depths.ctypes.data, counts.ctypes.data, flags.ctypes.data, members.ctypes.data)
    return dict(code=codes, depth=depths, count=counts, flags=flags, members=members[: nm.value])


def select_node(pos, ids, mass, code, seed, n_sel, equal_mass):
    pos = np.ascontiguousarray(pos, np.uint32)
    out = np.zeros(max(pos.size, 1), np.uint32)
    lib().orc_select_node(pos, np.ascontiguousarray(ids, np.uint32), np.ascontiguousarray(mass, np.float32),
                          pos.size, code, seed, n_sel, int(bool(equal_mass)), out)
    return out[:n_sel].copy()


def select(tree: OracleTree, cam: dict, rp: RParams) -> np.ndarray:
    out = np.zeros(max(len(tree.nodes), 1), np.uint32)
    m = lib().orc_select(tree._ptr, tree.lo, tree.side, C.byref(camera(cam)), C.byref(rp), out)
    return np.sort(out[:m])


def render_lod(tree: OracleTree, cam: dict, rp: RParams):
    acc = np.zeros(cam["height"] * cam["width"], np.uint64)
    nd, npnt = C.c_uint64(), C.c_uint64()
    st = lib().orc_render_lod(tree._ptr, tree.lo, tree.side, C.byref(camera(cam)), C.byref(rp), acc, C.byref(nd),
                              C.byref(npnt))
    return acc.reshape(cam["height"], cam["width"]), st, int(nd.value), int(npnt.value)


def render_lod_counted(tree: OracleTree, cam: dict, rp: RParams):
    """render_lod plus the frame's pixel updates ((splat, pixel) pairs inside the support)."""
    acc = np.zeros(cam["height"] * cam["width"], np.uint64)
    nd, npnt, nu = C.c_uint64(), C.c_uint64(), C.c_uint64()
    st = lib().orc_render_lod_counted(tree._ptr, tree.lo, tree.side, C.byref(camera(cam)), C.byref(rp), acc,
                                      C.byref(nd), C.byref(npnt), C.byref(nu))
    return acc.reshape(cam["height"], cam["width"]), st, int(nd.value), int(npnt.value), int(nu.value)


def render_lod_rows(tree: OracleTree, cam: dict, rp: RParams, row0: int, row1: int):
    """Rows [row0, row1) of render_lod's frame (the same values), with the frame's counts for those rows."""
    acc = np.zeros((row1 - row0) * cam["width"], np.uint64)
    nd, npnt, nu = C.c_uint64(), C.c_uint64(), C.c_uint64()
    st = lib().orc_render_lod_rows(tree._ptr, tree.lo, tree.side, C.byref(camera(cam)), C.byref(rp), int(row0),
                                   int(row1), acc, C.byref(nd), C.byref(npnt), C.byref(nu))
    return acc.reshape(row1 - row0, cam["width"]), st, int(nd.value), int(npnt.value), int(nu.value)


def render_lod_part(tree: OracleTree, cam: dict, rp: RParams, part: int, n_parts: int):
    """Part `part` of `n_parts` of render_lod's frame: the selected nodes with index = part (mod n_parts)."""
    acc = np.zeros(cam["height"] * cam["width"], np.uint64)
    nd, npnt = C.c_uint64(), C.c_uint64()
    st = lib().orc_render_lod_part(tree._ptr, tree.lo, tree.side, C.byref(camera(cam)), C.byref(rp), int(part),
                                   int(n_parts), acc, C.byref(nd), C.byref(npnt))
    return acc.reshape(cam["height"], cam["width"]), st, int(nd.value), int(npnt.value)


def splat_particles(xyz, mass, h, cam: dict, rp: RParams):
    xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
    acc = np.zeros(cam["height"] * cam["width"], np.uint64)
    nd = C.c_uint64()
    st = lib().orc_splat_particles(xyz, np.ascontiguousarray(mass, np.float32), np.ascontiguousarray(h, np.float32),
                                   xyz.shape[0], C.byref(camera(cam)), C.byref(rp), acc, C.byref(nd))
    return acc.reshape(cam["height"], cam["width"]), st, int(nd.value)


def splat_points(pts4, hs, cam: dict, rp: RParams):
    pts4 = np.ascontiguousarray(pts4, np.float32).reshape(-1, 4)
    acc = np.zeros(cam["height"] * cam["width"], np.uint64)
    nd = C.c_uint64()
    st = lib().orc_splat_points(pts4, np.ascontiguousarray(hs, np.float32), pts4.shape[0], C.byref(camera(cam)),
                                C.byref(rp), acc, C.byref(nd))
    return acc.reshape(cam["height"], cam["width"]), st, int(nd.value)


def count_updates(pts4, hs, cam: dict, rp: RParams) -> int:
    """Pixel updates of drawing the points: (splat, pixel) pairs with a table index below 1024."""
    pts4 = np.ascontiguousarray(pts4, np.float32).reshape(-1, 4)
    return int(lib().orc_count_updates(pts4, np.ascontiguousarray(hs, np.float32), pts4.shape[0],
                                       C.byref(camera(cam)), C.byref(rp)))


def pixel_value(pts4, hs, cam: dict, rp: RParams, px: int, py: int) -> int:
    pts4 = np.ascontiguousarray(pts4, np.float32).reshape(-1, 4)
    return int(lib().orc_pixel_value(pts4, np.ascontiguousarray(hs, np.float32), pts4.shape[0],
                                     C.byref(camera(cam)), C.byref(rp), px, py))


def block_quantize(tree: OracleTree):
    """16-bit block codes of every stored point (storage paragraph): returns codes (n_pts x 5 uint16:
    x, y, z, w, h), per-node constants (n_nodes x 8 float32: qlo x y z, qstep, w lo, w step, h lo,
    h step) and the decoded tree (same nodes, decoded points, bounds and h_cull of the decoded
    subtrees)."""
    npt, nn = len(tree.pts4), len(tree.nodes)
    codes = np.zeros((max(npt, 1), 5), np.uint16)
    qa = np.zeros((max(nn, 1), 8), np.float32)
    out = C.POINTER(Tree)()
    st = lib().orc_block_quantize(tree._ptr, tree.lo, tree.side, codes, qa, C.byref(out))
    if st != 0:
        raise RuntimeError(f"orc_block_quantize failed: {st}")
    return codes[:npt], qa[:nn], OracleTree(out, tree.lo, tree.side, tree.n_max, tree.seed)


def block_code_pos(x, lo: float, step: float) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32).reshape(-1)
    out = np.zeros(max(x.size, 1), np.uint16)
    lib().orc_block_code_pos(x, x.size, lo, step, out)
    return out[: x.size]


def block_decode_pos(c, lo: float, step: float) -> np.ndarray:
    c = np.ascontiguousarray(c, np.uint16).reshape(-1)
    out = np.zeros(max(c.size, 1), np.float32)
    lib().orc_block_decode_pos(c, c.size, lo, step, out)
    return out[: c.size]


def block_code_lin(v, lo: float, step: float) -> np.ndarray:
    v = np.ascontiguousarray(v, np.float32).reshape(-1)
    out = np.zeros(max(v.size, 1), np.uint16)
    lib().orc_block_code_lin(v, v.size, lo, step, out)
    return out[: v.size]


def block_decode_lin(c, lo: float, step: float) -> np.ndarray:
    c = np.ascontiguousarray(c, np.uint16).reshape(-1)
    out = np.zeros(max(c.size, 1), np.float32)
    lib().orc_block_decode_lin(c, c.size, lo, step, out)
    return out[: c.size]


def tonemap(acc, rp: RParams) -> np.ndarray:
    acc = np.ascontiguousarray(acc, np.uint64)
    out = np.zeros(acc.size, np.uint8)
    lib().orc_tonemap(acc.reshape(-1), acc.size, C.byref(rp), out)
    return out.reshape(acc.shape)
