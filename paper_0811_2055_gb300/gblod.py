"""Thin Python binding of libgblod (include/gblod.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; torch supplies device memory and the
current stream.  Importing this module raises if libgblod.so has not been built, so nothing can
silently fall back to another implementation.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgblod.so")

OK, ERR_INVALID_ARG, ERR_RANGE, ERR_OOM, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_NOT_IMPLEMENTED, ERR_CAPACITY = range(8)
NODE_LEAF, NODE_INTERNAL, NODE_LOSSY, NODE_REPS = 1, 2, 4, 8
KERNEL_GAUSSIAN, KERNEL_CUBIC = 0, 1
POINTS_FLOAT, POINTS_BLOCK16 = 0, 1
RENDER_COUNT_UPDATES = 1
QUANTIZE_DROP_FLOAT = 1
(K_ANY, K_MORTON, K_SORT_UPSWEEP, K_SORT_SCATTER, K_SCAN, K_BUILD_OTHER, K_SEL_HIST, K_SEL_MARK, K_SEL_WRITE,
 K_SELECT_NODES, K_PROJECT_COUNT, K_PROJECT_SCATTER, K_SPLAT, K_TONEMAP, K_RENDER_OTHER) = range(15)

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")


class GblodError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: status {code}: {msg}")
        self.code = code


class BuildParams(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("n_max", C.c_uint32), ("reserved", C.c_uint32),
                ("root_lo", C.c_double * 3), ("root_side", C.c_double)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("right", C.c_double * 3), ("up", C.c_double * 3),
                ("fwd", C.c_double * 3), ("f_px", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("z_near", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class RenderParams(C.Structure):
    _fields_ = [("lambda_px", C.c_double), ("sigma_min_px", C.c_double), ("sigma_max_px", C.c_double),
                ("tone_lo", C.c_double), ("tone_hi", C.c_double), ("kernel", C.c_int32),
                ("tone_auto", C.c_int32), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("record_budget", C.c_uint64), ("point_format", C.c_int32), ("flags", C.c_int32)]


class View(C.Structure):
    _fields_ = [("octree", C.c_void_p), ("camera", Camera), ("d_image", C.c_void_p), ("d_accum", C.c_void_p)]


class OctreeInfo(C.Structure):
    _fields_ = [("n_particles", C.c_uint64), ("n_nodes", C.c_uint64), ("n_points", C.c_uint64),
                ("device_bytes", C.c_uint64), ("depth_max", C.c_int32), ("equal_mass", C.c_int32),
                ("n_max", C.c_uint32), ("formats", C.c_uint32)]


class FrameStats(C.Structure):
    _fields_ = [("nodes_selected", C.c_uint64), ("points", C.c_uint64), ("splats", C.c_uint64),
                ("pairs", C.c_uint64), ("tiles", C.c_uint64), ("amplitude_lo", C.c_uint64),
                ("amplitude_hi", C.c_uint64), ("pixel_updates", C.c_uint64), ("pixel_updates_total", C.c_uint64)]


class Allocator(C.Structure):
    _fields_ = [("alloc", C.c_void_p), ("free", C.c_void_p), ("ctx", C.c_void_p)]


NODE_DTYPE = np.dtype([("code", "<u8"), ("seg_first", "<u8"), ("point_first", "<u8"), ("mass_lo", "<u8"),
                       ("mass_hi", "<u8"), ("seg_count", "<u4"), ("point_count", "<u4"),
                       ("child_first", "<u4"), ("child_count", "<u4"), ("depth", "<i4"), ("flags", "<i4"),
                       ("parent", "<i4"), ("pad", "<i4"), ("h_cull", "<f4"), ("w_rep", "<f4"),
                       ("s_rep", "<f4"), ("pad2", "<f4"), ("bmin", "<f4", (3,)), ("bmax", "<f4", (3,))])
assert NODE_DTYPE.itemsize == 112

_L = C.CDLL(LIB_PATH)
_vp, _u64, _u32, _i32, _d = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int32, C.c_double
_L.gblod_build_lod.argtypes = [_vp, _vp, _vp, _vp, _u64, C.POINTER(BuildParams), _vp, _vp, C.POINTER(_vp)]
_L.gblod_octree_free.argtypes = [_vp]
_L.gblod_octree_free.restype = None
_L.gblod_octree_get_info.argtypes = [_vp, C.POINTER(OctreeInfo)]
_L.gblod_octree_export.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp]
_L.gblod_octree_quantize.argtypes = [_vp, _u32, _vp]
_L.gblod_octree_export_block16.argtypes = [_vp, _vp, _vp, _vp]
_L.gblod_renderer_create.argtypes = [_vp, C.POINTER(_vp)]
_L.gblod_renderer_destroy.argtypes = [_vp]
_L.gblod_renderer_destroy.restype = None
_L.gblod_render.argtypes = [_vp, _vp, C.POINTER(Camera), C.POINTER(RenderParams), _vp, _vp, _vp]
_L.gblod_render_bruteforce.argtypes = [_vp, _vp, _vp, _vp, _u64, C.POINTER(Camera), C.POINTER(RenderParams), _vp,
                                       _vp, _vp]
_L.gblod_renderer_status.argtypes = [_vp, _vp, C.c_int]
_L.gblod_renderer_stats.argtypes = [_vp, _vp, C.POINTER(FrameStats)]
_L.gblod_renderer_last_selection.argtypes = [_vp, _vp, _vp, _u64, C.POINTER(_u64)]
_L.gblod_morton_keys.argtypes = [_vp, _u64, C.POINTER(_d), _d, _vp, _vp]
_L.gblod_renderer_reserve_batch.argtypes = [_vp, C.POINTER(View), _i32, C.POINTER(RenderParams), _u64, _vp]
_L.gblod_render_batch.argtypes = [_vp, C.POINTER(View), _i32, C.POINTER(RenderParams), _vp]
_L.gblod_autotune_tiles.argtypes = [_vp, C.POINTER(View), _i32, C.POINTER(RenderParams), _u64, _vp,
                                    C.POINTER(_d)]
_L.gblod_autotune_cache_clear.argtypes = []
_L.gblod_autotune_cache_clear.restype = None
_L.gblod_project.argtypes = [_vp, _vp, _u64, C.POINTER(Camera), C.POINTER(RenderParams), _vp, _vp]
_L.gblod_diff_render.argtypes = [_vp, _vp, _vp, _vp, _u64, C.POINTER(Camera), _i32, C.POINTER(RenderParams), _vp,
                                 _vp]
_L.gblod_diff_backward.argtypes = [_vp, _vp, _vp, _vp, _u64, C.POINTER(Camera), _i32, C.POINTER(RenderParams), _vp,
                                   _vp, _vp, _vp, _vp]
_L.gblod_launch_count.restype = _u64
_L.gblod_trim_cache.argtypes = [_u64]
_L.gblod_probe_enable.argtypes = [_i32]
_L.gblod_probe_read.argtypes = [C.POINTER(_d), C.POINTER(_u64)]
_L.gblod_microbench.argtypes = [_i32, C.c_uint32, _vp, C.POINTER(_d), C.POINTER(_d)]
_L.gblod_octree_node_points.argtypes = [_vp, _u32, _vp, _vp, C.POINTER(_u32), _vp]
_L.gblod_octree_node_members.argtypes = [_vp, _u32, _vp, C.POINTER(_u32), _vp]
_L.gblod_octree_set_points.argtypes = [_vp, _u32, _vp, _vp, _u32, _vp]
_L.gblod_render_part.argtypes = [_vp, _vp, C.POINTER(Camera), C.POINTER(RenderParams), _i32, _i32, _vp, _vp]
_L.gblod_tonemap.argtypes = [_vp, _vp, _i32, _i32, C.POINTER(RenderParams), _vp, _vp]
_L.gblod_status_string.restype = C.c_char_p
_L.gblod_status_string.argtypes = [C.c_int]
_L.gblod_last_error.restype = C.c_char_p
for _f in ("gblod_build_lod", "gblod_octree_get_info", "gblod_octree_export", "gblod_renderer_create",
           "gblod_render", "gblod_render_bruteforce", "gblod_renderer_status", "gblod_renderer_stats",
           "gblod_renderer_last_selection", "gblod_morton_keys", "gblod_project", "gblod_probe_enable",
           "gblod_probe_read", "gblod_renderer_reserve_batch", "gblod_render_batch", "gblod_autotune_tiles",
           "gblod_diff_render", "gblod_diff_backward", "gblod_octree_quantize", "gblod_octree_export_block16",
           "gblod_microbench", "gblod_render_part", "gblod_tonemap", "gblod_octree_node_points",
           "gblod_octree_node_members", "gblod_octree_set_points", "gblod_trim_cache"):
    getattr(_L, _f).restype = C.c_int


def lib() -> C.CDLL:
    return _L


def _check(st: int, where: str):
    if st != OK:
        raise GblodError(st, where, _L.gblod_last_error().decode(errors="replace"))


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return int(t.data_ptr())


def make_camera(cam: dict) -> Camera:
    c = Camera()
    for k in ("eye", "right", "up", "fwd"):
        getattr(c, k)[:] = [float(v) for v in cam[k]]
    c.f_px, c.cx, c.cy, c.z_near = float(cam["f_px"]), float(cam["cx"]), float(cam["cy"]), float(cam["z_near"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


def make_params(lambda_px=None, sigma_min_px=0.5, sigma_max_px=128.0, kernel=KERNEL_GAUSSIAN, tone_auto=True,
                tone_lo=0.0, tone_hi=0.0, tile_w=0, tile_h=0, record_budget=0,
                point_format=POINTS_FLOAT, count_updates=False) -> RenderParams:
    p = RenderParams()
    p.lambda_px = -1.0 if lambda_px is None else float(lambda_px)
    p.sigma_min_px, p.sigma_max_px = float(sigma_min_px), float(sigma_max_px)
    p.tone_lo, p.tone_hi = float(tone_lo), float(tone_hi)
    p.kernel, p.tone_auto = int(kernel), int(bool(tone_auto))
    p.tile_w, p.tile_h = int(tile_w), int(tile_h)
    p.record_budget = int(record_budget)
    p.point_format = int(point_format)
    p.flags = RENDER_COUNT_UPDATES if count_updates else 0
    return p


# ------------------------------------------------------------------ octree

class Octree:
    """Device-resident octree built by gblod_build_lod."""

    def __init__(self, handle: int, root_lo=(0.0, 0.0, 0.0), root_side: float = 1.0):
        self._h = handle
        self.root = (tuple(float(v) for v in root_lo), float(root_side))

    def export_nodes(self) -> np.ndarray:
        """Host copy of the node table only."""
        nodes = np.zeros(int(self.info().n_nodes), NODE_DTYPE)
        _check(_L.gblod_octree_export(self._h, nodes.ctypes.data, None, None, None, None, None),
               "gblod_octree_export")
        return nodes

    @property
    def handle(self) -> int:
        return self._h

    def info(self) -> OctreeInfo:
        i = OctreeInfo()
        _check(_L.gblod_octree_get_info(self._h, C.byref(i)), "gblod_octree_get_info")
        return i

    def node_points(self, node: int, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
        """(count x 4 float32 points x, y, z, weight; count float32 h) stored in `node`, on the device."""
        n = _u32()
        _check(_L.gblod_octree_node_points(self._h, int(node), None, None, C.byref(n), _stream(stream)),
               "gblod_octree_node_points")
        dev = torch.device("cuda", torch.cuda.current_device())
        p4 = torch.empty((int(n.value), 4), dtype=torch.float32, device=dev)
        hs = torch.empty(int(n.value), dtype=torch.float32, device=dev)
        if n.value:
            _check(_L.gblod_octree_node_points(self._h, int(node), _ptr(p4), _ptr(hs), C.byref(n), _stream(stream)),
                   "gblod_octree_node_points")
        return p4, hs

    def node_members(self, node: int, stream=None) -> torch.Tensor:
        """Input indices (ids) of the node's member particles, int32 on the device."""
        n = _u32()
        _check(_L.gblod_octree_node_members(self._h, int(node), None, C.byref(n), _stream(stream)),
               "gblod_octree_node_members")
        ids = torch.empty(int(n.value), dtype=torch.int32, device=torch.device("cuda", torch.cuda.current_device()))
        if n.value:
            _check(_L.gblod_octree_node_members(self._h, int(node), _ptr(ids), C.byref(n), _stream(stream)),
                   "gblod_octree_node_members")
        return ids

    def set_points(self, node: int, pts4: torch.Tensor, hs: torch.Tensor, stream=None):
        """Overwrites the node's stored points (gblod_octree_set_points)."""
        assert pts4.dtype == torch.float32 and hs.dtype == torch.float32 and pts4.shape[1] == 4
        _check(_L.gblod_octree_set_points(self._h, int(node), _ptr(pts4.contiguous()), _ptr(hs.contiguous()),
                                          int(pts4.shape[0]), _stream(stream)), "gblod_octree_set_points")

    def export(self) -> dict:
        i = self.info()
        nn, npt, n = int(i.n_nodes), int(i.n_points), int(i.n_particles)
        nodes = np.zeros(nn, NODE_DTYPE)
        pts4 = np.zeros((npt, 4), np.float32)
        hs = np.zeros(npt, np.float32)
        src = np.zeros(npt, np.uint32)
        skey = np.zeros(n, np.uint64)
        sidx = np.zeros(n, np.uint32)
        _check(_L.gblod_octree_export(self._h, nodes.ctypes.data, pts4.ctypes.data, hs.ctypes.data, src.ctypes.data,
                                      skey.ctypes.data, sidx.ctypes.data), "gblod_octree_export")
        return dict(nodes=nodes, pts4=pts4, hs=hs, pt_src=src, skey=skey, sidx=sidx, depth_max=int(i.depth_max),
                    equal_mass=bool(i.equal_mass), n_max=int(i.n_max))

    def quantize(self, drop_float: bool = False, stream=None) -> "Octree":
        """Codes every stored point as 16-bit block codes (gblod_octree_quantize)."""
        _check(_L.gblod_octree_quantize(self._h, QUANTIZE_DROP_FLOAT if drop_float else 0, _stream(stream)),
               "gblod_octree_quantize")
        return self

    def export_block16(self) -> dict:
        i = self.info()
        nn, npt = int(i.n_nodes), int(i.n_points)
        codes = np.zeros((max(npt, 1), 5), np.uint16)
        qa = np.zeros((max(nn, 1), 8), np.float32)
        qnodes = np.zeros(max(nn, 1), NODE_DTYPE)
        _check(_L.gblod_octree_export_block16(self._h, codes.ctypes.data, qa.ctypes.data, qnodes.ctypes.data),
               "gblod_octree_export_block16")
        return dict(codes=codes[:npt], qa=qa[:nn], qnodes=qnodes[:nn])

    def free(self):
        if self._h:
            _L.gblod_octree_free(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_lod(xyz: torch.Tensor, mass: torch.Tensor, h: torch.Tensor, ids: torch.Tensor | None = None,
              n_max: int = 16000, seed: int = 1, root_lo=(0.0, 0.0, 0.0), root_side: float = 1.0,
              stream=None) -> Octree:
    n = int(xyz.shape[0]) if xyz.numel() else 0
    assert xyz.dtype == torch.float32 and mass.dtype == torch.float32 and h.dtype == torch.float32
    if ids is not None:
        assert ids.dtype in (torch.int32,) and ids.numel() == n
    p = BuildParams()
    p.seed, p.n_max = int(seed), int(n_max)
    p.root_lo[:] = [float(v) for v in root_lo]
    p.root_side = float(root_side)
    out = _vp()
    _check(_L.gblod_build_lod(_ptr(xyz) if n else None, _ptr(mass) if n else None, _ptr(h) if n else None,
                              _ptr(ids) if ids is not None and n else None, n, C.byref(p), None, _stream(stream),
                              C.byref(out)), "gblod_build_lod")
    return Octree(out.value, root_lo, root_side)


# ------------------------------------------------------------------ rendering

class Renderer:
    """Render workspace (gblod_renderer)."""

    def __init__(self):
        h = _vp()
        _check(_L.gblod_renderer_create(None, C.byref(h)), "gblod_renderer_create")
        self._h = h.value

    def render(self, octree: Octree, cam: dict, params: RenderParams | None = None, image=True, accum=None,
               stream=None):
        """LOD frame; returns (uint8 image or None, int64 accumulator tensor viewed as the u64 image)."""
        return self._frame(octree, None, cam, params, image, accum, stream)

    def render_part(self, octree: Octree, cam: dict, part: int, n_parts: int, params: RenderParams | None = None,
                    accum=None, stream=None) -> torch.Tensor:
        """Partial accumulation image of part `part` of `n_parts` of a split frame (gblod_render_part)."""
        params = params if params is not None else make_params()
        W, H = int(cam["width"]), int(cam["height"])
        acc = torch.empty((H, W), dtype=torch.int64, device=torch.device("cuda", torch.cuda.current_device())) \
            if accum is None else accum
        c = make_camera(cam)
        _check(_L.gblod_render_part(self._h, octree.handle, C.byref(c), C.byref(params), int(part), int(n_parts),
                                    _ptr(acc), _stream(stream)), "gblod_render_part")
        return acc

    def tonemap(self, accum: torch.Tensor, params: RenderParams | None = None, image=None, stream=None):
        """8-bit log tone map of an accumulation image (gblod_tonemap)."""
        params = params if params is not None else make_params()
        H, W = int(accum.shape[0]), int(accum.shape[1])
        img = torch.empty((H, W), dtype=torch.uint8, device=accum.device) if image is None else image
        _check(_L.gblod_tonemap(self._h, _ptr(accum), W, H, C.byref(params), _ptr(img), _stream(stream)),
               "gblod_tonemap")
        return img

    def render_bruteforce(self, xyz, mass, h, cam: dict, params: RenderParams | None = None, image=True,
                          accum=None, stream=None):
        return self._frame(None, (xyz, mass, h), cam, params, image, accum, stream)

    def _frame(self, octree, parts, cam, params, image, accum, stream):
        params = params if params is not None else make_params()
        W, H = int(cam["width"]), int(cam["height"])
        dev = torch.device("cuda", torch.cuda.current_device())
        img = torch.empty((H, W), dtype=torch.uint8, device=dev) if image is True else image
        acc = torch.empty((H, W), dtype=torch.int64, device=dev) if accum is None else accum
        c = make_camera(cam)
        if octree is not None:
            st = _L.gblod_render(self._h, octree.handle, C.byref(c), C.byref(params), _ptr(img), _ptr(acc),
                                 _stream(stream))
            _check(st, "gblod_render")
        else:
            xyz, mass, h = parts
            n = int(xyz.shape[0])
            st = _L.gblod_render_bruteforce(self._h, _ptr(xyz) if n else None, _ptr(mass) if n else None,
                                            _ptr(h) if n else None, n, C.byref(c), C.byref(params), _ptr(img),
                                            _ptr(acc), _stream(stream))
            _check(st, "gblod_render_bruteforce")
        return img, acc

    # ---- batched views: each view is (octree, camera dict, uint8 image tensor or None, int64 accum tensor)
    @staticmethod
    def _views(views):
        arr = (View * len(views))()
        for i, (octree, cam, img, acc) in enumerate(views):
            arr[i].octree = octree.handle
            arr[i].camera = make_camera(cam)
            arr[i].d_image = _ptr(img) if img is not None else None
            arr[i].d_accum = _ptr(acc)
        return arr

    def reserve_batch(self, views, params: RenderParams | None = None, record_capacity: int = 0, stream=None):
        params = params if params is not None else make_params()
        arr = self._views(views)
        _check(_L.gblod_renderer_reserve_batch(self._h, arr, len(views), C.byref(params), int(record_capacity),
                                               _stream(stream)), "gblod_renderer_reserve_batch")

    def render_batch(self, views, params: RenderParams | None = None, stream=None):
        params = params if params is not None else make_params()
        arr = self._views(views)
        _check(_L.gblod_render_batch(self._h, arr, len(views), C.byref(params), _stream(stream)),
               "gblod_render_batch")

    def autotune(self, views, params: RenderParams | None = None, record_capacity: int = 0, stream=None):
        params = params if params is not None else make_params()
        arr = self._views(views)
        best = _d()
        _check(_L.gblod_autotune_tiles(self._h, arr, len(views), C.byref(params), int(record_capacity),
                                       _stream(stream), C.byref(best)), "gblod_autotune_tiles")
        return params, float(best.value)

    @staticmethod
    def autotune_cache_clear():
        _L.gblod_autotune_cache_clear()

    def status(self, reset: bool = True, stream=None) -> int:
        return int(_L.gblod_renderer_status(self._h, _stream(stream), int(reset)))

    def stats(self, stream=None) -> dict:
        s = FrameStats()
        _check(_L.gblod_renderer_stats(self._h, _stream(stream), C.byref(s)), "gblod_renderer_stats")
        return {k: int(getattr(s, k)) for k, _ in FrameStats._fields_}

    def last_selection(self, stream=None) -> np.ndarray:
        cnt = _u64()
        _check(_L.gblod_renderer_last_selection(self._h, _stream(stream), None, 0, C.byref(cnt)),
               "gblod_renderer_last_selection")
        out = np.zeros(max(int(cnt.value), 1), np.uint32)
        _check(_L.gblod_renderer_last_selection(self._h, _stream(stream), out.ctypes.data, out.size, C.byref(cnt)),
               "gblod_renderer_last_selection")
        return np.sort(out[: int(cnt.value)])

    def close(self):
        if self._h:
            _L.gblod_renderer_destroy(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _cams(cams):
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = make_camera(c)
    return arr


def diff_render(r: Renderer, xyz, w, logh, cams, params: RenderParams | None = None, stream=None) -> torch.Tensor:
    """Float splat images (n_views, H, W) of points (xyz n x 3, w, logh), see gblod_diff_render."""
    params = params if params is not None else make_params()
    n = int(xyz.shape[0])
    H, W = int(cams[0]["height"]), int(cams[0]["width"])
    img = torch.empty((len(cams), H, W), dtype=torch.float32, device=xyz.device)
    _check(_L.gblod_diff_render(r._h, _ptr(xyz), _ptr(w), _ptr(logh), n, _cams(cams), len(cams), C.byref(params),
                                _ptr(img), _stream(stream)), "gblod_diff_render")
    return img


def diff_backward(r: Renderer, xyz, w, logh, cams, grad_images, params: RenderParams | None = None, stream=None):
    """dL/dxyz, dL/dw, dL/dlogh from dL/dI (gblod_diff_backward)."""
    params = params if params is not None else make_params()
    n = int(xyz.shape[0])
    gx, gw, gl = torch.empty_like(xyz), torch.empty_like(w), torch.empty_like(logh)
    grad_images = grad_images.contiguous()
    _check(_L.gblod_diff_backward(r._h, _ptr(xyz), _ptr(w), _ptr(logh), n, _cams(cams), len(cams), C.byref(params),
                                  _ptr(grad_images), _ptr(gx), _ptr(gw), _ptr(gl), _stream(stream)),
           "gblod_diff_backward")
    return gx, gw, gl


class SplatImages(torch.autograd.Function):
    """images = SplatImages.apply(xyz, w, logh, cams, renderer, params): differentiable float splat
    whose backward is the library's adjoint kernel (recomputation, nothing stored per pixel)."""

    @staticmethod
    def forward(ctx, xyz, w, logh, cams, renderer, params):
        xyz, w, logh = xyz.contiguous(), w.contiguous(), logh.contiguous()
        ctx.save_for_backward(xyz, w, logh)
        ctx.cams, ctx.renderer, ctx.params = cams, renderer, params
        return diff_render(renderer, xyz, w, logh, cams, params)

    @staticmethod
    def backward(ctx, grad):
        xyz, w, logh = ctx.saved_tensors
        gx, gw, gl = diff_backward(ctx.renderer, xyz, w, logh, ctx.cams, grad, ctx.params)
        return gx, gw, gl, None, None, None


def morton_keys(xyz: torch.Tensor, root_lo=(0.0, 0.0, 0.0), root_side: float = 1.0, stream=None) -> torch.Tensor:
    n = int(xyz.shape[0])
    keys = torch.empty(n, dtype=torch.int64, device=xyz.device)
    lo = (C.c_double * 3)(*[float(v) for v in root_lo])
    _check(_L.gblod_morton_keys(_ptr(xyz), n, lo, float(root_side), _ptr(keys), _stream(stream)), "gblod_morton_keys")
    return keys


def project(pts4: torch.Tensor, h: torch.Tensor, cam: dict, params: RenderParams | None = None,
            stream=None) -> torch.Tensor:
    n = int(pts4.shape[0])
    out = torch.empty((n, 5), dtype=torch.int64, device=pts4.device)
    params = params if params is not None else make_params()
    c = make_camera(cam)
    _check(_L.gblod_project(_ptr(pts4), _ptr(h), n, C.byref(c), C.byref(params), _ptr(out), _stream(stream)),
           "gblod_project")
    return out


def launch_count() -> int:
    return int(_L.gblod_launch_count())


def trim_cache(keep_bytes: int = 0):
    """Returns the device memory the library's pool keeps cached (beyond keep_bytes) to the device."""
    _check(_L.gblod_trim_cache(int(keep_bytes)), "gblod_trim_cache")


def probe_enable(kernel: int):
    _check(_L.gblod_probe_enable(int(kernel)), "gblod_probe_enable")


def probe_read() -> tuple[float, int]:
    ms, n = _d(), _u64()
    _check(_L.gblod_probe_read(C.byref(ms), C.byref(n)), "gblod_probe_read")
    return float(ms.value), int(n.value)


MB_ALU, MB_IMAD, MB_IMAD_WIDE, MB_IMAD_HI, MB_LDS, MB_RADIAL, MB_SEPARABLE = range(7)


def microbench(kind: int, iters: int = 4096, stream=None) -> tuple[float, float]:
    """(device ms, operations or pixel updates) of one timed launch of an issue-rate probe."""
    ms, units = _d(), _d()
    _check(_L.gblod_microbench(int(kind), int(iters), _stream(stream), C.byref(ms), C.byref(units)),
           "gblod_microbench")
    return float(ms.value), float(units.value)


def u64(t: torch.Tensor) -> np.ndarray:
    """Host copy of an int64 accumulator tensor, reinterpreted as uint64."""
    return t.detach().cpu().numpy().view(np.uint64)


def default_lambda(n_max: int) -> float:
    return math.sqrt(n_max)
