"""Allocation failure through the C ABI's allocator hook (host-injected: the hook refuses once a byte
budget is spent; no GPU fault is involved).  A build, a frame and a batch reservation that run out
mid-way must return GBLOD_ERR_OOM, leave their out-parameters untouched and give back every byte
they took; the objects involved stay usable afterwards."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Budget:
    """Device memory from torch's caching allocator, refused once `budget` bytes are live."""

    def __init__(self, budget):
        self.budget, self.live, self.used, self.peak, self.refused = budget, {}, 0, 0, 0
        self._a, self._f = ALLOC(self.alloc), FREE(self.free)

    def alloc(self, nbytes, stream, ctx):
        if self.used + nbytes > self.budget:
            self.refused += 1
            return None
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        self.used += t.numel()
        self.peak = max(self.peak, self.used)
        return t.data_ptr()

    def free(self, ptr, nbytes, stream, ctx):
        t = self.live.pop(ptr)
        self.used -= t.numel()

    def hook(self):
        from paper_0811_2055_gb300 import gblod
        return gblod.Allocator(C.cast(self._a, C.c_void_p), C.cast(self._f, C.c_void_p), None)


def _inputs():
    from paper_0811_2055_gb300 import synth
    p = synth.tiny(200000, seed=41)
    dev = torch.device("cuda", 0)
    return p, [torch.from_numpy(a).to(dev) for a in (p.xyz, p.mass, p.h)]


def _build(L, xyz, mass, h, n, hook, out):
    from paper_0811_2055_gb300 import gblod
    bp = gblod.BuildParams()
    bp.seed, bp.n_max = 1, 2000
    bp.root_lo[:] = [0.0, 0.0, 0.0]
    bp.root_side = 1.0
    return L.gblod_build_lod(xyz.data_ptr(), mass.data_ptr(), h.data_ptr(), None, n, C.byref(bp),
                             C.byref(hook) if hook is not None else None,
                             torch.cuda.current_stream().cuda_stream, C.byref(out))


def test_build_out_of_memory_leaks_nothing():
    from paper_0811_2055_gb300 import gblod
    torch.cuda.set_device(0)
    L = gblod.lib()
    p, (xyz, mass, h) = _inputs()
    full = Budget(1 << 40)
    out = C.c_void_p()
    assert _build(L, xyz, mass, h, p.n, full.hook(), out) == gblod.OK
    assert full.used > 0 and out.value
    L.gblod_octree_free(out)
    torch.cuda.synchronize()
    assert full.used == 0 and not full.live
    for frac in (0.05, 0.3, 0.6, 0.9):
        b = Budget(int(full.peak * frac))
        sentinel = C.c_void_p(0x1234)
        st = _build(L, xyz, mass, h, p.n, b.hook(), sentinel)
        torch.cuda.synchronize()
        assert st == gblod.ERR_OOM, (frac, st)
        assert b.refused >= 1
        assert sentinel.value == 0x1234            # out-parameter untouched
        assert b.used == 0 and not b.live, frac    # every byte given back
    # the library is still usable: a build with enough budget succeeds and matches the unhooked one
    ok = Budget(1 << 40)
    out2 = C.c_void_p()
    assert _build(L, xyz, mass, h, p.n, ok.hook(), out2) == gblod.OK
    t2 = gblod.Octree(out2.value)
    t0 = gblod.build_lod(xyz, mass, h, n_max=2000, seed=1)
    a, b = t2.export(), t0.export()
    assert np.array_equal(a["nodes"], b["nodes"]) and np.array_equal(a["pts4"], b["pts4"])
    t2.free()
    t0.free()
    torch.cuda.synchronize()
    assert ok.used == 0


def test_frame_and_batch_reservation_out_of_memory():
    from paper_0811_2055_gb300 import gblod, synth
    torch.cuda.set_device(0)
    L = gblod.lib()
    p, (xyz, mass, h) = _inputs()
    tree = gblod.build_lod(xyz, mass, h, n_max=2000, seed=1)
    cam = synth.look_at((0.5, 0.5, -0.6), (0.5, 0.5, 0.5), width=640, height=480)
    par = gblod.make_params(lambda_px=8.0)
    want_img, want_acc = gblod.Renderer().render(tree, cam, par)
    b = Budget(64 << 10)  # far too small for the frame's records
    r = C.c_void_p()
    assert L.gblod_renderer_create(C.byref(b.hook()), C.byref(r)) == gblod.OK
    acc = torch.zeros((480, 640), dtype=torch.int64, device="cuda")
    c = gblod.make_camera(cam)
    stream = torch.cuda.current_stream().cuda_stream
    st = L.gblod_render(r, tree.handle, C.byref(c), C.byref(par), None, acc.data_ptr(), stream)
    torch.cuda.synchronize()
    assert st == gblod.ERR_OOM and b.refused >= 1
    # reserving batch scratch beyond the budget fails the same way
    views = (gblod.View * 2)()
    for k in range(2):
        views[k].octree = tree.handle
        views[k].camera = c
        views[k].d_image = None
        views[k].d_accum = acc.data_ptr()
    st = L.gblod_renderer_reserve_batch(r, views, 2, C.byref(par), 1 << 26, stream)
    torch.cuda.synchronize()
    assert st == gblod.ERR_OOM
    # with the budget raised the same renderer draws the frame exactly
    b.budget = 1 << 40
    st = L.gblod_render(r, tree.handle, C.byref(c), C.byref(par), None, acc.data_ptr(), stream)
    torch.cuda.synchronize()
    assert st == gblod.OK and torch.equal(acc, want_acc)
    L.gblod_renderer_destroy(r)
    torch.cuda.synchronize()
    assert b.used == 0 and not b.live
    tree.free()
