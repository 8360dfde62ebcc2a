"""The fixed-scratch brute-force entry point, through the C ABI.

gblod_render_bruteforce_noalloc exists for callers that cannot allocate device memory (a host
application that owns the whole device memory budget, a plug-in whose host forbids allocation, a
real-time loop that must not call cudaMalloc/cudaFree because they can block or synchronise).
Its scratch is one static device array in the library.  Checked here: on two calls in a row with
different inputs -- so a stale scratch from the first call would show in the second -- its
fixed-point image equals the allocating entry point's bit for bit (the tolerance every integer
image in these tests uses) and its 8-bit image is within +-1; oversized frames are rejected; no
torch allocation happens during the calls.  Runs alone or after the other tests.
"""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu


def _entry(lib):
    f = lib.gblod_render_bruteforce_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                  C.c_void_p]
    return f


def test_noalloc_matches_allocating_entry_point():
    from paper_0811_2055_gb300 import gblod, synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    f = _entry(gblod.lib())
    cases = [
        (synth.tiny(30000, seed=31), synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=320, height=200)),
        (synth.clustered(50000, 40, 0.1, 0.2, seed=32),
         synth.look_at((0.45, 0.55, 0.5), (0.9, 0.4, 0.6), width=333, height=197, z_near=1e-3)),
    ]
    ref = gblod.Renderer()
    params = gblod.make_params()
    stream = torch.cuda.current_stream()
    for p, cam in cases:
        xyz, mass, h = (torch.from_numpy(a).to(dev) for a in (p.xyz, p.mass, p.h))
        want_img, want_acc = ref.render_bruteforce(xyz, mass, h, cam, params)
        H, W = cam["height"], cam["width"]
        img = torch.full((H, W), 7, dtype=torch.uint8, device=dev)
        acc = torch.full((H, W), 12345, dtype=torch.int64, device=dev)
        c = gblod.make_camera(cam)
        torch.cuda.synchronize()
        before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        st = f(xyz.data_ptr(), mass.data_ptr(), h.data_ptr(), p.n, C.addressof(c), C.addressof(params),
               img.data_ptr(), acc.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        assert st == gblod.OK, gblod.lib().gblod_last_error()
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == before  # no torch allocation
        assert torch.equal(acc, want_acc)
        assert int((img.int() - want_img.int()).abs().max()) <= 1
        assert int(acc.count_nonzero()) > 1000
    ref.close()


def test_noalloc_rejects_frames_beyond_its_maximum():
    from paper_0811_2055_gb300 import gblod, synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    f = _entry(gblod.lib())
    p = synth.uniform(100, seed=2)
    xyz, mass, h = (torch.from_numpy(a).to(dev) for a in (p.xyz, p.mass, p.h))
    cam = synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=8192, height=8192)  # 65,536 tiles of 64x16
    acc = torch.zeros((16, 16), dtype=torch.int64, device=dev)
    c, params = gblod.make_camera(cam), gblod.make_params()
    st = f(xyz.data_ptr(), mass.data_ptr(), h.data_ptr(), p.n, C.addressof(c), C.addressof(params), None,
           acc.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == gblod.ERR_INVALID_ARG
    assert b"fixed maximum" in gblod.lib().gblod_last_error()
    # the caller must provide the accumulation output
    small = synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=64, height=64)
    c = gblod.make_camera(small)
    st = f(xyz.data_ptr(), mass.data_ptr(), h.data_ptr(), p.n, C.addressof(c), C.addressof(params), None, None,
           torch.cuda.current_stream().cuda_stream)
    assert st == gblod.ERR_INVALID_ARG


def test_noalloc_rejects_frames_beyond_its_record_maximum_then_still_matches():
    # a frame within the tile limit that needs more than GBLOD_NOALLOC_MAX_RECORDS (tile, splat)
    # records: 20,000 blobs of sigma ~ 100 px at 1920 x 1080 touch ~380 tiles each.  The count is
    # read back on the host before anything is scattered, so the call stops there with
    # GBLOD_ERR_RANGE; the next good call must still equal the allocating entry point.
    from paper_0811_2055_gb300 import gblod, synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    f = _entry(gblod.lib())
    big = synth.uniform(20000, seed=33, h=0.15)
    cam = synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=1920, height=1080)
    xyz, mass, h = (torch.from_numpy(a).to(dev) for a in (big.xyz, big.mass, big.h))
    acc = torch.zeros((1080, 1920), dtype=torch.int64, device=dev)
    c, params = gblod.make_camera(cam), gblod.make_params()
    stream = torch.cuda.current_stream()
    st = f(xyz.data_ptr(), mass.data_ptr(), h.data_ptr(), big.n, C.addressof(c), C.addressof(params), None,
           acc.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    assert st == gblod.ERR_RANGE
    assert b"fixed maximum" in gblod.lib().gblod_last_error()

    p = synth.tiny(40000, seed=34)
    small = synth.look_at((0.5, 0.45, -0.8), (0.5, 0.5, 0.5), width=640, height=360)
    xyz, mass, h = (torch.from_numpy(a).to(dev) for a in (p.xyz, p.mass, p.h))
    ref = gblod.Renderer()
    want_img, want_acc = ref.render_bruteforce(xyz, mass, h, small, params)
    acc = torch.full((360, 640), 99, dtype=torch.int64, device=dev)
    c = gblod.make_camera(small)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = f(xyz.data_ptr(), mass.data_ptr(), h.data_ptr(), p.n, C.addressof(c), C.addressof(params), None,
           acc.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    assert st == gblod.OK, gblod.lib().gblod_last_error()
    assert torch.cuda.mem_get_info()[0] == free0  # no device memory taken or kept by the call
    assert torch.equal(acc, want_acc) and int(acc.count_nonzero()) > 1000
    ref.close()
