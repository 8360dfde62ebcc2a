"""The library's own memory pool (no allocator hook): memory the library frees stays mapped in the
pool, so a second build of the same size takes no new device memory, and gblod_trim_cache returns
the cached memory to the device."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_pool_reuses_freed_memory_and_trim_returns_it():
    from paper_0811_2055_gb300 import gblod, synth

    torch.cuda.set_device(0)
    p = synth.clustered(1 << 21, 200, seed=41)
    d = [torch.from_numpy(a).cuda() for a in (p.xyz, p.mass, p.h)]
    torch.cuda.synchronize()
    gblod.trim_cache(0)
    t = gblod.build_lod(*d, n_max=4000, seed=1)
    nbytes = t.info().device_bytes
    want = t.export()["nodes"]
    t.free()
    torch.cuda.synchronize()
    f0 = torch.cuda.mem_get_info()[0]
    # the same build again: served from the memory the first one returned to the pool
    t = gblod.build_lod(*d, n_max=4000, seed=1)
    torch.cuda.synchronize()
    assert f0 - torch.cuda.mem_get_info()[0] <= 64 << 20
    assert (t.export()["nodes"] == want).all()
    t.free()
    torch.cuda.synchronize()
    gblod.trim_cache(0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] - f0 >= nbytes
