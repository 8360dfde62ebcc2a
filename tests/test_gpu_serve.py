"""Serving (NEXT-3 of the hot path): sessions admitted by an HBM budget, continuous batching over
two streams; every served frame equals the same view rendered alone, bit for bit, including
frames of batches that overflowed their record capacity and fell back to exact single views."""
import numpy as np
import pytest
import torch

from paper_0811_2055_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_0811_2055_gb300 import gblod
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = synth.timesteps_recipe(120_000)
    x0 = torch.from_numpy(base.xyz).to(dev)
    vel = torch.from_numpy(base.vel).to(dev)
    mass, h = torch.from_numpy(base.mass).to(dev), torch.from_numpy(base.h).to(dev)
    trees = []
    for t in range(3):
        xt = torch.remainder(x0 + t * vel, 1.0).contiguous()
        trees.append(gblod.build_lod(xt, mass, h, n_max=2000, seed=1))
    return gblod, trees


def _check_alone(gblod, trees, loop, done, k=12):
    r = gblod.Renderer()
    rng = np.random.default_rng(0)
    for i in rng.choice(len(done), min(k, len(done)), replace=False):
        rq = done[i]
        img, acc = r.render(trees[rq.timestep], rq.camera, loop.params)
        assert np.array_equal(img.cpu().numpy(), rq.image)
        assert np.array_equal(gblod.u64(acc), rq.accum)  # the 64-bit image, element by element
    r.close()


def test_serving_admits_by_budget_and_matches_views_alone(setup):
    from paper_0811_2055_gb300 import serve
    gblod, trees = setup
    res_choices = [(160, 120), (320, 180), (256, 256)]
    res, reqs = serve.poisson_requests(6, 20.0, 1.5, len(trees), res_choices, seed=1)
    need = [serve.ServingLoop.session_bytes(w, h, 2) for (w, h) in res]
    budget = sum(need[:5])  # the sixth session cannot fit
    loop = serve.ServingLoop(trees, hbm_budget_bytes=budget, max_views=8, keep_images=True,
                             record_capacity=1 << 22)
    admitted = [loop.admit(s, w, h) for s, (w, h) in enumerate(res)]
    assert admitted[:5] == [True] * 5 and not admitted[5]
    loop.reserve([(trees[0], synth.look_at((0.5, 0.5, -1), (0.5, 0.5, 0.5), width=320, height=256))] * 8)
    done = loop.run(reqs, 1.5)
    served = {q.session for q in done}
    assert 5 not in served and len(done) == sum(1 for q in reqs if q.session < 5)
    assert loop.stats["unserved"] == 0 and loop.stats["batches"] >= 2
    assert all(q.ready >= q.arrival for q in done)
    st = serve.latency_stats(done, 1.5)
    assert st["completed"] == len(done) and st["p99_ms"] >= st["p50_ms"] > 0
    _check_alone(gblod, trees, loop, done)
    loop.close()


def test_overflowing_batches_fall_back_to_exact_views(setup):
    from paper_0811_2055_gb300 import serve
    gblod, trees = setup
    res, reqs = serve.poisson_requests(3, 15.0, 1.0, len(trees), [(256, 192)], seed=2)
    loop = serve.ServingLoop(trees, hbm_budget_bytes=1 << 30, max_views=6, keep_images=True, record_capacity=2000)
    for s, (w, h) in enumerate(res):
        assert loop.admit(s, w, h)
    loop.reserve([(trees[0], synth.look_at((0.5, 0.5, -1), (0.5, 0.5, 0.5), width=256, height=192))] * 6)
    done = loop.run(reqs, 1.0)
    assert loop.stats["overflow_batches"] >= 1 and loop.stats["unserved"] == 0
    _check_alone(gblod, trees, loop, done)
    loop.close()


def test_full_size_timestep_batch_equals_views_alone():
    """One 75M-particle timestep of the serving workload at full size: a mixed-resolution batch of
    session views (720p, 1080p, 4K) renders every view exactly as it renders alone."""
    from paper_0811_2055_gb300 import gblod, serve
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = synth.timesteps_recipe()
    x0, vel = torch.from_numpy(base.xyz).to(dev), torch.from_numpy(base.vel).to(dev)
    mass, h = torch.from_numpy(base.mass).to(dev), torch.from_numpy(base.h).to(dev)
    del base
    xt = torch.remainder(x0 + 3 * vel, 1.0).contiguous()
    del x0, vel
    tree = gblod.build_lod(xt, mass, h, n_max=16000, seed=1)
    del xt, mass, h
    par = gblod.make_params()
    cams = [serve.session_camera(s, 1.5 * s, w, hh) for s, (w, hh) in
            enumerate([(1280, 720), (1920, 1080), (3840, 2160), (1920, 1080)])]
    single = gblod.Renderer()
    alone = []
    for cam in cams:
        img, acc = single.render(tree, cam, par)
        alone.append((img.cpu().numpy(), gblod.u64(acc).copy()))
    assert single.status() == gblod.OK
    views = [(tree, cam, torch.empty((cam["height"], cam["width"]), dtype=torch.uint8, device=dev),
              torch.empty((cam["height"], cam["width"]), dtype=torch.int64, device=dev)) for cam in cams]
    rb = gblod.Renderer()
    rb.reserve_batch(views, par, record_capacity=1 << 29)
    rb.render_batch(views, par)
    assert rb.status() == gblod.OK
    for (_, _, img, acc), (ai, aa) in zip(views, alone):
        assert np.array_equal(gblod.u64(acc), aa)
        assert np.array_equal(img.cpu().numpy(), ai)
    single.close()
    rb.close()
    tree.free()
