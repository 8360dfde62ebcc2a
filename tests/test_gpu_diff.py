"""Differentiation (NEXT-2 of the hot path): the float splat and its hand-written adjoint kernel
against the FP64 oracle (forward image, analytic gradient) and against FP64 central finite
differences of the oracle's forward on a 4,096-point / 64x64 subset, relative error <= 1e-3."""
import numpy as np
import pytest
import torch

from oracle import diff_oracle as D
from paper_0811_2055_gb300 import synth

from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_0811_2055_gb300 import gblod
    torch.cuda.set_device(0)
    return gblod


def _problem(n=4096, W=64, H=64, seed=0, n_views=3):
    rng = np.random.default_rng(seed)
    p = synth.clustered(n, 8, 0.2, 0.0, seed=seed + 100)
    xyz = p.xyz.astype(np.float32)
    w = rng.uniform(0.5, 2.0, n).astype(np.float32)
    logh = np.log(rng.uniform(0.004, 0.03, n)).astype(np.float32)
    cams = [synth.look_at(e, (0.5, 0.5, 0.5), width=W, height=H)
            for e in [(0.5, 0.5, -0.6), (1.4, 0.8, 0.6), (0.2, -0.5, 0.3)][:n_views]]
    return xyz, w, logh, cams


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_forward_matches_fp64_oracle(G):
    xyz, w, logh, cams = _problem()
    r = G.Renderer()
    img = G.diff_render(r, *to_dev(xyz, w, logh), cams).cpu().numpy()
    for v, cam in enumerate(cams):
        want = D.forward(cam, xyz.astype(np.float64), w.astype(np.float64), logh.astype(np.float64))
        assert _rel(img[v], want) < 1e-4
        # and pixel by pixel (a local error, e.g. at a tile edge, cannot hide in the norm)
        assert float(np.abs(img[v] - want).max()) <= 1e-4 * float(np.abs(want).max())
    r.close()


def test_adjoint_matches_analytic_fp64_gradient(G):
    xyz, w, logh, cams = _problem(seed=1)
    rng = np.random.default_rng(5)
    g = rng.normal(size=(len(cams), 64, 64)).astype(np.float32)
    r = G.Renderer()
    gx, gw, gl = (t.cpu().numpy() for t in G.diff_backward(r, *to_dev(xyz, w, logh), cams, to_dev(g)[0]))
    wx, ww, wl = np.zeros((len(w), 3)), np.zeros(len(w)), np.zeros(len(w))
    for v, cam in enumerate(cams):
        a, b, c = D.backward(cam, xyz.astype(np.float64), w.astype(np.float64), logh.astype(np.float64),
                             g[v].astype(np.float64))
        wx, ww, wl = wx + a, ww + b, wl + c
    assert _rel(gx, wx) < 1e-3 and _rel(gw, ww) < 1e-3 and _rel(gl, wl) < 1e-3
    r.close()


def test_adjoint_matches_fp64_finite_differences(G):
    """4,096 points, 64x64: directional and per-coordinate central differences in FP64."""
    xyz, w, logh, cams = _problem(seed=2, n_views=1)
    cam = cams[0]
    rng = np.random.default_rng(7)
    g = rng.normal(size=(64, 64))
    r = G.Renderer()
    gx, gw, gl = (t.cpu().numpy().astype(np.float64)
                  for t in G.diff_backward(r, *to_dev(xyz, w, logh), [cam], to_dev(g.astype(np.float32)[None])[0]))
    P, Wt, Lh = xyz.astype(np.float64), w.astype(np.float64), logh.astype(np.float64)

    def L(p, ww, ll):
        return float(np.sum(g * D.forward(cam, p, ww, ll)))

    eps = 1e-7
    for k in range(6):  # random directions through all 5 x 4096 parameters
        dp, dw, dl = rng.normal(size=P.shape), rng.normal(size=Wt.shape), rng.normal(size=Lh.shape)
        dp *= 0.1
        fd = (L(P + eps * dp, Wt + eps * dw, Lh + eps * dl) - L(P - eps * dp, Wt - eps * dw, Lh - eps * dl)) / (2 * eps)
        an = float(np.sum(gx * dp) + np.sum(gw * dw) + np.sum(gl * dl))
        assert abs(an - fd) <= 1e-3 * abs(fd), (k, an, fd)
    # per-coordinate on the points with the largest gradients
    top = np.argsort(-np.abs(gx).sum(1))[:8]
    an_s, fd_s = [], []
    for i in top:
        for a in range(3):
            q1, q2 = P.copy(), P.copy()
            q1[i, a] += 1e-6
            q2[i, a] -= 1e-6
            fd = (L(q1, Wt, Lh) - L(q2, Wt, Lh)) / 2e-6
            # per component: relative 1e-3, with a floor of 1e-6 of the largest component for the
            # components near zero (where a relative bound means nothing)
            assert abs(gx[i, a] - fd) <= 1e-3 * max(abs(fd), 1e-3 * np.abs(gx).max()), (i, a, gx[i, a], fd)
            an_s.append(gx[i, a])
            fd_s.append(fd)
    # and over the sampled components together, the plain relative error
    assert _rel(np.array(an_s), np.array(fd_s)) <= 1e-3
    r.close()


def test_autograd_function(G):
    xyz, w, logh, cams = _problem(n=2000, seed=3)
    r = G.Renderer()
    tx, tw, tl = (t.clone().requires_grad_(True) for t in to_dev(xyz, w, logh))
    target = torch.rand((len(cams), 64, 64), device=tx.device) * 1e-3
    img = G.SplatImages.apply(tx, tw, tl, cams, r, G.make_params())
    loss = ((img - target) ** 2).sum()
    loss.backward()
    gx, gw, gl = G.diff_backward(r, *to_dev(xyz, w, logh), cams, 2 * (img.detach() - target))
    # the adjoint sums with float atomics, so two calls agree to rounding, not bit for bit
    for a, b in ((tx.grad, gx), (tw.grad, gw), (tl.grad, gl)):
        assert float((a - b).norm() / b.norm()) <= 1e-5
    r.close()


def test_fitting_reduces_the_image_loss(G):
    """Fit 500 representatives to the images of 8,000 parent particles (the paper's visual
    equivalence goal at small scale): Adam on (xyz, w, log h) lowers the L2 image loss."""
    parent = synth.clustered(8000, 6, 0.1, 0.0, seed=9)
    cams = [synth.look_at(e, (0.5, 0.5, 0.5), width=64, height=64)
            for e in [(0.5, 0.5, -0.8), (1.6, 0.5, 0.5), (0.5, 1.7, 0.4), (-0.6, 0.3, 0.6)]]
    r = G.Renderer()
    pxyz, pw, pl = to_dev(parent.xyz, parent.mass, np.log(np.maximum(parent.h, 1e-4)).astype(np.float32))
    target = G.diff_render(r, pxyz, pw, pl, cams)
    rng = np.random.default_rng(0)
    pick = rng.choice(parent.n, 500, replace=False)
    x = torch.tensor(parent.xyz[pick], device=pxyz.device, requires_grad=True)
    wv = torch.full((500,), parent.n / 500.0, device=pxyz.device, requires_grad=True)
    lh = torch.tensor(np.log(np.maximum(parent.h[pick], 1e-4) * (parent.n / 500) ** (1 / 3)).astype(np.float32),
                      device=pxyz.device, requires_grad=True)
    opt = torch.optim.Adam([{"params": [x], "lr": 2e-3}, {"params": [wv], "lr": 0.5}, {"params": [lh], "lr": 1e-2}])
    losses = []
    for _ in range(40):
        opt.zero_grad()
        loss = ((G.SplatImages.apply(x, wv, lh, cams, r, G.make_params()) - target) ** 2).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.7 * losses[0], losses[::8]
    r.close()
