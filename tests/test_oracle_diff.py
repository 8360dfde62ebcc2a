"""Pins of the FP64 oracle of the differentiable float splat (CPU only): the kernel integrates to
one and vanishes continuously at its support edge, the image is linear in the weights, and the
analytic gradient equals FP64 central finite differences."""
import math

import numpy as np
import pytest

from oracle import diff_oracle as D
from paper_0811_2055_gb300 import synth


def _cam(W=64, H=64, f=60.0):
    cam = synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=W, height=H)
    cam["f_px"] = f
    return cam


def test_kernel_integrates_to_one_and_is_continuous():
    cam = _cam(W=200, H=200, f=200.0)
    for sigma in (3.0, 7.5, 20.0):
        h = sigma * 1.5 / cam["f_px"]
        img = D.forward(cam, np.array([[0.5, 0.5, 0.5]]), np.array([2.0]), np.log([h]))
        assert abs(img.sum() - 2.0) < 2e-3 * 2.0, (sigma, img.sum())
    s2 = 4.0
    k_edge = (math.exp(-9 * s2 / (2 * s2)) - D.E45) / (2 * math.pi * s2 * D.CPRIME)
    assert abs(k_edge) < 1e-15


def test_image_is_linear_in_weights():
    cam = _cam()
    rng = np.random.default_rng(0)
    p = rng.uniform(0.3, 0.7, (30, 3))
    l = np.log(rng.uniform(0.01, 0.05, 30))
    w1, w2 = rng.uniform(0.5, 2, 30), rng.uniform(0.5, 2, 30)
    a = D.forward(cam, p, w1, l) + D.forward(cam, p, w2, l)
    assert np.allclose(a, D.forward(cam, p, w1 + w2, l), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("seed", [1, 2])
def test_analytic_gradient_equals_finite_differences(seed):
    cam = _cam()
    rng = np.random.default_rng(seed)
    n = 12
    p = rng.uniform(0.35, 0.65, (n, 3))
    w = rng.uniform(0.5, 2.0, n)
    l = np.log(rng.uniform(0.02, 0.08, n))  # sigma well inside (0.5, 128) px
    g = rng.normal(size=(cam["height"], cam["width"]))

    def L(p_, w_, l_):
        return float(np.sum(g * D.forward(cam, p_, w_, l_)))

    dp, dw, dl = D.backward(cam, p, w, l, g)
    eps = 1e-6
    for i in range(n):
        for a in range(3):
            q1, q2 = p.copy(), p.copy()
            q1[i, a] += eps
            q2[i, a] -= eps
            fd = (L(q1, w, l) - L(q2, w, l)) / (2 * eps)
            assert abs(fd - dp[i, a]) <= 1e-5 * max(1.0, abs(fd)), (i, a, fd, dp[i, a])
        w1, w2 = w.copy(), w.copy()
        w1[i] += eps
        w2[i] -= eps
        fd = (L(p, w1, l) - L(p, w2, l)) / (2 * eps)
        assert abs(fd - dw[i]) <= 1e-6 * max(1.0, abs(fd))
        l1, l2 = l.copy(), l.copy()
        l1[i] += eps
        l2[i] -= eps
        fd = (L(p, w, l1) - L(p, w, l2)) / (2 * eps)
        assert abs(fd - dl[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, dl[i])


def test_clamped_sigma_has_no_log_h_gradient():
    cam = _cam()
    p = np.array([[0.5, 0.5, 0.5]])
    g = np.ones((cam["height"], cam["width"]))
    _, _, dl = D.backward(cam, p, np.array([1.0]), np.log([1e-6]), g)
    assert dl[0] == 0.0


def _int_splat(cam, x, y, z, w, h):
    from oracle import oracle as O
    return O.splat_points(np.array([[x, y, z, w]], np.float32), np.array([h], np.float32), cam,
                          O.rparams())[0].astype(np.float64) / 2**32


@pytest.mark.parametrize("eye,target", [((0.5, 0.5, -1.0), (0.5, 0.5, 0.5)),
                                        ((1.4, 0.9, -0.6), (0.45, 0.55, 0.5))])
@pytest.mark.parametrize("off", [(0.08, 0.0, 0.0), (0.0, 0.06, 0.0), (0.07, 0.05, 0.0), (-0.05, -0.07, 0.04)])
def test_camera_convention_matches_integer_oracle(eye, target, off):
    # one splat: the float image's centroid must sit where the integer oracle projects the point
    # (U/256, V/256), for points displaced along +x and +y (both signs of both image axes), and
    # the two images must agree as truncated Gaussians of the same sigma
    from oracle import oracle as O
    cam = synth.look_at(eye, target, width=128, height=96)
    cam["f_px"] = 120.0
    p = np.array([target[0] + off[0], target[1] + off[1], target[2] + off[2]], np.float32)
    h = np.float32(0.006)
    drawn, U, V, _, _ = O.project(cam, O.rparams(), float(p[0]), float(p[1]), float(p[2]), 1.0, float(h))
    assert drawn == 1
    img = D.forward(cam, p[None].astype(np.float64), np.array([1.0]), np.log([float(h)]))
    H, W = img.shape
    py, px = np.mgrid[0:H, 0:W]
    m = img.sum()
    u = float((img * (px + 0.5)).sum() / m)
    v = float((img * (py + 0.5)).sum() / m)
    assert abs(u - U / 256.0) < 0.02 and abs(v - V / 256.0) < 0.02, (u, v, U / 256.0, V / 256.0)
    # image orientation by definition: displaced along the camera's right vector -> right of
    # the image centre; along its up vector -> above it (image y grows downwards)
    d = p.astype(np.float64) - np.asarray(target, np.float64)
    along_r, along_u = float(d @ np.asarray(cam["right"])), float(d @ np.asarray(cam["up"]))
    if abs(along_r) > 1e-3:
        assert (u > cam["cx"]) == (along_r > 0)
    if abs(along_u) > 1e-3:
        assert (v < cam["cy"]) == (along_u > 0)
    ref = _int_splat(cam, float(p[0]), float(p[1]), float(p[2]), 1.0, float(h))
    assert np.abs(img - ref).sum() < 0.1 * ref.sum()


def test_float_splat_mirror_symmetric_on_axis():
    cam = _cam(W=96, H=64, f=150.0)
    img = D.forward(cam, np.array([[0.5, 0.5, 0.5]]), np.array([1.0]), np.log([0.05]))
    assert img.sum() > 0
    assert np.allclose(img, img[:, ::-1], rtol=0, atol=1e-15 * img.max())
    assert np.allclose(img, img[::-1, :], rtol=0, atol=1e-15 * img.max())
