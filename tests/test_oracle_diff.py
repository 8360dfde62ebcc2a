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
