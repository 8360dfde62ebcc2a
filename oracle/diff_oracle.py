"""FP64 oracle of the differentiable float splat (test infrastructure only).

The paper's goal is an LOD image "indistinguishable from a full rendering" (abstract); fitting a
node's representatives to the full-data image needs the derivative of the rendered image with
respect to the representatives' positions, weights and (log) smoothing lengths.  Reading used by
the float path (not the exact integer path):

  projection   d = p - E; xc = right.d, yc = up.d, zc = fwd.d (drawn iff zc > z_near);
               u = cx + F xc / zc, v = cy - F yc / zc, s = F exp(l) / zc,
               sigma = clamp(s, sigma_min, sigma_max)  (zero derivative through a clamp)
  kernel       K(r) = (exp(-r^2 / (2 sigma^2)) - exp(-4.5)) / (2 pi sigma^2 C'),  r < 3 sigma,
               C' = 1 - 5.5 exp(-4.5) (so K integrates to 1 and is continuous at r = 3 sigma)
  image        I(x, y) = sum_i w_i K_i(r),  r^2 = (x + 1/2 - u)^2 + (y + 1/2 - v)^2
  adjoint      with g = dL/dI:  dL/dw = sum g K;  with E = exp(-r^2/2s^2) / (2 pi s^2 C'),
               dL/du = sum g w E (x+1/2-u)/s^2,  dL/dv = sum g w E (y+1/2-v)/s^2,
               dL/ds = sum g w (E r^2/s^3 - 2 K/s);  then u, v, s -> p, l by the chain rule.

Pinned by central finite differences of `forward` in FP64 (tests/test_oracle_diff.py), by the
kernel's closed forms (unit integral, continuity at the support edge, mirror symmetry on axis),
and, for the camera convention, by the integer oracle: one splat's centroid lies at the integer
oracle's projected position (U/256, V/256) within 0.02 px for points off axis in +x, +y and both
together, seen from an axis-aligned and an oblique camera, and both images agree as truncated
Gaussians of the same sigma.
"""
from __future__ import annotations

import math

import numpy as np

E45 = math.exp(-4.5)
CPRIME = 1.0 - 5.5 * E45


def _cam(cam):
    E = np.asarray(cam["eye"], np.float64)
    R = np.stack([np.asarray(cam["right"], np.float64), np.asarray(cam["up"], np.float64),
                  np.asarray(cam["fwd"], np.float64)])
    return E, R


def project(cam, p, logh, sigma_min=0.5, sigma_max=128.0):
    """Returns u, v, sigma, zc, xc, yc, visible, clamped for points p (n, 3)."""
    E, R = _cam(cam)
    d = np.asarray(p, np.float64) - E
    xc, yc, zc = d @ R[0], d @ R[1], d @ R[2]
    vis = zc > cam["z_near"]
    zs = np.where(vis, zc, 1.0)
    F = cam["f_px"]
    u = cam["cx"] + F * xc / zs
    v = cam["cy"] - F * yc / zs
    s = F * np.exp(np.asarray(logh, np.float64)) / zs
    sig = np.clip(s, sigma_min, sigma_max)
    clamped = (s < sigma_min) | (s > sigma_max)
    return u, v, sig, zs, xc, yc, vis, clamped


def forward(cam, p, w, logh, sigma_min=0.5, sigma_max=128.0):
    W, H = cam["width"], cam["height"]
    u, v, sig, _, _, _, vis, _ = project(cam, p, logh, sigma_min, sigma_max)
    img = np.zeros((H, W))
    w = np.asarray(w, np.float64)
    for i in np.nonzero(vis)[0]:
        R = 3.0 * sig[i]
        x0, x1 = max(0, int(math.floor(u[i] - R - 1))), min(W - 1, int(math.ceil(u[i] + R + 1)))
        y0, y1 = max(0, int(math.floor(v[i] - R - 1))), min(H - 1, int(math.ceil(v[i] + R + 1)))
        if x0 > x1 or y0 > y1:
            continue
        xs = np.arange(x0, x1 + 1) + 0.5 - u[i]
        ys = np.arange(y0, y1 + 1) + 0.5 - v[i]
        r2 = ys[:, None] ** 2 + xs[None, :] ** 2
        s2 = sig[i] ** 2
        k = (np.exp(-r2 / (2 * s2)) - E45) / (2 * math.pi * s2 * CPRIME)
        img[y0:y1 + 1, x0:x1 + 1] += w[i] * np.where(r2 < 9 * s2, k, 0.0)
    return img


def backward(cam, p, w, logh, g, sigma_min=0.5, sigma_max=128.0):
    """Analytic gradient of sum(g * forward) with respect to p (n, 3), w (n,), logh (n,)."""
    W, H = cam["width"], cam["height"]
    E_, R_ = _cam(cam)
    u, v, sig, zc, xc, yc, vis, clamped = project(cam, p, logh, sigma_min, sigma_max)
    n = len(w)
    dp = np.zeros((n, 3))
    dw = np.zeros(n)
    dl = np.zeros(n)
    F = cam["f_px"]
    w = np.asarray(w, np.float64)
    for i in np.nonzero(vis)[0]:
        R = 3.0 * sig[i]
        x0, x1 = max(0, int(math.floor(u[i] - R - 1))), min(W - 1, int(math.ceil(u[i] + R + 1)))
        y0, y1 = max(0, int(math.floor(v[i] - R - 1))), min(H - 1, int(math.ceil(v[i] + R + 1)))
        if x0 > x1 or y0 > y1:
            continue
        dx = np.arange(x0, x1 + 1) + 0.5 - u[i]
        dy = np.arange(y0, y1 + 1) + 0.5 - v[i]
        r2 = dy[:, None] ** 2 + dx[None, :] ** 2
        s = sig[i]
        s2 = s * s
        inside = r2 < 9 * s2
        e = np.where(inside, np.exp(-r2 / (2 * s2)) / (2 * math.pi * s2 * CPRIME), 0.0)
        k = np.where(inside, e - E45 / (2 * math.pi * s2 * CPRIME), 0.0)
        gg = g[y0:y1 + 1, x0:x1 + 1]
        dw[i] = np.sum(gg * k)
        du = w[i] * np.sum(gg * e * dx[None, :]) / s2
        dv = w[i] * np.sum(gg * e * dy[:, None]) / s2
        ds = w[i] * np.sum(gg * (e * r2 / (s2 * s) - 2.0 * k / s))
        if clamped[i]:
            ds_dz, dl_i = 0.0, 0.0
        else:
            ds_dz, dl_i = -s / zc[i], ds * s
        dxc = du * F / zc[i]
        dyc = -dv * F / zc[i]
        dzc = du * (-F * xc[i] / zc[i] ** 2) + dv * (F * yc[i] / zc[i] ** 2) + ds * ds_dz
        dp[i] = R_[0] * dxc + R_[1] * dyc + R_[2] * dzc
        dl[i] = dl_i
    return dp, dw, dl
