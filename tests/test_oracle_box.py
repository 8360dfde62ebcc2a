"""Pins of the oracle's separable (box-truncated) Gaussian, kernel 2 (CPU only).

Reading: the Gaussian blob of smoothing length h (sigma = F h / z on screen) is the product of two
1D Gaussians, one per image axis; truncated at 3 sigma on each axis (a square support) and
renormalised to it.  Each axis reads the radial Gaussian's 1024-entry table at its own squared
offset, and a pixel gets floor(Wq K[j] K[i] / 2^32).  The pins: the normalisation constant
against a 200-bit evaluation; total intensity = mass; the image of one splat is an outer product
(rank one up to the floor), its support is a full square of half-width 3 sigma, its per-axis
second moment is that of a truncated normal, its centroid is the FP64 pinhole projection, and it
is mirror symmetric on axis; the FP64 analytic separable Gaussian within the table-bin bound;
pixel updates by exact enumeration; and full-depth LOD == brute force.
"""
import math

import mpmath as mp
import numpy as np
import pytest

from oracle import oracle as O
from paper_0811_2055_gb300 import synth

KBOX = 2


def _cam(W=256, H=256, f=200.0):
    cam = synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=W, height=H)
    cam["f_px"] = f
    return cam


def _single(cam, x, y, z, w, h, kernel=KBOX):
    return O.splat_points(np.array([[x, y, z, w]], np.float32), np.array([h], np.float32), cam,
                          O.rparams(kernel=kernel))[0]


def test_box_normalisation_constant():
    mp.mp.prec = 200
    A = mp.mpf(2) ** 32 / (2 * mp.pi * mp.erf(3 / mp.sqrt(2)) ** 2)
    # round to 24 significant bits, to nearest (A lies in [2^29, 2^30))
    q = A / mp.mpf(2) ** 29 * 2**23
    want = float(mp.nint(q)) * 2.0 ** (29 - 23)
    assert float(O.constants()["A_box"]) == want
    assert np.array_equal(O.kernel_table(KBOX), O.kernel_table(0))  # same 1D Gaussian table


@pytest.mark.parametrize("sigma_px", [1.0, 2.0, 4.0, 16.0])
def test_total_intensity_is_mass(sigma_px):
    cam = _cam()
    h = sigma_px * 1.5 / cam["f_px"]
    acc = _single(cam, 0.5, 0.5, 0.5, 3.0, h)
    assert abs(acc.sum(dtype=np.float64) / 2**32 - 3.0) <= 0.01 * 3.0


@pytest.mark.parametrize("sigma_px", [3.0, 8.0, 20.0])
def test_square_support_outer_product_moments_centroid(sigma_px):
    cam = _cam()
    x, y, z = 0.5 - 0.1, 0.5 + 0.05, 0.5  # right = -x for this view
    D = 1.5
    h = sigma_px * D / cam["f_px"]
    acc = _single(cam, x, y, z, 1.0, h)
    nz = np.argwhere(acc > 0)
    (y0, x0), (y1, x1) = nz.min(0), nz.max(0)
    # the support is a full square of half-width about 3 sigma (no corners cut)
    assert np.all(acc[y0:y1 + 1, x0:x1 + 1] > 0)
    assert abs((x1 - x0 + 1) - 6 * sigma_px) <= 2.0 and abs((y1 - y0 + 1) - 6 * sigma_px) <= 2.0
    # outer product: the image is rank one up to the per-pixel floor
    M = acc[y0:y1 + 1, x0:x1 + 1].astype(np.float64)
    col, row = M.sum(0), M.sum(1)
    R = np.outer(row, col) / M.sum()
    assert np.abs(M - R).max() <= 1e-3 * M.max() + 2.0
    # centroid = FP64 pinhole projection; per-axis second moment of a normal truncated at 3 sigma
    H, W = acc.shape
    py, px = np.mgrid[0:H, 0:W]
    a = acc.astype(np.float64)
    m = a.sum()
    u = (a * (px + 0.5)).sum() / m
    v = (a * (py + 0.5)).sum() / m
    assert abs(u - (cam["cx"] + cam["f_px"] * 0.1 / D)) < 0.02
    assert abs(v - (cam["cy"] - cam["f_px"] * 0.05 / D)) < 0.02
    phi3 = math.exp(-4.5) / math.sqrt(2 * math.pi)
    var1 = 1.0 - 2 * 3 * phi3 / math.erf(3 / math.sqrt(2))  # E[t^2 | |t| < 3]
    mx = (a * (px + 0.5 - u) ** 2).sum() / m
    my = (a * (py + 0.5 - v) ** 2).sum() / m
    for mom in (mx, my):
        assert abs(mom / (sigma_px**2 * var1) - 1.0) < 0.01, (mom, sigma_px)


def test_mirror_symmetry_on_axis():
    cam = _cam(W=128, H=96)
    acc = _single(cam, 0.5, 0.5, 0.5, 1.0, 6.0 * 1.5 / cam["f_px"])
    assert acc.sum() > 0
    assert np.array_equal(acc, acc[:, ::-1]) and np.array_equal(acc, acc[::-1, :])


def test_transpose_symmetry():
    # on a square image a splat on the axis is symmetric under swapping x and y (kernel 2 only
    # treats the axes alike if both axes read the table the same way)
    cam = _cam(W=96, H=96)
    acc = _single(cam, 0.5, 0.5, 0.5, 1.0, 5.0 * 1.5 / cam["f_px"])
    assert np.array_equal(acc, acc.T)


def test_matches_fp64_analytic_separable_gaussian():
    cam = _cam()
    x, y, z, w = 0.47, 0.52, 0.4, 2.0
    D = 0.4 - (-1.0)
    sigma = 3.3
    h = sigma * D / cam["f_px"]
    acc = _single(cam, x, y, z, w, h).astype(np.float64) / 2**32
    u = cam["cx"] + cam["f_px"] * (0.5 - x) / D
    v = cam["cy"] - cam["f_px"] * (y - 0.5) / D
    H, W = acc.shape
    py, px = np.mgrid[0:H, 0:W]
    tx = ((px + 0.5 - u) / sigma) ** 2
    ty = ((py + 0.5 - v) / sigma) ** 2
    C2 = math.erf(3 / math.sqrt(2)) ** 2
    inside = (tx < 9.0) & (ty < 9.0)
    g = np.where(inside, w * np.exp(-(tx + ty) / 2) / (2 * math.pi * sigma**2 * C2), 0.0)
    peak = w / (2 * math.pi * sigma**2 * C2)
    err = np.abs(acc - g) / peak
    inner = (tx < 8.9) & (ty < 8.9)
    # two table bins of half-width 9/2048 in t: exp(t/2) error <= 0.22% each
    assert err[inner].max() < 0.005
    assert err.max() < 0.0125  # a pixel right on the 3-sigma edge may fall either side


def test_pixel_update_count_and_pixel_value():
    cam = _cam(W=160, H=160, f=200.0)
    rp = O.rparams(kernel=KBOX)
    for h in (0.002, 0.01, 0.03):
        pts = np.array([[0.5, 0.5, 0.5, 1.0]], np.float32)
        hs = np.array([h], np.float32)
        n = O.count_updates(pts, hs, cam, rp)
        ok, U, V, S, Wq = (int(v) for v in O.project(cam, rp, 0.5, 0.5, 0.5, 1.0, h))
        assert ok == 1
        nx = sum(1 for px in range(160) if ((px * 256 + 128 - U) ** 2) * S < (1 << 47))
        ny = sum(1 for py in range(160) if ((py * 256 + 128 - V) ** 2) * S < (1 << 47))
        assert n == nx * ny
        acc = O.splat_points(pts, hs, cam, rp)[0]
        for (px, py) in ((80, 80), (81, 77), (70, 90), (0, 0)):
            assert O.pixel_value(pts, hs, cam, rp, px, py) == int(acc[py, px])


@pytest.mark.parametrize("view", ["outside", "inside"])
def test_full_depth_lod_equals_brute_force(view):
    p = synth.tiny(30000, seed=21)
    T = O.build_tree(p.xyz, p.mass, p.h, seed=3, n_max=200)
    cams = {"outside": synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=160, height=120),
            "inside": synth.look_at((0.45, 0.55, 0.5), (0.9, 0.4, 0.6), width=160, height=120, z_near=1e-3)}
    rp0 = O.rparams(lambda_px=0.0, kernel=KBOX)
    lod, st, nd, _ = O.render_lod(T, cams[view], rp0)
    brute, st2, nd2 = O.splat_particles(p.xyz, p.mass, p.h, cams[view], rp0)
    assert st == 0 and st2 == 0
    assert np.array_equal(lod, brute) and nd == nd2 and brute.sum() > 0
