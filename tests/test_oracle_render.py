"""Pins of the oracle's per-frame path (CPU only).

The paper has the graphics card draw every point as a smeared blob whose radial kernel is
evaluated at every pixel it covers; the drawn set comes from a view-dependent cut of the
octree (near nodes deep, far nodes shallow), and the goal is an image the user cannot tell
from a full rendering.  Pins below: the kernel table against a 200-bit evaluation of its
formula, closed forms of a single splat (total intensity, second moment, centroid, mirror
symmetry, whole-pixel shift, the FP64 analytic Gaussian), full-depth LOD == brute force,
the limiting cases of the detail criterion, and the tone map's closed forms.
"""
import math

import mpmath as mp
import numpy as np
import pytest

from oracle import oracle as O
from paper_0811_2055_gb300 import synth


def _rne(x: mp.mpf) -> int:
    f = int(mp.floor(x))
    r = x - f
    if r > mp.mpf(0.5) or (r == mp.mpf(0.5) and f % 2 == 1):
        return f + 1
    return f


def test_gaussian_table_exact():
    mp.mp.prec = 200
    K = O.kernel_table(0)
    for i in range(1024):
        q = (mp.mpf(i) + mp.mpf(0.5)) * 9 / 1024
        assert K[i] == _rne(65536 * mp.exp(-q / 2)), i


def test_cubic_table_exact():
    mp.mp.prec = 200
    K = O.kernel_table(1)
    for i in range(1024):
        q = (mp.mpf(i) + mp.mpf(0.5)) * 4 / 1024
        xi = mp.sqrt(q)
        f = 1 - mp.mpf(1.5) * q + mp.mpf(0.75) * q * xi if xi < 1 else mp.mpf(0.25) * (2 - xi) ** 3
        want = _rne(65536 * f)
        # the oracle evaluates the polynomial in double; allow the exact value to sit on a
        # rounding boundary only within double precision
        assert abs(int(K[i]) - want) <= (1 if abs(65536 * f - mp.floor(65536 * f) - mp.mpf(0.5)) < 1e-9 else 0), i


def test_normalisation_constants():
    mp.mp.prec = 200
    c = O.constants()
    assert c["A_gauss"] == np.float32(float(mp.mpf(2) ** 32 / (2 * mp.pi * (1 - mp.exp(-4.5)))))
    assert c["A_cubic"] == np.float32(float(mp.mpf(2) ** 32 * 10 / (7 * mp.pi)))
    assert c["B_gauss"] == np.float32(float(mp.mpf(2) ** 31 / 9))
    assert c["B_cubic"] == np.float32(2.0 ** 29)


def _axis_camera(W=256, H=256, f=200.0, z_eye=-1.0):
    cam = synth.look_at((0.5, 0.5, z_eye), (0.5, 0.5, 0.5), width=W, height=H)
    cam["f_px"] = f
    return cam


def _single(cam, rp, x, y, z, w, h):
    return O.splat_points(np.array([[x, y, z, w]], np.float32), np.array([h], np.float32), cam, rp)[0]


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("sigma_px", [2.0, 4.0, 16.0])
def test_total_intensity_is_mass(kernel, sigma_px):
    cam = _axis_camera()
    rp = O.rparams(kernel=kernel)
    D = 1.5  # eye at z=-1, point at z=0.5
    h = sigma_px * D / cam["f_px"]
    w = 3.0
    acc = _single(cam, rp, 0.5, 0.5, 0.5, w, h)
    tot = acc.sum(dtype=np.float64) / 2**32
    assert abs(tot - w) <= 0.01 * w, tot


@pytest.mark.parametrize("sigma_px", [4.0, 8.0, 20.0])
def test_second_moment_and_centroid(sigma_px):
    cam = _axis_camera()
    rp = O.rparams(kernel=0)
    # off-axis point: 0.1 to the camera's right (right = -x for this view), 0.05 up
    x, y, z = 0.5 - 0.1, 0.5 + 0.05, 0.5
    D = 1.5
    h = sigma_px * D / cam["f_px"]
    acc = _single(cam, rp, x, y, z, 1.0, h).astype(np.float64)
    H, W = acc.shape
    py, px = np.mgrid[0:H, 0:W]
    cxp, cyp = px + 0.5, py + 0.5
    m = acc.sum()
    u = (acc * cxp).sum() / m
    v = (acc * cyp).sum() / m
    u_ref = cam["cx"] + cam["f_px"] * 0.1 / D     # FP64 pinhole projection
    v_ref = cam["cy"] - cam["f_px"] * 0.05 / D    # image y grows downwards
    assert abs(u - u_ref) < 0.02 and abs(v - v_ref) < 0.02
    r2 = ((cxp - u) ** 2 + (cyp - v) ** 2)
    m2 = (acc * r2).sum() / m
    trunc = 1.0 - 4.5 * math.exp(-4.5) / (1.0 - math.exp(-4.5))  # E[t | t < 4.5], t ~ Exp(1)
    assert abs(m2 / (2 * sigma_px**2 * trunc) - 1.0) < 0.01


def test_mirror_symmetry_on_axis():
    cam = _axis_camera(W=128, H=96)
    rp = O.rparams()
    acc = _single(cam, rp, 0.5, 0.5, 0.5, 1.0, 6.0 * 1.5 / cam["f_px"])
    assert acc.sum() > 0
    assert np.array_equal(acc, acc[:, ::-1]) and np.array_equal(acc, acc[::-1, :])


def test_whole_pixel_shift():
    cam = _axis_camera(W=128, H=96)
    rp = O.rparams()
    h = 5.0 * 1.5 / cam["f_px"]
    a = _single(cam, rp, 0.5, 0.5, 0.5, 1.0, h)
    cam2 = dict(cam, cx=cam["cx"] + 3.0, cy=cam["cy"] - 2.0)
    b = _single(cam2, rp, 0.5, 0.5, 0.5, 1.0, h)
    assert np.array_equal(b[:-2, 3:], a[2:, :-3])


def test_matches_fp64_analytic_gaussian():
    cam = _axis_camera()
    rp = O.rparams(kernel=0)
    x, y, z, w = 0.47, 0.52, 0.4, 2.0
    D = 0.4 - (-1.0)
    sigma = 3.3
    h = sigma * D / cam["f_px"]
    acc = _single(cam, rp, x, y, z, w, h).astype(np.float64) / 2**32
    u = cam["cx"] + cam["f_px"] * (0.5 - x) / D
    v = cam["cy"] - cam["f_px"] * (y - 0.5) / D
    H, W = acc.shape
    py, px = np.mgrid[0:H, 0:W]
    q = ((px + 0.5 - u) ** 2 + (py + 0.5 - v) ** 2) / sigma**2
    C = 1.0 - math.exp(-4.5)
    g = np.where(q < 9.0, w * np.exp(-q / 2) / (2 * math.pi * sigma**2 * C), 0.0)
    peak = w / (2 * math.pi * sigma**2 * C)
    err = np.abs(acc - g) / peak
    inner = q < 8.9
    assert err[inner].max() < 0.004
    assert err.max() < 0.0125  # a pixel right on the 3-sigma edge may fall either side


def test_culling_rules():
    cam = _axis_camera(W=64, H=64)
    rp = O.rparams()
    assert O.project(cam, rp, 0.5, 0.5, -2.0, 1.0, 0.01)[0] == 0        # behind the eye
    assert O.project(cam, rp, 0.5, 0.5, -1.0 + 1e-4, 1.0, 0.01)[0] == 0  # inside z_near
    assert O.project(cam, rp, 50.0, 0.5, 0.5, 1.0, 0.001)[0] == 0        # far off screen
    assert O.project(cam, rp, 0.5, 0.5, 0.5, 1.0, 0.01)[0] == 1
    assert O.project(cam, rp, 0.5, 0.5, 0.5, float("nan"), 0.01)[0] == -1  # amplitude out of range
    assert O.project(cam, rp, float("nan"), 0.5, 0.5, 1.0, 0.01)[0] == 0
    # sigma is clamped to [sigma_min, sigma_max]
    a = O.project(cam, rp, 0.5, 0.5, 0.5, 1.0, 0.0)
    b = O.project(cam, rp, 0.5, 0.5, 0.5, 1.0, 1e-9)
    assert a == b
    big = O.project(cam, rp, 0.5, 0.5, 0.5, 1.0, 100.0)
    huge = O.project(cam, rp, 0.5, 0.5, 0.5, 1.0, 1e6)
    assert big == huge


def _lod_inputs():
    p = synth.tiny(30000, seed=21)
    return p, 200


@pytest.mark.parametrize("view", ["outside", "inside", "grazing"])
def test_full_depth_lod_equals_brute_force(view):
    p, n_max = _lod_inputs()
    # a few particles outside the root cube and one clamped onto its boundary cell
    xyz = p.xyz.copy()
    xyz[:5] = np.array([[1.2, 0.5, 0.5], [-0.3, 0.2, 0.1], [0.5, 1.5, 0.5], [0.4, 0.4, -0.2], [2.0, 2.0, 2.0]])
    T = O.build_tree(xyz, p.mass, p.h, seed=3, n_max=n_max)
    cams = {"outside": synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=160, height=120),
            "inside": synth.look_at((0.45, 0.55, 0.5), (0.9, 0.4, 0.6), width=160, height=120, z_near=1e-3),
            "grazing": synth.look_at((1.3, 0.5, 0.5), (0.5, 1.2, 0.4), width=160, height=120, vfov_deg=30.0)}
    cam = cams[view]
    for kernel in (0, 1):
        rp0 = O.rparams(lambda_px=0.0, kernel=kernel)
        lod, st, nd, npts = O.render_lod(T, cam, rp0)
        brute, st2, nd2 = O.splat_particles(xyz, p.mass, p.h, cam, rp0)
        assert st == 0 and st2 == 0
        assert np.array_equal(lod, brute)
        assert nd == nd2 and brute.sum() > 0


def test_selection_limits():
    p, n_max = _lod_inputs()
    T = O.build_tree(p.xyz, p.mass, p.h, seed=3, n_max=n_max)
    cam = synth.look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), width=160, height=120)
    leaves = {i for i, nd in enumerate(T.nodes) if not int(nd["flags"]) & O.INTERNAL}
    sel0 = set(O.select(T, cam, O.rparams(lambda_px=0.0)).tolist())
    assert sel0 <= leaves and len(sel0) > 0.5 * len(leaves)
    assert O.select(T, cam, O.rparams(lambda_px=float("inf"))).tolist() == [0]
    # camera inside the root box: its distance is 0, so the root is always refined
    cam_in = synth.look_at((0.5, 0.5, 0.5), (0.5, 0.5, 1.0), width=160, height=120)
    assert 0 not in set(O.select(T, cam_in, O.rparams(lambda_px=1e4)).tolist())
    # default lambda: every emitted internal node is far enough to be coarse
    sel = O.select(T, cam, O.rparams(n_max=n_max))
    assert len(sel) < len(sel0) + 50


def test_depth_never_increases_with_distance():
    p = synth.tiny(30000, seed=22)
    T = O.build_tree(p.xyz, p.mass, p.h, seed=3, n_max=100)
    # aim at a particle of the deepest node, so the chain of nodes above it is long
    deep = int(np.argmax(T.nodes["depth"]))
    target32 = p.xyz[T.sidx[int(T.nodes[deep]["seg_first"])]]
    target = target32.astype(np.float64)
    key = O.morton_key(*target32.tolist())
    codes = {int(nd["code"]): i for i, nd in enumerate(T.nodes)}
    chain = []
    for d in range(T.depth_max + 1):
        c = (1 << (3 * d)) | (key >> (63 - 3 * d)) if d else 1
        if c in codes:
            chain.append(codes[c])
    assert len(chain) == T.depth_max + 1
    seen = []
    for dist in [0.002, 0.005, 0.01, 0.02, 0.05, 0.1, 0.2, 0.4, 0.8, 1.6, 3.2, 6.4, 12.8]:
        eye = target - np.array([0.0, 0.0, dist])
        cam = synth.look_at(eye, target, width=320, height=240, z_near=1e-4)
        sel = set(O.select(T, cam, O.rparams(lambda_px=20.0)).tolist())
        hit = [int(T.nodes[i]["depth"]) for i in chain if i in sel]
        assert len(hit) == 1
        if seen:
            assert hit[0] <= seen[-1]
        seen.append(hit[0])
    assert len(set(seen)) >= 4, seen


def test_tonemap_closed_forms():
    hi = 3 << 40
    lo = int(hi * 1e-4)
    acc = np.array([0, lo, lo - 1, hi, int(math.sqrt(hi * (hi * 1e-4))), hi // 10], np.uint64)
    out = O.tonemap(acc, O.rparams(tone_auto=1))
    assert out[0] == 0 and out[1] == 0 and out[2] == 0 and out[3] == 255
    assert abs(int(out[4]) - 128) <= 1                       # geometric mean maps to the middle
    assert abs(int(out[5]) - round(255 * 0.75)) <= 1          # one decade below the top of four
    out2 = O.tonemap(acc, O.rparams(tone_auto=0, tone_lo=hi * 1e-4 / 2**32, tone_hi=hi / 2**32))
    assert np.array_equal(out, out2)
    z = O.tonemap(np.zeros(10, np.uint64), O.rparams(tone_auto=1))
    assert not z.any()
    # monotone
    ramp = np.sort(np.random.default_rng(0).integers(0, 2**50, 1000).astype(np.uint64))
    r = O.tonemap(ramp, O.rparams(tone_auto=1)).astype(int)
    assert np.all(np.diff(r) >= 0)


def test_pixel_update_count():
    """The counter of (splat, pixel) pairs inside the support, pinned by exact integer enumeration of
    q S < 2^47 over a window around one splat (independent of the oracle's box logic), additivity
    and the area of the 3-sigma disc."""
    cam = _axis_camera(W=256, H=256, f=200.0)
    rp = O.rparams()
    pts = np.array([[0.5, 0.5, 0.5, 1.0]], np.float32)
    for h in (0.002, 0.01, 0.03):
        hs = np.array([h], np.float32)
        n = O.count_updates(pts, hs, cam, rp)
        ok, U, V, S, Wq = (int(v) for v in O.project(cam, rp, 0.5, 0.5, 0.5, 1.0, h))
        assert ok == 1
        brute = 0
        for py in range(256):
            dy = py * 256 + 128 - V
            for px in range(256):
                dx = px * 256 + 128 - U
                if (dx * dx + dy * dy) * S < (1 << 47):
                    brute += 1
        assert n == brute
        sigma = 200.0 * h / 1.5
        if 3 * sigma < 100:
            assert abs(n - math.pi * (3 * sigma) ** 2) < 0.1 * math.pi * (3 * sigma) ** 2 + 20
    a = np.array([[0.5, 0.5, 0.5, 1.0], [0.45, 0.52, 0.5, 2.0], [0.6, 0.4, 0.55, 0.5]], np.float32)
    ha = np.array([0.01, 0.004, 0.02], np.float32)
    assert O.count_updates(a, ha, cam, rp) == sum(O.count_updates(a[i:i + 1], ha[i:i + 1], cam, rp) for i in range(3))


def test_frame_independent_of_thread_count():
    # the frame loops share points out between threads with images of their own, summed as
    # integers at the end: one thread and all threads give the same image bit for bit
    p = synth.tiny(60000, seed=23)
    T = O.build_tree(p.xyz, p.mass, p.h, seed=3, n_max=300)
    cam = synth.look_at((0.45, 0.55, -0.4), (0.5, 0.5, 0.5), width=200, height=150)
    rp = O.rparams(lambda_px=8.0)
    try:
        O.set_threads(1)
        a, st_a, nd_a, _ = O.render_lod(T, cam, rp)
        ba, _, _ = O.splat_particles(p.xyz, p.mass, p.h, cam, rp)
        O.set_threads(0)
        b, st_b, nd_b, _ = O.render_lod(T, cam, rp)
        bb, _, _ = O.splat_particles(p.xyz, p.mass, p.h, cam, rp)
    finally:
        O.set_threads(0)
    assert st_a == st_b == 0 and nd_a == nd_b and a.sum() > 0
    assert np.array_equal(a, b) and np.array_equal(ba, bb)


def test_lod_update_count_equals_the_point_list_count():
    p = synth.tiny(30000, seed=24)
    T = O.build_tree(p.xyz, p.mass, p.h, seed=3, n_max=300)
    cam = synth.look_at((0.5, 0.45, -0.6), (0.5, 0.5, 0.5), width=160, height=120)
    rp = O.rparams(lambda_px=6.0)
    acc, st, nd, npts, nu = O.render_lod_counted(T, cam, rp)
    sel = O.select(T, cam, rp)
    rows = np.concatenate([np.arange(int(T.nodes[i]["point_first"]), int(T.nodes[i]["point_first"]) +
                                     int(T.nodes[i]["point_count"])) for i in sel])
    assert st == 0 and npts == len(rows) and nu > 0
    assert nu == O.count_updates(T.pts4[rows], T.hs[rows], cam, rp)
    assert np.array_equal(acc, O.render_lod(T, cam, rp)[0])
