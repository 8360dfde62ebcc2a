"""Seeded synthetic particle sets and camera paths.

This module produces *inputs* only: particle positions, masses and smoothing lengths
shaped like the paper's data (an N-body snapshot dominated by dark-matter halos, 150M
particles per timestep; Szalay, Springel & Lemson, data paragraph), plus the camera
paths the renderer is driven with.  It holds none of the renderer's arithmetic, so
both the CUDA path and the CPU oracle may consume what it returns.

Every array is a pure function of (recipe, size, seed): numpy's counter-based
``Philox`` bit generator is keyed with the seed and nothing else.

Recipes
-------
``tiny``      262,144 particles: 80% in 64 Plummer spheres (scale radius log-uniform in
              [0.005, 0.05]), 20% uniform background, h = 0.002*exp(0.5*Z), unit mass.
``clustered`` the NFW-halo recipe: a uniform background fraction plus halos whose masses
              follow dN/dM ~ M^-1.9 over [1, 1000], concentrations uniform in [5, 15],
              virial radius 0.05*(M/1000)^(1/3), centres uniform in the unit cube, and
              optionally one dominant central halo.  h is 1.2 times the local mean
              inter-particle spacing of the host halo's analytic NFW profile.

All positions are wrapped periodically into [0, 1)^3 (the simulation box is periodic)
and stored as float32; the particle order is a seeded random permutation, so no
spatial order is handed to the renderer for free.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 0x081120550000
ONE_MINUS = np.float32(np.nextafter(np.float32(1.0), np.float32(0.0)))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def _wrap_f32(p: np.ndarray) -> np.ndarray:
    p = p - np.floor(p)
    out = p.astype(np.float32)
    np.minimum(out, ONE_MINUS, out=out)
    np.maximum(out, np.float32(0.0), out=out)
    return out


@dataclass
class Particles:
    xyz: np.ndarray   # (N, 3) float32
    mass: np.ndarray  # (N,) float32
    h: np.ndarray     # (N,) float32
    name: str = ""
    vel: np.ndarray | None = None  # (N, 3) float32 drift per timestep (halo bulk motion), optional

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    def subset(self, idx) -> "Particles":
        return Particles(np.ascontiguousarray(self.xyz[idx]), np.ascontiguousarray(self.mass[idx]),
                         np.ascontiguousarray(self.h[idx]), self.name + "[sub]")


def tiny(n: int = 262_144, seed: int = SEED_BASE + 0) -> Particles:
    """Plummer-sphere recipe (64 spheres + 20% background)."""
    rng = _rng(seed)
    n_cl = (4 * n) // 5
    n_sph = 64
    counts = np.full(n_sph, n_cl // n_sph, dtype=np.int64)
    counts[: n_cl - counts.sum()] += 1
    a = np.exp(rng.uniform(math.log(0.005), math.log(0.05), n_sph))
    centres = rng.uniform(0.0, 1.0, (n_sph, 3))
    sph = np.repeat(np.arange(n_sph), counts)
    u = rng.uniform(1e-12, 1.0, n_cl)
    r = a[sph] / np.sqrt(np.maximum(u ** (-2.0 / 3.0) - 1.0, 1e-300))
    r = np.minimum(r, 0.5)
    pos_cl = centres[sph] + r[:, None] * _isotropic(rng, n_cl)
    pos_bg = rng.uniform(0.0, 1.0, (n - n_cl, 3))
    pos = np.concatenate([pos_cl, pos_bg], axis=0)
    h = (0.002 * np.exp(0.5 * rng.standard_normal(n))).astype(np.float32)
    perm = rng.permutation(n)
    return Particles(_wrap_f32(pos[perm]), np.ones(n, np.float32), h[perm], f"tiny{n}")


def _nfw_mu(x):
    return np.log1p(x) - x / (1.0 + x)


def _nfw_radii(rng, n_per_halo, conc, r_vir, n_buckets=64):
    """Radii drawn from the NFW enclosed-mass profile truncated at r_vir (tabulated inverse)."""
    halo = np.repeat(np.arange(len(n_per_halo)), n_per_halo)
    u = rng.uniform(0.0, 1.0, halo.size)
    # concentrations are snapped to bucket centres so one inverse table serves each bucket
    lo, hi = 5.0, 15.0
    if np.all(conc == conc[0]):
        bucket_c = np.array([conc[0]])
        bidx = np.zeros(len(conc), np.int64)
    else:
        bucket_c = lo + (hi - lo) * (np.arange(n_buckets) + 0.5) / n_buckets
        bidx = np.clip(((conc - lo) / (hi - lo) * n_buckets).astype(np.int64), 0, n_buckets - 1)
    x_over_c = np.empty(halo.size)
    hb = bidx[halo]
    grid = np.linspace(0.0, 1.0, 8193)
    order = np.argsort(hb, kind="stable")
    bounds = np.searchsorted(hb[order], np.arange(len(bucket_c) + 1))
    for b, c in enumerate(bucket_c):
        sel = order[bounds[b]:bounds[b + 1]]
        if sel.size == 0:
            continue
        cdf = _nfw_mu(c * grid) / _nfw_mu(c)
        x_over_c[sel] = np.interp(u[sel], cdf, grid)
    c_used = bucket_c[hb]
    r = x_over_c * r_vir[halo]
    return halo, r, c_used


def clustered(n: int, n_halos: int, bg_frac: float = 0.10, central_frac: float = 0.0,
              central_c: float = 10.0, central_rvir: float = 0.25, seed: int = SEED_BASE + 1,
              name: str = "clustered", drift: float = 0.0) -> Particles:
    """NFW-halo recipe: background + power-law halo population (+ optional central halo)."""
    rng = _rng(seed)
    n_bg = int(round(bg_frac * n))
    n_central = int(round(central_frac * n))
    n_halo = n - n_bg - n_central
    # halo masses: dN/dM ~ M^-1.9 on [1, 1000] by inverse CDF
    uu = rng.uniform(0.0, 1.0, n_halos)
    g = 1.0 - 1.9
    m_h = (1.0 + uu * (1000.0 ** g - 1.0)) ** (1.0 / g)
    # particle counts proportional to mass, largest remainder
    share = m_h / m_h.sum() * n_halo
    cnt = np.floor(share).astype(np.int64)
    rem = n_halo - int(cnt.sum())
    if rem > 0:
        cnt[np.argsort(-(share - cnt), kind="stable")[:rem]] += 1
    conc = rng.uniform(5.0, 15.0, n_halos)
    r_vir = 0.05 * (m_h / 1000.0) ** (1.0 / 3.0)
    centres = rng.uniform(0.0, 1.0, (n_halos, 3))
    if n_central > 0:
        cnt = np.concatenate([cnt, [n_central]])
        conc = np.concatenate([conc, [central_c]])
        r_vir = np.concatenate([r_vir, [central_rvir]])
        centres = np.concatenate([centres, [[0.5, 0.5, 0.5]]], axis=0)
    halo, r, c_used = _nfw_radii(rng, cnt, conc, r_vir)
    dirs = _isotropic(rng, halo.size)
    pos_h = centres[halo] + r[:, None] * dirs
    # analytic local number density of the host halo at radius r
    r_s = r_vir[halo] / c_used
    rho_s = cnt[halo] / (4.0 * np.pi * r_s ** 3 * _nfw_mu(c_used))
    xr = np.maximum(r / r_s, 1e-12)
    n_loc = rho_s / (xr * (1.0 + xr) ** 2)
    h_h = np.clip(1.2 * n_loc ** (-1.0 / 3.0), 1e-5, 0.02)
    pos_bg = rng.uniform(0.0, 1.0, (n_bg, 3))
    h_bg = np.full(n_bg, 1.2 * max(n_bg, 1) ** (-1.0 / 3.0))
    pos = np.concatenate([pos_h, pos_bg], axis=0)
    h = np.concatenate([h_h, h_bg]).astype(np.float32)
    perm = rng.permutation(n)
    vel = None
    if drift > 0.0:
        # halo bulk velocities ~ N(0, drift) per timestep, drawn last so the positions above do not
        # depend on it; every particle of a halo moves with it, the background stays
        v_h = rng.normal(0.0, drift, (len(cnt), 3))
        vel = np.concatenate([v_h[halo], np.zeros((n_bg, 3))], axis=0)[perm].astype(np.float32)
    return Particles(_wrap_f32(pos[perm]), np.ones(n, np.float32), h[perm], name, vel)


def mid(n: int = 1 << 24, seed: int = SEED_BASE + 1) -> Particles:
    """4096 NFW halos + 10% background (16.8M particles at full size)."""
    n_halos = max(1, int(round(4096 * n / (1 << 24))))
    return clustered(n, n_halos, 0.10, 0.0, seed=seed, name=f"mid{n}")


def timesteps_recipe(n: int = 75_000_000, seed: int = SEED_BASE + 4) -> Particles:
    """The serving workload's base snapshot: mid recipe with 32,768 halos at 75M particles, plus
    halo drift velocities N(0, 0.002) per timestep (timestep t = wrap(xyz + t vel))."""
    n_halos = max(1, int(round(32768 * n / 75_000_000)))
    return clustered(n, n_halos, 0.10, 0.0, seed=seed, name=f"timesteps{n}", drift=0.002)


def paper_scale(n: int = 150_000_000, seed: int = SEED_BASE + 2) -> Particles:
    """65,536 NFW halos + one central halo holding 30% + 10% background (150M at full size)."""
    n_halos = max(1, int(round(65536 * n / 150_000_000)))
    return clustered(n, n_halos, 0.10, 0.30, seed=seed, name=f"paper{n}")


def uniform(n: int, seed: int = 7, h: float = 0.01) -> Particles:
    rng = _rng(seed)
    pos = rng.uniform(0.0, 1.0, (n, 3))
    return Particles(_wrap_f32(pos), np.ones(n, np.float32), np.full(n, h, np.float32), f"uniform{n}")


# ----------------------------------------------------------------------------- cameras

def look_at(eye, target, up=(0.0, 1.0, 0.0), vfov_deg: float = 60.0, width: int = 512,
            height: int = 512, z_near: float = 1e-3) -> dict:
    """Pinhole camera with orthonormal right/up/forward rows; image y grows downwards."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    nr = np.linalg.norm(right)
    if nr < 1e-12:
        right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
        nr = np.linalg.norm(right)
    right /= nr
    upv = np.cross(right, fwd)
    f_px = (height / 2.0) / math.tan(math.radians(vfov_deg) / 2.0)
    return dict(eye=eye.tolist(), right=right.tolist(), up=upv.tolist(), fwd=fwd.tolist(),
                f_px=float(f_px), cx=width / 2.0, cy=height / 2.0, z_near=float(z_near),
                width=int(width), height=int(height))


def tiny_view() -> dict:
    return look_at((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), vfov_deg=60.0, width=512, height=512, z_near=1e-3)


def helix_view(k: int, n_frames: int = 240, width: int = 1920, height: int = 1080) -> dict:
    """Frame k of the fly-through: a helix that closes in on the box centre."""
    th = 3.0 * math.pi * k / n_frames
    rad = 1.2 - 0.9 * k / (n_frames - 1)
    eye = (0.5 + rad * math.cos(th), 0.5 + 0.25 * math.sin(2.0 * math.pi * k / n_frames),
           0.5 + rad * math.sin(th))
    return look_at(eye, (0.5, 0.5, 0.5), vfov_deg=60.0, width=width, height=height, z_near=1e-3)


def paper_view(j: int, width: int = 1920, height: int = 1080) -> dict:
    """View j of 8 at distance 0.01*150^(j/7) along -z from the central halo, looking at it."""
    d = 0.01 * 150.0 ** (j / 7.0)
    return look_at((0.5, 0.5, 0.5 - d), (0.5, 0.5, 0.5), vfov_deg=60.0, width=width,
                   height=height, z_near=1e-4)
