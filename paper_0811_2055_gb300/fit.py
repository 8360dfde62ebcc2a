"""Fitting a node's representatives to the image of its particles (abstract: an LOD image
"indistinguishable from a full rendering"; octree paragraph: a node's n points stand for all of its
particles).

The random density-weighted subselection keeps n of a node's particles and gives each the weight
M/n and a smoothing length grown as (count/n)^(1/3).  fit_node moves those n points -- positions,
weights and log smoothing lengths -- so that their float splat images match the float images of all
of the node's particles from a set of views at the distance where the node is drawn, by gradient
descent (Adam) on the L2 image difference, with gradients from the library's adjoint splat kernel
(gblod.SplatImages).  The fitted points are written back into the octree (gblod_octree_set_points),
where the exact integer renderer draws them like any stored points.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gblod, synth


def node_box(tree: gblod.Octree, node: int) -> tuple[np.ndarray, float]:
    """(cell centre, cell edge) of a node, from its locational code and the octree's root cube."""
    info = tree.export_nodes()
    nd = info[node]
    d = int(nd["depth"])
    pfx = int(nd["code"]) ^ (1 << (3 * d))
    q = [0, 0, 0]
    for lvl in range(d):
        o = (pfx >> (3 * (d - 1 - lvl))) & 7
        q[0] = (q[0] << 1) | ((o >> 2) & 1)
        q[1] = (q[1] << 1) | ((o >> 1) & 1)
        q[2] = (q[2] << 1) | (o & 1)
    lo, side = tree.root
    e = side / (1 << d)
    return np.array([lo[a] + e * (q[a] + 0.5) for a in range(3)]), e


def node_views(tree: gblod.Octree, node: int, lambda_px: float, n_views: int = 8, size: int = 128,
               margin: float = 1.25) -> list[dict]:
    """Cameras on a Fibonacci sphere around the node's cell, far enough that the node is drawn, not
    refined: its projected edge is lambda / margin pixels."""
    c, e = node_box(tree, node)
    F = (size / 2.0) / math.tan(math.radians(30.0))
    D = margin * F * e / lambda_px + e * math.sqrt(3.0) / 2.0
    g = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for k in range(n_views):
        y = 1.0 - 2.0 * (k + 0.5) / n_views
        rr = math.sqrt(max(0.0, 1.0 - y * y))
        eye = c + D * np.array([rr * math.cos(g * k), y, rr * math.sin(g * k)])
        cams.append(synth.look_at(eye.tolist(), c.tolist(), vfov_deg=60.0, width=size, height=size,
                                  z_near=1e-4))
    return cams


def fit_node(tree: gblod.Octree, node: int, xyz: torch.Tensor, mass: torch.Tensor, h: torch.Tensor,
             cams: list[dict], steps: int = 60, renderer: gblod.Renderer | None = None,
             lr_pos: float = 0.1, lr_w: float = 0.02, lr_logh: float = 0.02, write: bool = True,
             log_floor: float | None = 1e-3) -> dict:
    """Fits node `node`'s stored points to the images of its member particles (rows of xyz, mass,
    h: the arrays the octree was built from).  The loss is the L2 difference of log(1 + I / I0) with
    I0 = log_floor x the brightest target pixel (the display maps intensity logarithmically, so
    faint and bright regions count alike; log_floor=None: plain intensities).  Learning rates are
    relative: positions move in units of the points' mean spacing (cell edge / n^(1/3)), weights
    and smoothing lengths in log units.  The iterate with the lowest loss is kept (the starting
    points if no step lowered it).  Returns the loss before and after; with `write` the fitted points
    replace the node's points in the octree (only if they lowered the loss)."""
    r = renderer or gblod.Renderer()
    par = gblod.make_params()
    p4, hs = tree.node_points(node)
    ids = tree.node_members(node).long()
    mx, mm, mh = xyz[ids].contiguous(), mass[ids].contiguous(), h[ids].contiguous()
    target = gblod.diff_render(r, mx, mm, torch.log(mh), cams, par)
    i0 = float(target.max()) * log_floor if log_floor else 0.0
    tmap = (lambda im: torch.log1p(im / i0)) if i0 > 0.0 else (lambda im: im)
    target = tmap(target)
    _, edge = node_box(tree, node)
    e = edge / max(float(p4.shape[0]), 1.0) ** (1.0 / 3.0)  # mean spacing of the node's points
    x0 = p4[:, :3].contiguous()
    u = torch.zeros_like(x0, requires_grad=True)           # position offset in mean spacings
    a = torch.zeros_like(p4[:, 3], requires_grad=True)     # log weight change
    b = torch.zeros_like(hs, requires_grad=True)           # log smoothing-length change
    w0, lh0 = p4[:, 3].contiguous(), torch.log(hs)
    opt = torch.optim.Adam([{"params": [u], "lr": lr_pos}, {"params": [a], "lr": lr_w},
                            {"params": [b], "lr": lr_logh}])
    losses = []
    best = (float("inf"), None)
    for _ in range(steps + 1):
        opt.zero_grad()
        img = gblod.SplatImages.apply(x0 + e * u, w0 * torch.exp(a), lh0 + b, cams, r, par)
        loss = ((tmap(torch.clamp(img, min=0.0)) - target) ** 2).sum()
        lv = float(loss.detach())
        losses.append(lv)
        if lv < best[0]:  # the loss of the current iterate, before this step moves it
            best = (lv, (u.detach().clone(), a.detach().clone(), b.detach().clone()))
        if len(losses) == steps + 1:
            break
        loss.backward()
        opt.step()
    bu, ba, bb = best[1]
    with torch.no_grad():
        fitted = torch.cat([(x0 + e * bu), (w0 * torch.exp(ba))[:, None]], 1).contiguous()
        fh = torch.exp(lh0 + bb).contiguous()
    improved = best[0] < losses[0]
    if write and improved:
        tree.set_points(node, fitted, fh)
    if renderer is None:
        r.close()
    return {"loss_first": losses[0], "loss_last": best[0], "steps": steps, "improved": improved,
            "points": int(p4.shape[0]), "members": int(ids.numel()), "pts4": fitted, "hs": fh}
