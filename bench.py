#!/usr/bin/env python
"""Benchmark of the GB300 level-of-detail renderer (one JSON line on stdout, rank 0).

Workload (default `paper`): one paper-scale timestep of 150M synthetic particles (65,536 NFW
halos, a central halo holding 30% of them, 10% uniform background), octree with n_max = 16000,
and the eight 1920x1080 views from inside the central halo out to the whole box.  One step = one
pass of the whole hot path: build the octree on the device (A1-A5), then render the eight views
`--view-repeats` times at level of detail (R1-R4).  `value` is LOD frames/s over the timed steps
(build included); per view: p50/p99, splats/s and both rooflines (pixel updates against the
measured per-pixel ceiling, bytes against HBM).  The same views rendered from every particle
(brute force) are timed under "all_points".  `--workload mid` runs the 2^24-particle 240-frame
fly-through instead.

--impl reference times the CPU oracle (test infrastructure, plain C) on the host cores instead.
Multi-GPU (torchrun): every rank runs the full step on its own replica (weak scaling, no
collective on the data path); value = frames of all ranks / slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "splats/s & 1080p frames/s (LOD vs all points); p50/p99 frame latency"
# integer operations of one (splat, pixel) contribution by the rule's definition: two subtractions, two
# squares and an add (squared distance), a multiply and a shift (table index), a compare, a table read, a
# multiply and a shift (amplitude times table value), an add (accumulation)
OPS_PER_PIXEL_UPDATE = 12


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-block16", action="store_true", help="skip the 16-bit block-code fly-through")
    ap.add_argument("--workload", choices=["paper", "mid", "tiny", "diff", "serve", "paper-views", "fit"], default="paper")
    ap.add_argument("--fit-steps", type=int, default=40, help="fit: Adam steps per node")
    ap.add_argument("--view-repeats", type=int, default=4, help="paper: passes over the eight views per step")
    ap.add_argument("--view-list", type=str, default="", help="paper: comma-separated views (default: all eight)")
    ap.add_argument("--repeats", type=int, default=20, help="paper-views: timed repeats per view")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of offered load")
    ap.add_argument("--sessions", type=int, default=64)
    ap.add_argument("--session-budget-gb", type=float, default=4.0)
    ap.add_argument("--frames", type=int, default=0, help="frames per step (0 = the workload's path)")
    ap.add_argument("--path-frames", type=str, default="", help="mid: comma-separated frames of the 240-frame path")
    ap.add_argument("--particles", type=int, default=0, help="particles (0 = the workload's size)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-brute", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-views", type=int, default=16, help="views per batch in the batched measurement")
    ap.add_argument("--batch-capacity-log2", type=int, default=0,
                    help="log2 of the batch record capacity (0: 31 for paper, 29 otherwise)")
    return ap.parse_args()


def workload(name: str, frames: int, particles: int = 0, path_frames: str = "", view_list: str = ""):
    from paper_0811_2055_gb300 import synth
    if name == "mid":
        p = synth.mid(particles) if particles else synth.mid()
        ks = [int(x) for x in path_frames.split(",") if x.strip()] if path_frames else \
            [k * 240 // (frames or 240) for k in range(frames or 240)]
        cams = [synth.helix_view(k) for k in ks]
        desc = (f"mid: {p.n} particles (NFW halos, dN/dM ~ M^-1.9, c in [5,15], + 10% uniform), n_max 16000, "
                + (f"frames {path_frames} of " if path_frames else f"{len(ks)} frames of ")
                + "the 240-frame 1920x1080 helical fly-through")
    elif name == "paper":
        p = synth.paper_scale(particles) if particles else synth.paper_scale()
        js = [int(x) for x in view_list.split(",") if x.strip()] if view_list else list(range(8))
        cams = [synth.paper_view(j) for j in js]
        desc = (f"paper: {p.n} particles (65,536 NFW halos + central halo with 30% + 10% uniform), n_max 16000, "
                + (f"views {view_list} of " if view_list else "") +
                "the 8 views at 1920x1080 at d_j = 0.01 * 150^(j/7) from inside the central halo out to the whole box")
    else:
        p = synth.tiny()
        nf = frames or 1
        cams = [synth.tiny_view()] * nf
        desc = "tiny: 262,144 particles (64 Plummer spheres + 20% uniform), n_max 16000, 512x512 view"
    return p, cams, 16000, desc


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        sel = str(gpu)
        try:
            import torch
            u = getattr(torch.cuda.get_device_properties(gpu), "uuid", None)
            if u is not None:
                sel = "GPU-" + str(u) if not str(u).startswith("GPU-") else str(u)
        except Exception:
            pass
        self.gpu = sel
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", sel, f"--query-gpu={self.Q}", "--format=csv,noheader",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        rows = []
        for ln in open(self.f.name):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1].split()[0]), float(parts[2].split()[0]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows), "reasons": seen,
                "samples": len(rows)}


def combine_ranks(ms: float, e2e_s: float, frames: int, world: int, device=None):
    """Weak scaling over replicas: every rank rendered `frames` frames; the job takes as long as
    the slowest rank.  Returns (max ms, max end-to-end seconds, frames of all ranks)."""
    if world <= 1:
        return ms, e2e_s, frames
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, e2e_s, float(frames)], dtype=torch.float64, device=device)
    m = t.clone()
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(m[0]), float(m[1]), int(round(float(t[2])))


def dist_info():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


# ------------------------------------------------------------------ our implementation

def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_0811_2055_gb300 import gblod

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    p, views, n_max, desc = workload(a.workload, a.frames, a.particles, a.path_frames, a.view_list)
    reps = max(1, a.view_repeats) if a.workload == "paper" else 1
    cams = [c for _ in range(reps) for c in views]  # the frames of one step
    nv, nf = len(views), len(cams)
    W, H = views[0]["width"], views[0]["height"]
    xyz, mass, h = (torch.from_numpy(x).to(dev) for x in (p.xyz, p.mass, p.h))
    r = gblod.Renderer()
    lam = math.sqrt(n_max)
    par = gblod.make_params(lambda_px=lam)
    # the untimed census frames also count their pixel updates (the same frames as the timed ones)
    par_count = gblod.make_params(lambda_px=lam, count_updates=True)
    img = torch.empty((H, W), dtype=torch.uint8, device=dev)
    acc = torch.empty((H, W), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    hbm = measured_peaks().get("hbm_gbs")

    def barrier():
        if world > 1:
            dist.barrier()

    def lod_step(ev=None):
        if ev is not None:
            ev[0].record()
        tree = gblod.build_lod(xyz, mass, h, n_max=n_max, seed=1)
        if ev is not None:
            ev[1].record()
        for k, cam in enumerate(cams):
            if ev is not None:
                ev[2 + 2 * k].record()
            r.render(tree, cam, par, image=img, accum=acc)
            if ev is not None:
                ev[3 + 2 * k].record()
        return tree

    def brute_step(ev=None):
        for k, cam in enumerate(cams):
            if ev is not None:
                ev[2 * k].record()
            r.render_bruteforce(xyz, mass, h, cam, par, image=img, accum=acc)
            if ev is not None:
                ev[2 * k + 1].record()

    def timed(fn, n_ev, steps, warm, probe=None):
        for _ in range(warm):
            out = fn()
            if out is not None:
                out.free()
        torch.cuda.synchronize()
        tot_ms, frame_ms, build_ms = 0.0, [], []
        l0 = gblod.launch_count()
        if probe is not None:
            gblod.probe_enable(probe)
        for _ in range(steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            barrier()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn(ev)
            e1.record()
            torch.cuda.synchronize()
            barrier()
            tot_ms += e0.elapsed_time(e1)
            if out is not None:  # LOD step: build events first
                build_ms.append(ev[0].elapsed_time(ev[1]))
                frame_ms.append([ev[2 + 2 * k].elapsed_time(ev[3 + 2 * k]) for k in range(nf)])
                out.free()
            else:
                frame_ms.append([ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(nf)])
        launches = gblod.launch_count() - l0
        pr = gblod.probe_read() if probe is not None else None
        if probe is not None:
            gblod.probe_enable(gblod.K_ANY)
        return tot_ms, frame_ms, build_ms, launches, pr

    def per_view(frame_ms):
        """frame_ms[step][k] -> the times of each view over all steps and repeats"""
        return [[row[k] for row in frame_ms for k in range(j, nf, nv)] for j in range(nv)]

    # census of one LOD pass and one all-points pass over the views (untimed; the counts are
    # deterministic, so the timed frames have the same ones)
    tree = lod_step()
    lod_c = []
    for cam in views:
        r.render(tree, cam, par_count, image=img, accum=acc)
        lod_c.append(r.stats())
    all_c = []
    for cam in (views if not a.no_brute else []):
        r.render_bruteforce(xyz, mass, h, cam, par_count, image=img, accum=acc)
        all_c.append(r.stats())
    # visual equivalence (abstract: indistinguishable from a full rendering): LOD vs all points
    vis = []
    for cam in views[:: max(1, nv // 8)]:
        li, _ = r.render(tree, cam, par)
        bi, _ = r.render_bruteforce(xyz, mass, h, cam, par)
        d = (li.int() - bi.int()).abs().double()
        mse = float((d * d).mean())
        vis.append((float(d.max()), float(d.mean()), 10 * math.log10(255.0 ** 2 / mse) if mse > 0 else float("inf")))
    visual = {"frames": len(vis), "max_abs_u8": max(v[0] for v in vis),
              "mean_abs_u8": float(np.mean([v[1] for v in vis])), "psnr_db_mean": float(np.mean([v[2] for v in vis])),
              "psnr_db_min": float(min(v[2] for v in vis))}
    info = tree.info()
    tree.free()
    assert r.status() == gblod.OK

    # measured integer ceilings of this GPU (the per-pixel body of the radial rule, every pixel a hit;
    # and the issue rate of plain 32-bit adds)
    mb_ms, mb_units = gblod.microbench(gblod.MB_RADIAL, 4096)
    body_peak = mb_units / (mb_ms / 1e3) / 1e9  # G pixel updates/s
    alu_ms, alu_units = gblod.microbench(gblod.MB_ALU, 4096)
    alu_peak = alu_units / (alu_ms / 1e3) / 1e12  # T int32 ops/s

    clocks = Clocks(local)
    tot_ms, frame_ms, build_ms, launches, pr = timed(lod_step, 2 + 2 * nf, a.steps, a.warmup, probe=gblod.K_SPLAT)
    ck = clocks.stop()
    lod_view_ms = per_view(frame_ms)
    upd_step = reps * sum(c["pixel_updates"] for c in lod_c)  # pixel updates of one step's splat launches
    rec_step = reps * sum(c["pairs"] for c in lod_c)

    # 16-bit block codes (storage paragraph): the same frames drawn from 10-byte points
    block16 = None
    if not a.no_block16:
        tree = gblod.build_lod(xyz, mass, h, n_max=n_max, seed=1)
        bytes_f = int(tree.info().device_bytes)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record()
        tree.quantize(drop_float=True)
        q1.record()
        torch.cuda.synchronize()
        q_ms = q0.elapsed_time(q1)
        bytes_q = int(tree.info().device_bytes)
        par_q = gblod.make_params(lambda_px=lam, point_format=gblod.POINTS_BLOCK16)
        vq = []
        for cam in views[:: max(1, nv // 8)]:
            li, _ = r.render(tree, cam, par_q)
            bi, _ = r.render_bruteforce(xyz, mass, h, cam, par)
            d = (li.int() - bi.int()).abs().double()
            mse = float((d * d).mean())
            vq.append((float(d.max()), 10 * math.log10(255.0 ** 2 / mse) if mse > 0 else float("inf")))
        for cam in cams[: min(nf, 16)]:
            r.render(tree, cam, par_q, image=img, accum=acc)
        torch.cuda.synchronize()
        qf_ms = []
        qt_ms = 0.0
        for _ in range(a.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * nf)]
            for k, cam in enumerate(cams):
                ev[2 * k].record()
                r.render(tree, cam, par_q, image=img, accum=acc)
                ev[2 * k + 1].record()
            torch.cuda.synchronize()
            qf_ms += [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(nf)]
            qt_ms += ev[0].elapsed_time(ev[-1])
        assert r.status() == gblod.OK
        tree.free()
        block16 = {"bytes_per_point": 10, "bytes_per_point_fp32": 20,
                   "octree_device_bytes_fp32": bytes_f, "octree_device_bytes_block16_only": bytes_q,
                   "quantize_ms": q_ms, "frames_per_s_excl_build": a.steps * nf / (qt_ms / 1e3),
                   "p50_ms": float(np.percentile(qf_ms, 50)), "p99_ms": float(np.percentile(qf_ms, 99)),
                   "vs_all_points_max_abs_u8": max(v[0] for v in vq),
                   "vs_all_points_psnr_db_mean": float(np.mean([v[1] for v in vq]))}

    brute = None
    all_view_ms = None
    if not a.no_brute:
        b_ms, b_frames, _, _, _ = timed(brute_step, 2 * nf, a.steps, a.warmup)
        all_view_ms = per_view(b_frames)
        brute = dict(frames_per_s=a.steps * nf / (b_ms / 1e3), ms_per_frame=b_ms / (a.steps * nf),
                     splats_per_s=a.steps * reps * sum(c["splats"] for c in all_c) / (b_ms / 1e3),
                     points_per_s=a.steps * nf * p.n / (b_ms / 1e3),
                     p50_ms=float(np.percentile(b_frames, 50)), p99_ms=float(np.percentile(b_frames, 99)),
                     splats_per_frame=sum(c["splats"] for c in all_c) / nv,
                     pixel_updates_per_frame=sum(c["pixel_updates"] for c in all_c) / nv)
        if hbm:
            b_bytes = 20.0 * p.n + 17.0 * W * H
            brute["hbm_bytes_per_frame"] = b_bytes
            brute["hbm_frac"] = b_bytes / (b_ms / (a.steps * nf) / 1e3) / (hbm * 1e9)

    # batched views (one set of launches, no host waits) and its CUDA-graph replay
    batched = None
    if not a.no_batch:
        nbv = max(1, a.batch_views) if a.workload != "paper" else nv
        bcams = views[:: max(1, nv // nbv)][:nbv]
        # (tile, splat) records, 16 B each (2^29: 8 GiB; the eight paper-scale views need about 1.08e9
        # with 64x16 tiles, so 2^31: 32 GiB, and fewer with 32x32 tiles, which fit 2^30 but splat slower)
        cap = 1 << (a.batch_capacity_log2 or (31 if a.workload == "paper" else 29))
        tree = gblod.build_lod(xyz, mass, h, n_max=n_max, seed=1)
        bviews = [(tree, c, torch.empty((H, W), dtype=torch.uint8, device=dev),
                   torch.empty((H, W), dtype=torch.int64, device=dev)) for c in bcams]
        try:
            par_b, _ = r.autotune(bviews, gblod.make_params(lambda_px=lam), record_capacity=cap)
        except gblod.GblodError as e:  # every tile candidate overflowed the capacity: report, do not stop
            par_b = None
            batched = {"views": len(bviews), "record_capacity": cap, "status": int(e.code), "error": str(e)}
            r.status(reset=True)
            tree.free()
    if batched is None and not a.no_batch and par_b is not None:
        r.reserve_batch(bviews, par_b, record_capacity=cap)
        r.status(reset=True)

        def ev_time(fn, reps_):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps_):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps_

        def singles():
            for (t, c, im, ac) in bviews:
                r.render(t, c, par_b, image=im, accum=ac)

        ms_single = ev_time(singles, a.steps)
        ms_batch = ev_time(lambda: r.render_batch(bviews, par_b), a.steps)
        gs = torch.cuda.Stream()
        gs.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(gs):
            r.render_batch(bviews, par_b, stream=gs)
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=gs):
                r.render_batch(bviews, par_b, stream=gs)
        torch.cuda.synchronize()
        ms_graph = ev_time(graph.replay, a.steps)
        st = int(r.status())
        batched = {"views": len(bviews), "resolution": f"{W}x{H}", "tile": [par_b.tile_w, par_b.tile_h],
                   "record_capacity": cap, "status": st,
                   "views_per_s_one_at_a_time": len(bviews) / (ms_single / 1e3),
                   "views_per_s_batch": len(bviews) / (ms_batch / 1e3) if st == 0 else None,
                   "views_per_s_graph_replay": len(bviews) / (ms_graph / 1e3) if st == 0 else None}
        del graph
        tree.free()

    # end to end through the public API: pinned host particles in, every u8 frame out, every step.  The
    # copy of step s+1's particles runs on a second stream (into the other of two device buffers) while
    # step s renders; every step's copy is inside the timed region, the first one not overlapped.
    e2e = None
    if not a.no_e2e:
        hx, hm, hh = (torch.from_numpy(x).pin_memory() for x in (p.xyz, p.mass, p.h))
        out_h = torch.empty((nf, H, W), dtype=torch.uint8).pin_memory()
        bufs = [(torch.empty_like(xyz), torch.empty_like(mass), torch.empty_like(h)) for _ in range(2)]
        cs = torch.cuda.Stream()
        ready = [torch.cuda.Event(), torch.cuda.Event()]

        def copy_in(slot):
            with torch.cuda.stream(cs):
                dx, dm, dh = bufs[slot]
                dx.copy_(hx, non_blocking=True)
                dm.copy_(hm, non_blocking=True)
                dh.copy_(hh, non_blocking=True)
                ready[slot].record(cs)

        def e2e_step(slot, prefetch):
            torch.cuda.current_stream().wait_event(ready[slot])
            t = gblod.build_lod(*bufs[slot], n_max=n_max, seed=1)  # returns once the octree is built
            if prefetch:
                copy_in(slot ^ 1)
            for k, cam in enumerate(cams):
                im, _ = r.render(t, cam, par, image=img, accum=acc)
                out_h[k].copy_(im, non_blocking=True)
            torch.cuda.synchronize()
            t.free()

        copy_in(0)
        e2e_step(0, False)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        copy_in(0)
        for i in range(a.steps):
            e2e_step(i & 1, i + 1 < a.steps)
        torch.cuda.synchronize()
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": None, "unit": "frames/s", "h2d_bytes_per_step": int(p.xyz.nbytes + p.mass.nbytes + p.h.nbytes),
               "d2h_bytes_per_step": int(nf * W * H),
               "note": "each step's particles copied from pinned host memory on a second stream during the previous "
                       "step's frames (double-buffered); every frame's u8 image copied back", "_s": e2e_s}

    # reduce over ranks: slowest time, all frames
    tot_ms, e2e_s, frames_all = combine_ranks(tot_ms, e2e["_s"] if e2e else 0.0, a.steps * nf, world, dev)
    value = frames_all / (tot_ms / 1e3)
    if e2e:
        e2e.pop("_s")
        e2e["value"] = frames_all / e2e_s
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    splat_ms, splat_launches = pr
    achieved = a.steps * upd_step / (splat_ms / 1e3) / 1e9 if splat_ms > 0 else 0.0
    rec_per_launch = a.steps * rec_step / max(splat_launches, 1)
    lod_frame_s = float(np.sum(frame_ms)) / 1e3
    vlist = []
    for j, cam in enumerate(views):
        lm = lod_view_ms[j]
        v = {"view": j, "lod_p50_ms": float(np.percentile(lm, 50)), "lod_p99_ms": float(np.percentile(lm, 99)),
             "lod_fps": 1e3 / float(np.mean(lm)), "lod_splats": int(lod_c[j]["splats"]),
             "lod_pixel_updates": int(lod_c[j]["pixel_updates"]), "lod_records": int(lod_c[j]["pairs"]),
             "lod_splats_per_s": lod_c[j]["splats"] / (float(np.mean(lm)) / 1e3),
             "lod_gupdates_per_s": lod_c[j]["pixel_updates"] / (float(np.mean(lm)) / 1e3) / 1e9}
        v["lod_frac_of_body_peak"] = v["lod_gupdates_per_s"] / body_peak
        if hbm:
            v["lod_hbm_frac"] = (20.0 * lod_c[j]["points"] + 17.0 * W * H) / (float(np.mean(lm)) / 1e3) / (hbm * 1e9)
        if all_view_ms is not None:
            am = all_view_ms[j]
            v.update({"all_p50_ms": float(np.percentile(am, 50)), "all_p99_ms": float(np.percentile(am, 99)),
                      "all_fps": 1e3 / float(np.mean(am)), "all_splats": int(all_c[j]["splats"]),
                      "all_pixel_updates": int(all_c[j]["pixel_updates"]),
                      "all_gupdates_per_s": all_c[j]["pixel_updates"] / (float(np.mean(am)) / 1e3) / 1e9})
            v["all_frac_of_body_peak"] = v["all_gupdates_per_s"] / body_peak
            if hbm:
                v["all_hbm_frac"] = (20.0 * p.n + 17.0 * W * H) / (float(np.mean(am)) / 1e3) / (hbm * 1e9)
        vlist.append(v)
    flat = [x for row in frame_ms for x in row]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "frames/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": tot_ms / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 projection, u64 fixed-point accumulation, f64 node criterion",
        "data": "synthetic",
        "config": workload_config(a, p, views, reps, n_max, lam, desc, info),
        "lod": {"frames_per_s_excl_build": a.steps * nf / lod_frame_s,
                "splats_per_s": a.steps * reps * sum(c["splats"] for c in lod_c) / (tot_ms / 1e3),
                "p50_ms": float(np.percentile(flat, 50)), "p99_ms": float(np.percentile(flat, 99)),
                "points_per_frame": sum(c["points"] for c in lod_c) / nv,
                "splats_per_frame": sum(c["splats"] for c in lod_c) / nv,
                "nodes_per_frame": sum(c["nodes_selected"] for c in lod_c) / nv,
                "pixel_updates_per_frame": sum(c["pixel_updates"] for c in lod_c) / nv},
        "views": vlist,
        "build": {"ms": float(np.median(build_ms)), "particles_per_s": p.n / (np.median(build_ms) / 1e3)},
        "visual_equivalence": visual,
        "all_points": brute,
        "block16": block16,
        "batched": batched,
        "clocks": ck,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": {"kernel": "k_splat_tiles (R3)", "bound": "alu", "achieved": achieved, "peak": body_peak,
                     "unit": "G pixel updates/s", "frac": achieved / body_peak if body_peak else None,
                     "traffic": splat_traffic(rec_per_launch),
                     "peak_note": "measured: the radial rule's per-pixel body (every pixel inside the support, no "
                                  "list or staging work) on all SMs, gblod_microbench(GBLOD_MB_RADIAL); of measured",
                     "int32_issue_peak_tops": alu_peak, "ops_per_update": OPS_PER_PIXEL_UPDATE,
                     "achieved_int32_tops": achieved * OPS_PER_PIXEL_UPDATE / 1e3,
                     "traffic_note": "DRAM read + write bytes per launch: one ncu capture of the splat kernel, per "
                                     "(tile, splat) record, times this run's records per launch; null when the "
                                     "binning rule or the kernel source differs from the captured one",
                     "launches": int(splat_launches), "avg_launch_ms": splat_ms / max(splat_launches, 1),
                     "records_per_launch": rec_per_launch},
    }
    if not a.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(a, p, views, n_max, lod_c, info)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def workload_config(a, p, views, reps, n_max, lam, desc, info=None) -> dict:
    """The `config` object both arms print for a workload."""
    c = {"workload": desc, "particles": int(p.n), "views": len(views), "view_repeats_per_step": reps,
         "frames_per_step": len(views) * reps, "resolution": f"{views[0]['width']}x{views[0]['height']}",
         "n_max": n_max, "lambda_px": lam, "kernel": "gaussian, sigma = h, 3-sigma support",
         "step": "build_lod + every frame of the step at level of detail",
         "l2": "flushed between steps (256 MiB write); particles and octree exceed the 129 MB L2"}
    if info is not None:  # (nodes, stored points): the GPU octree's info or the oracle tree's sizes
        c["octree_nodes"], c["octree_points"] = (int(info.n_nodes), int(info.n_points)) \
            if hasattr(info, "n_nodes") else (int(info[0]), int(info[1]))
    return c


def measured_peaks() -> dict:
    f = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(f))
    except (OSError, ValueError):
        return {}


def splat_source(src: bytes) -> bytes:
    """The text the splat kernel's traffic depends on: render.cu's rule for which points are binned
    (from `constexpr int DIRECT_BOX` to the end of `direct_box`) followed by the kernel itself (from
    `struct SplatSmem` to the end of `k_splat_tiles`)."""
    r0 = src.index(b"constexpr int DIRECT_BOX")
    r1 = src.index(b"\n}\n", src.index(b"bool direct_box(", r0)) + 3
    a = src.index(b"struct SplatSmem {")
    b = src.index(b"\n}\n", src.index(b"k_splat_tiles(", a)) + 3
    return src[r0:r1] + src[a:b]


# DRAM bytes of one ncu capture of the splat kernel (--set full, default tile, one launch: the frame of the
# 240-frame mid path given by path_frame, drawn by the census pass), the (tile, splat) records that launch
# splatted, and the sha256 of the source text above at the time of the capture; the ncu summary under
# profiles/ lists the same numbers.
SPLAT_CAPTURE = {"source_sha256": "43431129b19828e79d7dd5b5cbfdb3ba480cc69ee7530652f95403c43cb1e979",
                 "path_frame": 160, "records": 24527161, "dram_read_bytes": 411.364096e6,
                 "dram_write_bytes": 16.684800e6}


def splat_traffic(records_per_launch: float):
    """DRAM bytes per splat launch: the capture above per record, times this run's records per launch;
    None if the kernel source differs from the captured one or the capture has no record count."""
    import hashlib
    try:
        src = open(os.path.join(ROOT, "paper_0811_2055_gb300", "csrc", "render.cu"), "rb").read()
    except OSError:
        return None
    if hashlib.sha256(splat_source(src)).hexdigest() != SPLAT_CAPTURE["source_sha256"]:
        return None
    if not SPLAT_CAPTURE["records"] or not records_per_launch:
        return None
    captured = SPLAT_CAPTURE["dram_read_bytes"] + SPLAT_CAPTURE["dram_write_bytes"]
    return captured / SPLAT_CAPTURE["records"] * records_per_launch


# ------------------------------------------------------------------ the oracle (CPU)

def _oracle_threads_all() -> int:
    from oracle import oracle as O
    O.set_threads(0)
    return O.get_threads()


def cpu_baseline(a, p, views, n_max, lod_c, info):
    """The oracle (test infrastructure, plain C) on the host cores, on a bounded sample of the same
    workload: it builds the octree of every 16th particle (1 thread; build time scaled to all
    particles by their count) and draws the sample octree's frames of the last two views at 1 thread
    and at all threads; its pixel-update rate (updates of the sample frames over their time) then
    prices the full workload's frames, whose update counts the census gave (the oracle's frames are
    bit-identical).  Returns the frames/s of one step of the full workload at all threads."""
    from oracle import oracle as O
    from paper_0811_2055_gb300 import synth
    k = 16
    sub = p.subset(np.arange(0, p.n, k))
    O.set_threads(1)
    t0 = time.perf_counter()
    T = O.build_tree(sub.xyz, sub.mass, sub.h, seed=1, n_max=n_max)
    t_build = time.perf_counter() - t0
    rp = O.rparams(lambda_px=math.sqrt(n_max))
    vs = views[-2:]
    rates = {}
    for th in (1, 0):
        O.set_threads(th)
        upd, secs = 0, 0.0
        for cam in vs:
            c = dict(cam, width=cam["width"] // 4, height=cam["height"] // 4, f_px=cam["f_px"] / 4,
                     cx=cam["cx"] / 4, cy=cam["cy"] / 4) if th == 1 else cam
            t0 = time.perf_counter()
            _, _, _, _, nu = O.render_lod_counted(T, c, rp)
            secs += time.perf_counter() - t0
            upd += nu
        rates[th] = upd / secs
    cores = _oracle_threads_all()
    reps = a.view_repeats if a.workload == "paper" else 1
    step_upd = reps * sum(c["pixel_updates"] for c in lod_c)
    t_step = t_build * k + step_upd / rates[0]
    O.set_threads(0)
    return {"value": reps * len(views) / t_step, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle octree of every {k}th particle ({sub.n}; 1-thread build {t_build:.1f} s, x{k} for all "
                      f"particles) and its LOD frames of views {len(views) - 2}..{len(views) - 1} (1 thread at "
                      f"quarter resolution, all {cores} threads at full resolution); the all-thread pixel-update "
                      f"rate prices the step's {step_upd:.3g} census updates",
            "updates_per_s_1_thread": rates[1], "updates_per_s_all_threads": rates[0],
            "build_s_1_thread_estimated_all_particles": t_build * k}


def band_rows(H: int, b: int, nb: int) -> tuple[int, int]:
    """Rows [b H/nb, (b+1) H/nb) of a frame of height H."""
    bh = H // nb
    return b * bh, (b + 1) * bh


def run_reference(a):
    """The CPU oracle on the same workload and metric.  Setup (untimed, reported): the oracle builds
    the octree of every particle.  Each step draws one horizontal band of 1/36 of one view's rows
    (the oracle's row window: the whole frame's selection and projection with the pixel loops limited
    to the band, so the band is exactly those rows of the frame), cycling over views and bands; value
    = frames drawn (band fractions) / time."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from oracle import oracle as O
    p, views, n_max, desc = workload(a.workload, a.frames, a.particles, a.path_frames, a.view_list)
    reps = max(1, a.view_repeats) if a.workload == "paper" else 1
    lam = math.sqrt(n_max)
    cores = _oracle_threads_all()
    t0 = time.perf_counter()
    T = O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=n_max)
    t_build = time.perf_counter() - t0
    rp = O.rparams(lambda_px=lam)
    H = views[0]["height"]
    nb = 36 if H % 36 == 0 else 1
    bh = H // nb

    def band(s):
        r0, r1 = band_rows(H, (7 * s + 11 * (s // len(views))) % nb, nb)
        return O.render_lod_rows(T, views[s % len(views)], rp, r0, r1)

    for s in range(a.warmup):
        band(s)
    ts = []
    for s in range(a.warmup, a.warmup + a.steps):
        t0 = time.perf_counter()
        band(s)
        ts.append(time.perf_counter() - t0)
    frac = bh / H
    value = a.steps * frac / sum(ts)
    sample = (f"oracle (plain C, {cores} threads): octree of all {p.n} particles built once before the steps "
              f"({t_build:.1f} s, 1 thread, not in the steps); each step draws a band of {bh} of the {H} rows of one "
              f"view ({frac:.4f} of a frame), cycling over views and bands")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * float(np.mean(ts)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 oracle, f32 projection",
            "data": "synthetic", "config": workload_config(a, p, views, reps, n_max, lam, desc,
                                                           (len(T.nodes), int(T.hs.shape[0]))),
            "oracle_build_s": t_build,
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fibonacci_views(n: int, radius: float = 1.5, size: int = 256):
    from paper_0811_2055_gb300 import synth
    out = []
    g = math.pi * (3.0 - math.sqrt(5.0))
    for k in range(n):
        y = 1.0 - 2.0 * (k + 0.5) / n
        rr = math.sqrt(max(0.0, 1.0 - y * y))
        e = (0.5 + radius * rr * math.cos(g * k), 0.5 + radius * y, 0.5 + radius * rr * math.sin(g * k))
        out.append(synth.look_at(e, (0.5, 0.5, 0.5), width=size, height=size))
    return out


def run_diff(a):
    """Differentiation workload: fit a 1M-point representative set (xyz, weight, log h) so that its
    float-splat images match those of a 2^24-particle parent from 256 views at 256x256 (L2 loss,
    Adam, gradients from the adjoint splat kernel).  One step = forward + adjoint over all views."""
    import torch

    from paper_0811_2055_gb300 import gblod, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n_parent = a.particles or (1 << 24)
    parent = synth.mid(n_parent, seed=synth.SEED_BASE + 3)
    n_rep = max(1, n_parent // 16)
    cams = fibonacci_views(256)
    r = gblod.Renderer()
    par = gblod.make_params()
    pxyz, pw = (torch.from_numpy(x).to(dev) for x in (parent.xyz, parent.mass))
    pl = torch.from_numpy(np.log(np.maximum(parent.h, 1e-6)).astype(np.float32)).to(dev)
    t0 = time.perf_counter()
    target = gblod.diff_render(r, pxyz, pw, pl, cams, par)
    torch.cuda.synchronize()
    t_target = time.perf_counter() - t0
    rng = np.random.Generator(np.random.Philox(key=synth.SEED_BASE + 33))
    pick = rng.choice(parent.n, n_rep, replace=False)
    scale = parent.n / n_rep
    x = torch.tensor(parent.xyz[pick], device=dev, requires_grad=True)
    wv = torch.full((n_rep,), float(parent.mass.sum()) / n_rep, device=dev, requires_grad=True)
    lh = torch.tensor(np.log(np.maximum(parent.h[pick], 1e-6) * scale ** (1 / 3)).astype(np.float32), device=dev,
                      requires_grad=True)
    opt = torch.optim.Adam([{"params": [x], "lr": 1e-4}, {"params": [wv], "lr": 0.05}, {"params": [lh], "lr": 5e-3}])
    losses = []

    def step():
        opt.zero_grad()
        img = gblod.SplatImages.apply(x, wv, lh, cams, r, par)
        loss = ((img - target) ** 2).sum()
        loss.backward()
        opt.step()
        return loss.detach()

    for _ in range(a.warmup):
        losses.append(float(step()))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        losses.append(float(step()))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    line = {"metric": "views/s, forward + adjoint float splat (fit of LOD representatives)",
            "value": len(cams) / (ms / 1e3), "unit": "views/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"diff: {n_rep} representatives fitted to a {parent.n}-particle mid-recipe parent, "
                                   "256 views on a Fibonacci sphere of radius 1.5, 256x256, L2 image loss, Adam",
                       "views": len(cams), "resolution": "256x256"},
            "target_render_s": t_target, "loss_first": losses[0], "loss_last": losses[-1],
            "loss_curve": losses}
    print(json.dumps(line), flush=True)


def run_fit(a):
    """Visual equivalence of fitted representatives: a 2^22-particle mid-recipe timestep, the internal
    nodes that eight 1920x1080 views of the fly-through draw are fitted to their particles' images
    (fit.fit_node: Adam on the adjoint splat, views around each node at the distance it is drawn) and
    written back; the eight LOD frames are compared with the all-particle frames before and after."""
    import torch

    from paper_0811_2055_gb300 import fit, gblod, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    p = synth.mid(a.particles or (1 << 22))
    d = [torch.from_numpy(x).to(dev) for x in (p.xyz, p.mass, p.h)]
    n_max = 16000
    lam = math.sqrt(n_max)
    tree = gblod.build_lod(*d, n_max=n_max, seed=1)
    r = gblod.Renderer()
    par = gblod.make_params(lambda_px=lam)
    cams = [synth.helix_view(k) for k in range(0, 240, 30)]
    nodes = tree.export_nodes()
    drawn = set()
    for cam in cams:
        r.render(tree, cam, par)
        drawn |= {int(i) for i in r.last_selection() if nodes[int(i)]["flags"] & gblod.NODE_INTERNAL}
    full = [r.render_bruteforce(*d, cam, par) for cam in cams]

    def score():
        out = []
        for cam, (bi, ba) in zip(cams, full):
            li, la = r.render(tree, cam, par)
            dd = (li.int() - bi.int()).double()
            mse = float((dd * dd).mean())
            ea = (gblod.u64(la).astype(np.float64) - gblod.u64(ba).astype(np.float64))
            rel = float(np.sqrt((ea ** 2).sum() / (gblod.u64(ba).astype(np.float64) ** 2).sum()))
            out.append((10 * math.log10(255.0 ** 2 / mse) if mse > 0 else float("inf"), float(dd.abs().max()), rel))
        return {"psnr_db_mean": float(np.mean([o[0] for o in out])), "psnr_db_min": float(min(o[0] for o in out)),
                "max_abs_u8": max(o[1] for o in out), "rel_l2_accum_mean": float(np.mean([o[2] for o in out]))}

    before = score()
    t0 = time.perf_counter()
    losses = []
    for node in sorted(drawn):
        views = fit.node_views(tree, node, lam, n_views=6, size=128) + \
            fit.node_views(tree, node, lam, n_views=6, size=128, margin=3.0)
        res = fit.fit_node(tree, node, *d, views, steps=a.fit_steps, renderer=r)
        losses.append(res["loss_last"] / max(res["loss_first"], 1e-30))
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    after = score()
    assert r.status() == gblod.OK
    line = {"metric": "visual equivalence of LOD frames with fitted representatives: PSNR (dB) of the 8-bit LOD frame "
                      "against the all-particle frame",
            "value": after["psnr_db_mean"], "unit": "dB", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 fit, u64 frames",
            "data": "synthetic",
            "config": {"workload": f"fit: {p.n} mid-recipe particles, n_max {n_max}, the internal nodes drawn by 8 views "
                                   "of the 240-frame 1920x1080 fly-through, 12 fit views of 128x128 per node at two distances, "
                                   "log-intensity L2 loss, "
                                   f"{a.fit_steps} Adam steps", "nodes_fitted": len(drawn)},
            "random_subselection": before, "fitted": after, "fit_s": t_fit,
            "node_loss_ratio_median": float(np.median(losses)) if losses else None}
    r.close()
    tree.free()
    print(json.dumps(line), flush=True)


def run_paper_views(a):
    """Paper-scale timestep (150M particles): build, then every one of the eight views at 1920x1080
    and 3840x2160, LOD and all points, each timed `--repeats` times (p50/p99 per view)."""
    import torch

    from paper_0811_2055_gb300 import gblod, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    p = synth.paper_scale(a.particles) if a.particles else synth.paper_scale()
    t_gen = time.perf_counter() - t0
    xyz, mass, h = (torch.from_numpy(x).to(dev) for x in (p.xyz, p.mass, p.h))
    n_max = 16000
    lam = math.sqrt(n_max)
    r = gblod.Renderer()
    par = gblod.make_params(lambda_px=lam)
    par_count = gblod.make_params(lambda_px=lam, count_updates=True)
    bms = []
    for _ in range(3 + a.warmup):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tree = gblod.build_lod(xyz, mass, h, n_max=n_max, seed=1)
        e1.record()
        torch.cuda.synchronize()
        bms.append(e0.elapsed_time(e1))
        info = tree.info()
        tree.free()
    bms = bms[a.warmup:]
    tree = gblod.build_lod(xyz, mass, h, n_max=n_max, seed=1)
    info = tree.info()
    peaks = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    def timed(fn, reps):
        for _ in range(a.warmup):
            fn()
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    views = []
    lod_1080 = []
    clocks = Clocks(0)
    for (W, H) in ((1920, 1080), (3840, 2160)):
        img = torch.empty((H, W), dtype=torch.uint8, device=dev)
        acc = torch.empty((H, W), dtype=torch.int64, device=dev)
        for j in range(8):
            cam = synth.paper_view(j, W, H)
            lms = timed(lambda: r.render(tree, cam, par, image=img, accum=acc), a.repeats)
            r.render(tree, cam, par_count, image=img, accum=acc)
            ls = r.stats()
            bms_ = timed(lambda: r.render_bruteforce(xyz, mass, h, cam, par, image=img, accum=acc), a.repeats)
            r.render_bruteforce(xyz, mass, h, cam, par_count, image=img, accum=acc)
            bs = r.stats()
            b_bytes = 20 * p.n + W * H
            v = {"view": j, "resolution": f"{W}x{H}", "lod_p50_ms": float(np.percentile(lms, 50)),
                 "lod_p99_ms": float(np.percentile(lms, 99)), "lod_fps": 1e3 / float(np.mean(lms)),
                 "lod_splats": ls["splats"], "lod_points": ls["points"], "lod_pixel_updates": ls["pixel_updates"],
                 "lod_splats_per_s": ls["splats"] / (float(np.mean(lms)) / 1e3),
                 "all_p50_ms": float(np.percentile(bms_, 50)), "all_p99_ms": float(np.percentile(bms_, 99)),
                 "all_fps": 1e3 / float(np.mean(bms_)), "all_splats": bs["splats"],
                 "all_pixel_updates": bs["pixel_updates"],
                 "all_hbm_frac": b_bytes / (float(np.mean(bms_)) / 1e3) / (hbm * 1e9)}
            views.append(v)
            if H == 1080:
                lod_1080.append(float(np.mean(lms)))
    ck = clocks.stop()
    assert r.status() == gblod.OK
    line = {"metric": "1080p LOD frames/s over the eight paper-scale views (150M particles); per-view LOD and "
                      "all-points frames/s, splats/s, p50/p99",
            "value": 8 / (sum(lod_1080) / 1e3), "unit": "frames/s", "n_gpus": 1, "steps": a.repeats,
            "warmup": a.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 projection, u64 fixed-point accumulation, f64 node criterion", "data": "synthetic",
            "config": {"workload": "paper: 150M particles (65,536 NFW halos + central halo with 30% + 10% uniform), "
                                   "n_max 16000, eight views d_j = 0.01 * 150^(j/7) from the central halo, "
                                   "1920x1080 and 3840x2160", "particles": p.n, "octree_nodes": int(info.n_nodes),
                       "octree_points": int(info.n_points), "octree_bytes": int(info.device_bytes)},
            "build_ms": float(np.median(bms)), "build_particles_per_s": p.n / (float(np.median(bms)) / 1e3),
            "generate_s": t_gen, "hbm_gbs_peak": hbm, "views": views, "clocks": ck}
    tree.free()
    print(json.dumps(line), flush=True)


def run_serve(a):
    """Serving workload: 16 device-resident timesteps (halo drift), 64 viewer sessions at mixed
    resolutions (720p/1080p/4K) with Poisson requests at 30 Hz each, admission by an HBM budget,
    continuous batching over two streams; a newer request of a session supersedes its queued one."""
    import torch

    from paper_0811_2055_gb300 import gblod, serve, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = a.particles or 75_000_000
    t0 = time.perf_counter()
    base = synth.timesteps_recipe(n)
    t_gen = time.perf_counter() - t0
    x0, vel = torch.from_numpy(base.xyz).to(dev), torch.from_numpy(base.vel).to(dev)
    mass, h = torch.from_numpy(base.mass).to(dev), torch.from_numpy(base.h).to(dev)
    del base
    trees = []
    t0 = time.perf_counter()
    for t in range(16):
        xt = torch.remainder(x0 + t * vel, 1.0).contiguous()
        trees.append(gblod.build_lod(xt, mass, h, n_max=16000, seed=1))
        del xt
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    del x0, vel
    res_choices = [(1280, 720), (1920, 1080), (3840, 2160)]
    res, reqs = serve.poisson_requests(a.sessions, 30.0, a.duration, len(trees), res_choices, seed=0)
    loop = serve.ServingLoop(trees, hbm_budget_bytes=int(a.session_budget_gb * (1 << 30)), max_views=16,
                             record_capacity=1 << 30, supersede=True)
    admitted = [loop.admit(s, w, hh) for s, (w, hh) in enumerate(res)]
    loop.reserve([(trees[0], synth.look_at((0.5, 0.5, -1), (0.5, 0.5, 0.5), width=3840, height=2160))] * 16)
    done = loop.run(reqs, a.duration)
    st = serve.latency_stats(done, a.duration)
    offered = sum(1 for q in reqs if admitted[q.session])
    line = {"metric": "serving: frames/s and p50/p99 frame latency (arrival -> 8-bit image on the host)",
            "value": st.get("frames_per_s", 0.0), "unit": "frames/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/u64", "data": "synthetic",
            "config": {"workload": f"serve: 16 timesteps x {n} particles (32,768 drifting NFW halos + 10% uniform), "
                                   f"{a.sessions} sessions at 720p/1080p/4K, Poisson 30 Hz each, {a.duration} s",
                       "session_budget_gb": a.session_budget_gb, "max_views_per_batch": 16, "streams": 2},
            "p50_ms": st.get("p50_ms"), "p99_ms": st.get("p99_ms"), "completed": st.get("completed", 0),
            "sessions_admitted": int(sum(admitted)), "sessions_rejected": int(len(admitted) - sum(admitted)),
            "requests_offered_admitted": offered, "superseded": loop.stats["superseded"],
            "batches": loop.stats["batches"], "overflow_batches": loop.stats["overflow_batches"],
            "generate_s": t_gen, "build_16_timesteps_s": t_build}
    loop.close()
    print(json.dumps(line), flush=True)


def main():
    a = args_()
    if a.warmup < 3:
        a.warmup = 3
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "diff":
        run_diff(a)
    elif a.workload == "serve":
        run_serve(a)
    elif a.workload == "paper-views":
        run_paper_views(a)
    elif a.workload == "fit":
        run_fit(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
