"""Serving loop: many concurrent viewers of device-resident octrees.

The paper has many users connect to one central data store, each running a viewer (the storage
paragraph); here the store is a set of octrees resident in HBM (one per timestep) and the viewers'
frame requests are rendered by continuous batching:

* sessions are admitted at start by an HBM budget (each admitted session holds `slots` frame
  buffers of its resolution: a uint64 fixed-point image and an 8-bit image);
* requests of admitted sessions queue FIFO; whenever one of the streams is free the scheduler takes
  the queued requests (up to `max_views`, one buffer slot each, and no more than the records the
  batch scratch holds, estimated from the (tile, splat) records per pixel of earlier batches) as
  one batch (`gblod_render_batch`, no host waits) and enqueues the copy of each 8-bit image to
  pinned host memory; requests that arrive while batches are on the GPU join the next batch as
  slots free up, and batches on different streams overlap on the device;
* a batch that overflows its reserved record capacity is re-rendered view by view with the exact
  single-view path, so every result is the same as that view rendered alone;
* latency = arrival of a request -> its 8-bit image in host memory.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np
import torch

from . import gblod


@dataclasses.dataclass
class Request:
    session: int
    arrival: float          # seconds since the loop started
    timestep: int
    camera: dict
    ready: float = math.nan
    slot: int = -1
    image: np.ndarray | None = None   # 8-bit image (kept with keep_images)
    accum: np.ndarray | None = None   # its 64-bit accumulation image (kept with keep_images)


@dataclasses.dataclass
class Session:
    sid: int
    width: int
    height: int
    admitted: bool = False
    free_slots: list = dataclasses.field(default_factory=list)


class ServingLoop:
    def __init__(self, octrees, params: gblod.RenderParams | None = None, hbm_budget_bytes: int = 2 << 30,
                 slots_per_session: int = 2, max_views: int = 16, streams: int = 2,
                 record_capacity: int = 1 << 27, keep_images: bool = False, supersede: bool = False):
        self.octrees = octrees
        self.params = params if params is not None else gblod.make_params()
        self.budget = int(hbm_budget_bytes)
        self.slots_per_session = slots_per_session
        self.max_views = max_views
        self.record_capacity = record_capacity
        self.keep_images = keep_images
        self.supersede = supersede
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.renderers = [gblod.Renderer() for _ in range(streams)]
        self.single = gblod.Renderer()
        self.sessions: dict[int, Session] = {}
        self.buffers = {}    # (sid, slot) -> (u8 image, u64 accum, pinned host image)
        self.used = 0
        self.reserved = [False] * streams
        self.rec_per_pixel = None   # (tile, splat) records per pixel seen so far (largest batch mean)
        self.safety = 1.5

    # ------------------------------------------------------------------ admission
    @staticmethod
    def session_bytes(width: int, height: int, slots: int) -> int:
        return slots * width * height * (8 + 1)

    def admit(self, sid: int, width: int, height: int) -> bool:
        need = self.session_bytes(width, height, self.slots_per_session)
        s = Session(sid, width, height)
        if self.used + need <= self.budget:
            s.admitted = True
            self.used += need
            for k in range(self.slots_per_session):
                img = torch.empty((height, width), dtype=torch.uint8, device=self.dev)
                acc = torch.empty((height, width), dtype=torch.int64, device=self.dev)
                host = torch.empty((height, width), dtype=torch.uint8).pin_memory()
                self.buffers[(sid, k)] = (img, acc, host)
                s.free_slots.append(k)
        self.sessions[sid] = s
        return s.admitted

    def reserve(self, worst_views):
        """Size every stream's batch scratch for `worst_views` (list of (octree, camera)): the
        cameras set the tiles and pixels; the octrees are replaced by the one with the most nodes
        and then by the deepest one, so that any batch of as many views fits."""
        infos = [t.info() for t in self.octrees]
        most = self.octrees[max(range(len(infos)), key=lambda i: infos[i].n_nodes)]
        deep = self.octrees[max(range(len(infos)), key=lambda i: infos[i].depth_max)]
        for tree in (most, deep):
            views = []
            for _, cam in worst_views[: self.max_views]:
                acc = torch.empty((cam["height"], cam["width"]), dtype=torch.int64, device=self.dev)
                views.append((tree, cam, None, acc))
            for k, r in enumerate(self.renderers):
                with torch.cuda.stream(self.streams[k]):
                    r.reserve_batch(views, self.params, record_capacity=self.record_capacity,
                                    stream=self.streams[k])
                self.reserved[k] = True
        torch.cuda.synchronize()

    # ------------------------------------------------------------------ the loop
    def run(self, requests: list[Request], duration: float, clock=time.perf_counter):
        """Serves `requests` (sorted by arrival, seconds from start) until `duration` has passed and
        every admitted request that arrived is done.  Returns the completed requests."""
        pending = [rq for rq in requests if self.sessions.get(rq.session) and self.sessions[rq.session].admitted]
        pending.sort(key=lambda q: q.arrival)
        queue: list[Request] = []
        inflight = [None] * len(self.streams)   # (event, [requests]) per stream
        done: list[Request] = []
        nxt = 0
        t0 = clock()
        overflow_batches = 0
        batches = 0
        superseded = 0
        while True:
            now = clock() - t0
            while nxt < len(pending) and pending[nxt].arrival <= now:
                rq = pending[nxt]
                if self.supersede:
                    before = len(queue)
                    queue = [q for q in queue if q.session != rq.session]
                    superseded += before - len(queue)
                queue.append(rq)
                nxt += 1
            # completions
            for k, fl in enumerate(inflight):
                if fl is None or not fl[0].query():
                    continue
                ev, reqs = fl
                st = self.renderers[k].status(reset=True, stream=self.streams[k])
                pairs = self.renderers[k].stats(stream=self.streams[k])["pairs"]
                pix = sum(self.sessions[q.session].width * self.sessions[q.session].height for q in reqs)
                rpp = pairs / max(pix, 1)
                self.rec_per_pixel = rpp if self.rec_per_pixel is None else max(0.9 * self.rec_per_pixel, rpp)
                if st == gblod.ERR_CAPACITY:
                    overflow_batches += 1
                    self._exact_fallback(reqs, k)
                tdone = clock() - t0
                for rq in reqs:
                    img, acc, host = self.buffers[(rq.session, rq.slot)]
                    rq.ready = tdone
                    if self.keep_images:
                        rq.image = host.numpy().copy()
                        rq.accum = acc.detach().cpu().numpy().view(np.uint64).copy()
                    self.sessions[rq.session].free_slots.append(rq.slot)
                    rq.slot = -1
                    done.append(rq)
                inflight[k] = None
            # launch a batch on every free stream
            for k in range(len(self.streams)):
                if inflight[k] is not None or not queue:
                    continue
                take, rest = [], []
                est = 0.0
                for rq in queue:
                    s = self.sessions[rq.session]
                    need = self._estimate(s)
                    fits = not take or est + need <= self.record_capacity
                    if len(take) < self.max_views and s.free_slots and fits:
                        rq.slot = s.free_slots.pop()
                        take.append(rq)
                        est += need
                    else:
                        rest.append(rq)
                if not take:
                    continue
                queue = rest
                self._launch(k, take)
                ev = torch.cuda.Event()
                ev.record(self.streams[k])
                inflight[k] = (ev, take)
                batches += 1
            if nxt >= len(pending) and not queue and all(f is None for f in inflight) and now >= duration:
                break
            if now > duration * 4 + 30:
                break  # overload guard: stop waiting for a backlog that cannot drain
        self.stats = {"batches": batches, "overflow_batches": overflow_batches, "superseded": superseded,
                      "unserved": len(pending) - len(done) - superseded}
        return done

    def _estimate(self, s: Session) -> float:
        """Records a view of this session is expected to need (unknown: a quarter of the capacity)."""
        if self.rec_per_pixel is None:
            return self.record_capacity / 4
        return self.safety * self.rec_per_pixel * s.width * s.height

    def _views(self, reqs):
        views = []
        for rq in reqs:
            img, acc, host = self.buffers[(rq.session, rq.slot)]
            views.append((self.octrees[rq.timestep], rq.camera, img, acc))
        return views

    def _launch(self, k, reqs):
        s = self.streams[k]
        views = self._views(reqs)
        with torch.cuda.stream(s):
            self.renderers[k].render_batch(views, self.params, stream=s)
            for rq, (_, _, img, _) in zip(reqs, views):
                host = self.buffers[(rq.session, rq.slot)][2]
                host.copy_(img, non_blocking=True)

    def _exact_fallback(self, reqs, k):
        s = self.streams[k]
        with torch.cuda.stream(s):
            for rq in reqs:
                img, acc, host = self.buffers[(rq.session, rq.slot)]
                self.single.render(self.octrees[rq.timestep], rq.camera, self.params, image=img, accum=acc, stream=s)
                host.copy_(img, non_blocking=True)
        s.synchronize()

    def close(self):
        for r in self.renderers:
            r.close()
        self.single.close()


# ------------------------------------------------------------------ synthetic viewers

def session_camera(sid: int, t: float, width: int, height: int, seed: int = 0) -> dict:
    """A smooth random camera path around the box centre (helix with a per-session phase)."""
    from . import synth
    rng = np.random.Generator(np.random.Philox(key=synth.SEED_BASE + 4000 + seed * 1000 + sid))
    ph, om, r0, dr, yy = rng.uniform(0, 2 * math.pi), rng.uniform(0.2, 0.8), rng.uniform(0.6, 1.4), \
        rng.uniform(0.05, 0.3), rng.uniform(-0.3, 0.3)
    ang = ph + om * t
    rad = r0 + dr * math.sin(0.5 * t + ph)
    eye = (0.5 + rad * math.cos(ang), 0.5 + yy + 0.1 * math.sin(0.3 * t), 0.5 + rad * math.sin(ang))
    return synth.look_at(eye, (0.5, 0.5, 0.5), width=width, height=height, z_near=1e-3)


def poisson_requests(n_sessions: int, rate_hz: float, duration: float, n_timesteps: int, resolutions,
                     seed: int = 0, advance_s: float = 2.0):
    """Poisson arrivals per session; each session starts at a random timestep that advances every
    `advance_s` seconds."""
    from . import synth
    rng = np.random.Generator(np.random.Philox(key=synth.SEED_BASE + 5000 + seed))
    res = [resolutions[int(rng.integers(len(resolutions)))] for _ in range(n_sessions)]
    t_start = rng.integers(0, n_timesteps, n_sessions)
    reqs = []
    for s in range(n_sessions):
        t = rng.exponential(1.0 / rate_hz)
        while t < duration:
            ts = int((t_start[s] + int(t // advance_s)) % n_timesteps)
            reqs.append(Request(s, float(t), ts, session_camera(s, t, res[s][0], res[s][1], seed)))
            t += rng.exponential(1.0 / rate_hz)
    reqs.sort(key=lambda q: q.arrival)
    return res, reqs


def latency_stats(done: list[Request], duration: float) -> dict:
    lat = np.array([q.ready - q.arrival for q in done]) * 1e3
    if lat.size == 0:
        return {"completed": 0}
    return {"completed": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "frames_per_s": lat.size / max(duration, max(q.ready for q in done))}
