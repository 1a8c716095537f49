"""Serving loop: resident scenes, admission by workspace memory, continuous
batching of render requests into one persistent launch per batch.

Every step that touches the GPU is a libaaag call (frame graphs and
aaag_render_batch); this module only schedules.

* Scenes stay resident in HBM (`DeviceScene`).
* Slots: a memory budget is divided into workspaces that each fit the
  largest view of the workload (any scene, any request resolution).  A request
  (1 view, or 2 for stereo) is admitted when enough slots are free: admission
  is by workspace memory.
* Per slot and (scene, resolution), preprocess -> cull -> sort is a captured
  CUDA graph re-aimed at each request's camera (aaag_graph_launch); slots run
  on their own streams, so requests overlap on the device.
* A batch of admitted views is rendered by one aaag_render_batch launch:
  persistent blocks take (view, tile) items from a shared counter.
* Continuous batching (`serve`): while one batch renders, the next one is
  prepared on other slots; a request arriving meanwhile joins the next batch
  as soon as slots free up.  At most two batches are in flight.
* Per-request pipelines (`serve_streams`): requests are admitted in arrival
  order as slots free up and run concurrently without a batch barrier; the
  views of a request (two for stereo) share one persistent render launch and
  the request completes on its own event.  Small requests may run on
  high-priority streams so that they overtake the blocks of large ones.

`plain_renderer` is the reference point: requests in arrival order, one at a
time, each view rendered with aaag_render_frame on one stream.

A request completes when its images (RGB and alpha of every view) have been
copied to pinned host memory: latency = that completion seen by the host minus
the arrival time.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import aaag


@dataclass
class Slot:
    ws: "aaag.Workspace"
    stream: torch.cuda.Stream
    rgb_flat: torch.Tensor
    alpha_flat: torch.Tensor
    graphs: dict = field(default_factory=dict)
    urgent: torch.cuda.Stream = None     # high-priority stream for small requests
    host_flat: torch.Tensor = None       # pinned host copy of the images (4 floats per pixel)

    def outputs(self, cam):
        hw = cam.width * cam.height
        return (self.rgb_flat[: 3 * hw].view(3, cam.height, cam.width),
                self.alpha_flat[:hw].view(cam.height, cam.width))

    def read_back(self, cam):
        """Queue the copy of this view's images to the slot's pinned host
        buffer on the current stream."""
        hw = cam.width * cam.height
        self.host_flat[: 3 * hw].copy_(self.rgb_flat[: 3 * hw], non_blocking=True)
        self.host_flat[3 * hw: 4 * hw].copy_(self.alpha_flat[:hw], non_blocking=True)


class Server:
    def __init__(self, scenes: dict, budget_bytes: int, max_width: int, max_height: int,
                 pair_capacity: int, max_batch_views: int = 8, device="cuda", params=None):
        self.scenes = {k: aaag.DeviceScene(v, device=device) for k, v in scenes.items()}
        self.structs = {k: v.struct() for k, v in self.scenes.items()}
        self.device = torch.device(device)
        self.params = params if params is not None else aaag.make_params()
        n_max = max(v.n for v in self.scenes.values())
        ws_bytes = aaag.aaag_workspace_bytes(n_max, max_width, max_height, pair_capacity)
        out_bytes = 16 * max_width * max_height
        n_slots = max(2, int(budget_bytes // (ws_bytes + out_bytes)))
        self.slot_bytes = ws_bytes + out_bytes
        self.slots = []
        for _ in range(n_slots):
            ws = aaag.Workspace(n_max, max_width, max_height, pair_capacity, device=device)
            self.slots.append(Slot(ws, torch.cuda.Stream(device=self.device),
                                   torch.empty(3 * max_width * max_height, device=device),
                                   torch.empty(max_width * max_height, device=device),
                                   urgent=torch.cuda.Stream(device=self.device, priority=-1),
                                   host_flat=torch.empty(4 * max_width * max_height, pin_memory=True)))
        self.render_stream = torch.cuda.Stream(device=self.device)
        self.max_batch_views = max_batch_views

    # -- graphs -----------------------------------------------------------
    def _graph(self, slot: Slot, scene: str, cam):
        key = (scene, cam.width, cam.height)
        g = slot.graphs.get(key)
        if g is None:
            g = aaag.aaag_graph_create(self.structs[scene], aaag.make_camera(cam), self.params, slot.ws.handle,
                                       aaag.AAAG_STAGE_PREPROCESS | aaag.AAAG_STAGE_CULL | aaag.AAAG_STAGE_SORT,
                                       None, None, slot.stream.cuda_stream)
            slot.graphs[key] = g
        return g

    def warm(self, requests):
        """Capture every (slot, scene, resolution) graph the trace will need."""
        shapes = {(r.scene, c.width, c.height): c for r in requests for c in r.cams}
        for slot in self.slots:
            for (scene, _, _), cam in shapes.items():
                self._graph(slot, scene, cam)
        torch.cuda.synchronize(self.device)

    def close(self):
        for slot in self.slots:
            for g in slot.graphs.values():
                aaag.aaag_graph_destroy(g)
            slot.graphs.clear()

    # -- one batch ----------------------------------------------------------
    def _launch(self, views):
        """views: list of (slot, request, camera).  Returns the done event."""
        events = []
        for slot, req, cam in views:
            aaag.aaag_graph_launch(self._graph(slot, req.scene, cam), aaag.make_camera(cam),
                                   slot.stream.cuda_stream)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
            events.append(ev)
        for ev in events:
            self.render_stream.wait_event(ev)
        outs = [slot.outputs(cam) for slot, _, cam in views]
        aaag.aaag_render_batch([slot.ws.handle for slot, _, _ in views], [o[0].data_ptr() for o in outs],
                               [o[1].data_ptr() for o in outs], self.render_stream.cuda_stream)
        with torch.cuda.stream(self.render_stream):
            for slot, _, cam in views:
                slot.read_back(cam)
        done = torch.cuda.Event()
        done.record(self.render_stream)
        return done

    def _launch_request(self, req, slots, urgent=False):
        """Per-request pipeline: every view's frame graph on its own slot
        stream, then one persistent render over the request's views on the
        first slot's stream.  `urgent` requests run on the slots'
        high-priority streams, so their blocks are scheduled before those of
        requests already running.  Returns the completion event."""
        streams = [s.urgent if urgent else s.stream for s in slots]
        for slot, cam, st in zip(slots, req.cams, streams):
            aaag.aaag_graph_launch(self._graph(slot, req.scene, cam), aaag.make_camera(cam), st.cuda_stream)
        lead = streams[0]
        for st in streams[1:]:
            ev = torch.cuda.Event()
            ev.record(st)
            lead.wait_event(ev)
        outs = [slot.outputs(cam) for slot, cam in zip(slots, req.cams)]
        aaag.aaag_render_batch([slot.ws.handle for slot in slots], [o[0].data_ptr() for o in outs],
                               [o[1].data_ptr() for o in outs], lead.cuda_stream)
        with torch.cuda.stream(lead):
            for slot, cam in zip(slots, req.cams):
                slot.read_back(cam)
        done = torch.cuda.Event()
        done.record(lead)
        return done

    def serve_streams(self, requests, capture=None, urgent_pixels=None, heavy_pixels=None, max_heavy=1):
        """Continuous per-request pipelines: requests are admitted as soon as
        their views fit into free slots (workspace memory), run concurrently
        on their slots' streams, and complete individually.
          urgent_pixels: requests of at most this many pixels in all run on
            high-priority streams, so they are not held behind the blocks of
            larger ones (None: no priorities).
          heavy_pixels: requests above this many pixels are "heavy": at most
            `max_heavy` of them are on the GPU at once, in arrival order,
            while lighter requests behind them are admitted (None: every
            request in arrival order).  Running heavy requests concurrently
            stretches each of them; running them one by one while the light
            ones overtake keeps their latency close to running alone.
        Same return value and `capture` as `serve`."""
        self.max_views_in_flight = 0
        order = sorted(requests, key=lambda r: r.arrival)
        pending = []
        free = list(self.slots)
        inflight = []
        lat = {}
        i = 0
        pixels = lambda r: sum(c.width * c.height for c in r.cams)
        heavy = lambda r: heavy_pixels is not None and pixels(r) > heavy_pixels
        n_heavy = 0
        t0 = time.perf_counter()
        while len(lat) < len(order):
            now = time.perf_counter() - t0
            while i < len(order) and order[i].arrival <= now:
                pending.append(order[i])
                i += 1
            progressed = False
            for item in list(inflight):
                done, req, slots = item
                if done.query():
                    lat[req.rid] = time.perf_counter() - t0 - req.arrival
                    if capture is not None:
                        for slot, cam in zip(slots, req.cams):
                            rgb, alpha = slot.outputs(cam)
                            capture.setdefault(req.rid, []).append((rgb.cpu(), alpha.cpu()))
                    free.extend(slots)
                    inflight.remove(item)
                    n_heavy -= heavy(req)
                    progressed = True
            # admission in arrival order; a heavy request waiting for its turn
            # blocks only later heavy ones
            k = 0
            heavy_blocked = False
            while k < len(pending):
                req = pending[k]
                is_heavy = heavy(req)
                if is_heavy and (heavy_blocked or n_heavy >= max_heavy):
                    heavy_blocked = True
                    k += 1
                    continue
                if len(free) < len(req.cams):
                    break
                pending.pop(k)
                slots = [free.pop() for _ in req.cams]
                urgent = urgent_pixels is not None and pixels(req) <= urgent_pixels
                inflight.append((self._launch_request(req, slots, urgent), req, slots))
                n_heavy += is_heavy
                self.max_views_in_flight = max(self.max_views_in_flight, len(self.slots) - len(free))
                progressed = True
            if not progressed:
                time.sleep(20e-6)
        return [lat[r.rid] for r in requests]

    def render_one(self, req):
        """Render one request through the serving path and wait (for tests)."""
        views = [(self.slots[i], req, cam) for i, cam in enumerate(req.cams)]
        self._launch(views).synchronize()
        return [slot.outputs(cam) for slot, _, cam in views]

    # -- the loop -----------------------------------------------------------
    def serve(self, requests, max_inflight: int = 2, capture=None):
        """Replay `requests` in real time (arrival offsets from now).  Returns
        per-request latency in seconds (completion observed by the host minus
        arrival).  With a dict `capture`, the images of every request are
        copied to it (rid -> [(rgb, alpha) per view], host tensors) before its
        slots are reused; `self.max_views_in_flight` records the peak number
        of views on the GPU."""
        self.max_views_in_flight = 0
        order = sorted(requests, key=lambda r: r.arrival)
        pending = collections.deque()
        free = list(self.slots)
        inflight = []
        lat = {}
        i = 0
        t0 = time.perf_counter()
        while len(lat) < len(order):
            now = time.perf_counter() - t0
            while i < len(order) and order[i].arrival <= now:
                pending.append(order[i])
                i += 1
            progressed = False
            for b in list(inflight):
                if b[0].query():
                    tdone = time.perf_counter() - t0
                    for r in b[1]:
                        lat[r.rid] = tdone - r.arrival
                    if capture is not None:
                        for slot, r, cam in b[3]:
                            rgb, alpha = slot.outputs(cam)
                            capture.setdefault(r.rid, []).append((rgb.cpu(), alpha.cpu()))
                    free.extend(b[2])
                    inflight.remove(b)
                    progressed = True
            if pending and len(inflight) < max_inflight:
                batch, views = [], []
                while pending and len(free) >= len(pending[0].cams) and \
                        len(views) + len(pending[0].cams) <= self.max_batch_views:
                    r = pending.popleft()
                    batch.append(r)
                    for cam in r.cams:
                        views.append((free.pop(), r, cam))
                if batch:
                    done = self._launch(views)
                    inflight.append((done, batch, [v[0] for v in views], views))
                    self.max_views_in_flight = max(self.max_views_in_flight,
                                                   len(self.slots) - len(free))
                    progressed = True
            if not progressed:
                time.sleep(20e-6)
        return [lat[r.rid] for r in requests]


def plain_renderer(scenes: dict, requests, max_width, max_height, pair_capacity, device="cuda", params=None):
    """The per-frame renderer: requests in arrival order, one at a time, every
    view through aaag_render_frame on one stream.  Returns per-request latency
    (s) on the same clock as Server.serve."""
    ds = {k: aaag.DeviceScene(v, device=device) for k, v in scenes.items()}
    structs = {k: v.struct() for k, v in ds.items()}
    n_max = max(v.n for v in ds.values())
    ws = aaag.Workspace(n_max, max_width, max_height, pair_capacity, device=device)
    stream = torch.cuda.Stream(device=device)
    rgb = torch.empty(3 * max_width * max_height, device=device)
    alpha = torch.empty(max_width * max_height, device=device)
    host = torch.empty(8 * max_width * max_height, pin_memory=True)   # two views
    prm = params if params is not None else aaag.make_params()
    # warm-up: one frame per shape
    for r in requests[:8]:
        for cam in r.cams:
            aaag.aaag_render_frame(structs[r.scene], aaag.make_camera(cam), prm, ws.handle, rgb.data_ptr(),
                                   alpha.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    lat = {}
    order = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in order:
        while time.perf_counter() - t0 < r.arrival:
            time.sleep(20e-6)
        for v, cam in enumerate(r.cams):
            aaag.aaag_render_frame(structs[r.scene], aaag.make_camera(cam), prm, ws.handle, rgb.data_ptr(),
                                   alpha.data_ptr(), stream.cuda_stream)
            hw = cam.width * cam.height
            with torch.cuda.stream(stream):
                host[4 * v * hw: 4 * v * hw + 3 * hw].copy_(rgb[: 3 * hw], non_blocking=True)
                host[4 * v * hw + 3 * hw: 4 * (v + 1) * hw].copy_(alpha[:hw], non_blocking=True)
        stream.synchronize()
        lat[r.rid] = time.perf_counter() - t0 - r.arrival
    return [lat[r.rid] for r in requests]


def latency_summary(lat_s, duration_s, n_views):
    a = np.asarray(lat_s) * 1e3
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "mean_ms": float(a.mean()), "max_ms": float(a.max()), "requests": int(a.size),
            "requests_per_s": a.size / duration_s, "views_per_s": n_views / duration_s}
