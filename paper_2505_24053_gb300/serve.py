"""Continuous-batching render server over the geer C ABI.

A scene stays resident on the device. Requests (a camera each: pinhole, equidistant
or Kannala-Brandt, any pose) arrive over time. Each GPU buffer is a workspace with
a fixed slot layout (geer_set_camera_slots): every launch of a step depends only
on the number of occupied slots k, so the step (preprocess -> bin/sort ->
render) is captured once per k in a CUDA graph per buffer and replayed with the
cameras of the admitted requests. With two or more buffers on their own streams, requests that arrive
while a batch is on the GPU are admitted into the next free buffer and their
work overlaps on the device.

Admission is by slots and by memory: each request kind carries an estimate of
its (tile, Gaussian) pairs (calibrated by rendering it alone), and a batch takes
requests first come, first served while the estimates fit the buffer's pair
capacity. A batch that overflows anyway (the device status says so) is split and
its requests go back to the head of the queue.

Latency = request arrival -> completion event of its batch, measured with CUDA
events against a start event recorded when the trace starts. Each request also
carries host timestamps (admitted into a batch, launch call returned, completion
seen by the loop) and the GPU time its batch started, so that a slow request can
be traced to the step that held it: the queue, the host's launch, the GPU or the
loop noticing completion. The cyclic garbage collector is paused while a trace
runs (objects alive before it are frozen out of later collections): a full
collection over a large process heap can hold the loop for tens of
milliseconds.
"""
from __future__ import annotations

import gc
import math
import statistics
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import geer


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the trace start
    camera: object          # workloads.Camera
    kind: int = 0
    done_ms: float | None = None   # completion time, ms after the trace start
    batch: int = -1
    image: object = None
    error: str | None = None
    # host clock, ms after the trace start: admitted into a batch, launch call
    # returned, completion seen by the loop; GPU clock: the batch's first work
    admit_ms: float | None = None
    launch_ms: float | None = None
    seen_ms: float | None = None
    gpu_start_ms: float | None = None

    @property
    def latency_ms(self) -> float | None:
        return None if self.done_ms is None else self.done_ms - 1e3 * self.arrival


@dataclass
class Scheduler:
    """First come, first served admission by free slots and estimated pair memory.

    With same_kind, a batch takes the queue head and then only queued requests of
    the head's kind (in arrival order): a batch completes with its costliest
    request, so mixing a small request into a batch of large ones delays it."""

    n_slots: int
    pair_budget: int
    estimates: dict = field(default_factory=dict)   # kind -> estimated pairs
    default_estimate: int = 1
    same_kind: bool = False

    def estimate(self, req: Request) -> int:
        return int(self.estimates.get(req.kind, self.default_estimate))

    def admit(self, queue: deque) -> list:
        if self.same_kind and queue:
            kind = queue[0].kind
            batch, used, rest = [], 0, deque()
            while queue and len(batch) < self.n_slots:
                r = queue.popleft()
                e = self.estimate(r)
                if r.kind != kind or (batch and used + e > self.pair_budget):
                    rest.append(r)
                    continue
                batch.append(r)
                used += e
            queue.extendleft(reversed(rest))
            return batch
        batch, used = [], 0
        while queue and len(batch) < self.n_slots:
            e = self.estimate(queue[0])
            if batch and used + e > self.pair_budget:
                break
            batch.append(queue.popleft())
            used += e
        return batch

    def observe(self, req: Request, pairs: int):
        """Raise the estimate of a kind when a request needed more pairs."""
        self.estimates[req.kind] = max(self.estimate(req), int(pairs * 1.25))


class _Buffer:
    def __init__(self, idx, engine):
        import torch
        self.idx = idx
        self.engine = engine
        self.stream = torch.cuda.Stream()
        cap_cam = engine.capacity_camera
        self.ws = geer.Workspace([cap_cam] * engine.n_slots, engine.g.n, engine.g.sh_degree, engine.pair_capacity)
        self.rgb = torch.zeros((engine.n_slots * engine.slot_pixels, 3), dtype=torch.float32, device="cuda")
        self.graph = False
        self.graphs = {}
        self.done = None
        self.start = None
        self.batch = []
        self.batch_id = -1

    def load(self, reqs):
        """Cameras of a batch into slots 0..len(reqs)-1 (the step's shape is the batch size)."""
        cams = [r.camera for r in reqs] if reqs else [self.engine.capacity_camera]
        self.ws.set_camera_slots(cams, [True] * len(cams), self.engine.slot_tiles, self.engine.slot_pixels,
                                 stream=self.stream)

    def step_body(self):
        self.ws.preprocess(self.engine.g, stream=self.stream)
        self.ws.bin_sort(sync=False, stream=self.stream)
        self.ws.render_fwd(self.rgb, None, stream=self.stream)

    def capture(self):
        """One graph per batch size k = 1..n_slots: every launch configuration of a
        step depends only on k, so each is captured once and replayed."""
        import torch
        self.graphs = {}
        from . import workloads as wl
        small = wl.Camera(wl.PINHOLE, 64, 64, math.radians(60))  # launch shapes do not depend on it
        for k in range(1, self.engine.n_slots + 1):
            dummy = [Request(-1, 0.0, small)] * k
            self.load(dummy)
            self.step_body()  # warm the path outside capture
            self.stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=self.stream):
                self.step_body()
            self.graphs[k] = g
        self.graph = True

    def launch(self, reqs, batch_id):
        import torch
        self.start = torch.cuda.Event(enable_timing=True)
        self.load(reqs)
        with torch.cuda.stream(self.stream):
            # recorded after load's camera-table copies: start -> done spans the step
            self.start.record(self.stream)
            if self.graph:
                self.graphs[len(reqs)].replay()
            else:
                self.step_body()
            self.done = torch.cuda.Event(enable_timing=True)
            self.done.record(self.stream)
        self.batch = list(reqs)
        self.batch_id = batch_id

    def busy(self) -> bool:
        return self.done is not None and not self.done.query()


class Engine:
    """Serving engine: n_buffers workspaces x n_slots camera slots each."""

    def __init__(self, gaussians: geer.Gaussians, n_slots: int = 4, n_buffers: int = 2,
                 pair_capacity: int = 200_000_000, max_width: int = 1920, max_height: int = 1280,
                 use_graphs: bool = True, same_kind: bool = False):
        from . import workloads as wl
        self.g = gaussians
        self.n_slots, self.n_buffers = n_slots, n_buffers
        self.pair_capacity = pair_capacity
        self.capacity_camera = wl.Camera(wl.PINHOLE, max_width, max_height, math.radians(60))
        self.slot_tiles = math.ceil(max_width / 16) * math.ceil(max_height / 16)
        self.slot_pixels = max_width * max_height
        self.scheduler = Scheduler(n_slots, int(pair_capacity * 0.9), same_kind=same_kind)
        self.buffers = [_Buffer(i, self) for i in range(n_buffers)]
        self.use_graphs = use_graphs
        self.failed: list = []

    def calibrate(self, sample_requests, margin: float = 1.25):
        """Pairs per request kind, from rendering each sample alone (synchronous)."""
        buf = self.buffers[0]
        for r in sample_requests:
            buf.load([r])
            buf.ws.preprocess(self.g, stream=buf.stream)
            try:
                need = buf.ws.bin_sort(sync=True, stream=buf.stream)
            except geer.GeerError as e:
                if e.status != geer.ERR_CAPACITY:
                    raise
                need = buf.ws.last_pairs
            self.scheduler.observe(r, int(need * margin / 1.25))
        buf.stream.synchronize()

    def prepare(self):
        for b in self.buffers:
            b.load([])
            if self.use_graphs:
                b.capture()
            else:
                b.step_body()
            b.stream.synchronize()
            # the warm-up steps may have overflowed the pair capacity: read and clear
            # the device status so the first real batch does not inherit it
            b.ws.device_status(stream=b.stream)

    def _slot_view(self, buf, k, cam):
        n = cam.width * cam.height
        off = k * self.slot_pixels
        return buf.rgb[off:off + n].view(cam.height, cam.width, 3)

    def _complete(self, buf, t0, keep_images, out_done, seen_ms=None):
        st, pairs = buf.ws.device_status(stream=buf.stream)
        t_ms = t0.elapsed_time(buf.done)
        s_ms = t0.elapsed_time(buf.start)
        if st == geer.ERR_CAPACITY and len(buf.batch) == 1:
            # a single request beyond the pair capacity can never be served here
            buf.batch[0].error = "pair capacity exceeded"
            self.failed.append(buf.batch[0])
            requeue = []
        elif st == geer.ERR_CAPACITY:
            # split and retry the batch: back to the head of the queue, estimates raised
            for r in buf.batch:
                self.scheduler.observe(r, max(pairs // max(1, len(buf.batch)), self.scheduler.estimate(r)))
            requeue = list(buf.batch)
        else:
            if st != geer.OK:
                raise geer.GeerError(st, "serving batch")
            requeue = []
            for k, r in enumerate(buf.batch):
                r.done_ms = t_ms
                r.gpu_start_ms = s_ms
                r.seen_ms = seen_ms
                r.batch = buf.batch_id
                if keep_images:
                    r.image = self._slot_view(buf, k, r.camera).clone()
                out_done.append(r)
        buf.batch = []
        buf.done = None
        return requeue

    def run(self, requests, keep_images: bool = False, realtime: bool = True):
        """Serve the trace. Requests are admitted once their arrival time has passed
        (wall clock since the start, or immediately if realtime=False)."""
        import torch
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: deque = deque()
        done: list = []
        gc_was_enabled = gc.isenabled()
        gc.collect()
        gc.freeze()
        gc.disable()
        try:
            t0 = torch.cuda.Event(enable_timing=True)
            t0.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            wall0 = time.perf_counter()

            def host_ms():
                return 1e3 * (time.perf_counter() - wall0)

            i = 0
            batch_id = 0
            while i < len(pending) or queue or any(b.batch for b in self.buffers):
                now = time.perf_counter() - wall0 if realtime else float("inf")
                while i < len(pending) and pending[i].arrival <= now:
                    queue.append(pending[i])
                    i += 1
                progressed = False
                for b in self.buffers:
                    if b.batch and not b.busy():
                        requeue = self._complete(b, t0, keep_images, done, seen_ms=host_ms())
                        for r in reversed(requeue):
                            queue.appendleft(r)
                        progressed = True
                for b in self.buffers:
                    if not b.batch and queue:
                        reqs = self.scheduler.admit(queue)
                        if reqs:
                            t_admit = host_ms()
                            b.launch(reqs, batch_id)
                            t_launch = host_ms()
                            for r in reqs:
                                r.admit_ms, r.launch_ms = t_admit, t_launch
                            batch_id += 1
                            progressed = True
                if not progressed:
                    # idle until the next arrival, but poll finely while a batch is on
                    # the GPU: its completion is noticed within tens of microseconds
                    in_flight = any(b.batch for b in self.buffers)
                    if realtime and not queue and i < len(pending) and not in_flight:
                        wait = pending[i].arrival - (time.perf_counter() - wall0)
                        if wait > 2e-4:
                            time.sleep(min(wait, 1e-3))
                    else:
                        time.sleep(2e-5)
            torch.cuda.synchronize()
        finally:
            gc.unfreeze()
            if gc_was_enabled:
                gc.enable()
        return done


def _pct(values, p):
    v = sorted(values)
    k = min(len(v) - 1, max(0, int(math.ceil(p / 100.0 * len(v))) - 1))
    return v[k]


def breakdown(r: Request) -> dict | None:
    """Where a request's latency went (ms): waiting in the queue (arrival ->
    admitted), the host's launch (admitted -> launch call returned), waiting
    for and running on the GPU (launch returned -> its batch done), and the loop
    noticing completion (done -> seen). None without timestamps."""
    if None in (r.admit_ms, r.launch_ms, r.done_ms, r.seen_ms):
        return None
    arr = 1e3 * r.arrival
    return {"queue": r.admit_ms - arr, "launch": r.launch_ms - r.admit_ms, "gpu": r.done_ms - r.launch_ms,
            "gpu_run": None if r.gpu_start_ms is None else r.done_ms - r.gpu_start_ms,
            "seen": r.seen_ms - r.done_ms}


def summarize(done, duration_s: float, window: tuple | None = None) -> dict:
    """Latency percentiles and throughput of served requests. duration_s: the
    trace's span the rates are taken over. window (start_s, end_s), if given:
    sustained throughput = requests completed inside the window per second of
    it (the service rate while requests keep arriving; below the arrival rate
    when the server saturates), and drain = time past the window's end until
    the last completion."""
    lat = sorted(r.latency_ms for r in done)
    pix = sum(r.camera.width * r.camera.height for r in done)
    out = {"requests": len(done), "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99), "mean_ms": statistics.mean(lat),
           "max_ms": lat[-1], "req_per_s": len(done) / duration_s, "mpix_per_s": pix / duration_s / 1e6,
           "batches": len({r.batch for r in done})}
    if window is not None:
        a, b = window
        inside = [r for r in done if a * 1e3 <= r.done_ms <= b * 1e3]
        out["completed_per_s"] = len(inside) / max(1e-9, b - a)
        out["completed_mpix_per_s"] = sum(r.camera.width * r.camera.height for r in inside) / max(1e-9, b - a) / 1e6
        out["drain_ms"] = max(0.0, max(r.done_ms for r in done) - b * 1e3)
    parts = [x for x in (breakdown(r) for r in done) if x is not None]
    if parts:
        comp = {}
        for k in ("queue", "launch", "gpu", "gpu_run", "seen"):
            v = [x[k] for x in parts if x[k] is not None]
            if v:
                comp[k] = {"p50": _pct(v, 50), "p99": _pct(v, 99), "max": max(v)}
        out["breakdown_ms"] = comp
        worst = max(done, key=lambda r: r.latency_ms)
        out["slowest"] = {"latency_ms": worst.latency_ms, "arrival_s": worst.arrival, "kind": worst.kind,
                          **(breakdown(worst) or {})}
    return out
