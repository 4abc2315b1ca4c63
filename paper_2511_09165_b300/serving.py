"""Continuous-batching server for sonar frames from several sensors.

Each sensor has a resident plan (delay tables and taps on the device).  Frames
arrive on the host at any time; the server

  * admits a frame when the device-memory budget has room for its frame,
    image and scratch (otherwise it waits in the FIFO queue; a frame that can
    never fit is rejected),
  * gathers every admitted frame that is waiting into one batch (up to
    `max_batch`) and runs it with one `dmas_beamform_batch` call: one launch
    per kernel stage and variant for the whole batch,
  * keeps up to `streams` batches in flight on separate CUDA streams, so
    frames that arrive while earlier batches run are batched and overlap with
    them on the GPU,
  * sorts frames into two lanes by their cost N * M * T: small frames go to a
    fast lane whose streams have high priority (the GPU schedules their CTAs
    ahead of waiting CTAs of big frames) and are batched generously; big frames
    go to a bulk lane in small batches, since batching them saves no launch
    overhead worth having and a batch completes only when its last frame does,
  * records, per frame, the time from its arrival to the completion of its
    batch on the device (the image is then resident in device memory; with
    `copy_back` the image is also copied to host memory first).

The host threads only move pointers and events; every step of the
beamforming path runs in the library's kernels.  Results do not depend on the
batch a frame lands in: each entry uses its own scratch, so its image is
bitwise identical to a `dmas_beamform` of that frame alone.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import beamform_batch_upload, batch_workspace_bytes


@dataclass
class Sensor:
    """A sensor: its plan and the device bytes one of its frames occupies."""
    plan: object
    name: str = ""

    @property
    def frame_shape(self):
        return (self.plan.n_mics, self.plan.n_samples)

    @property
    def image_shape(self):
        return (self.plan.n_dirs, self.plan.n_samples)

    @property
    def device_bytes(self) -> int:
        n, t = self.frame_shape
        m, _ = self.image_shape
        return 4 * (n * t + m * t) + self.plan.workspace_bytes()

    @property
    def cost(self) -> int:
        """Work of one frame: microphones x directions x samples."""
        return self.plan.n_mics * self.plan.n_dirs * self.plan.n_samples


# Frames of at most this cost (microphones x directions x samples) take the
# fast lane.
FAST_COST = 1.3e9
# Tensor-core envelope tiles per CTA for the bulk lane's plans
BULK_ENV_TILE_CAP = 16


# Device-to-host copies of big images go out in pieces of this many bytes, so
# the copy engine can interleave the small frames' copies (issued on other
# streams) between them instead of queueing them behind a whole gigabyte.
COPY_PIECE_BYTES = 32 << 20


def _copy_in_pieces(dst, src) -> None:
    """dst.copy_(src) (non-blocking) in COPY_PIECE_BYTES pieces."""
    d, s = dst.view(-1), src.view(-1)
    step = max(1, COPY_PIECE_BYTES // 4)
    for a in range(0, s.numel(), step):
        d[a:a + step].copy_(s[a:a + step], non_blocking=True)


class PinnedPool:
    """Page-locked host buffers reused by shape: allocating pinned memory
    takes milliseconds per gigabyte, so copies back to the host draw on this
    pool instead of allocating per frame.  When every buffer of a shape is in
    use, get() allocates another at once if it is smaller than `wait_bytes`,
    and otherwise waits (up to `wait_s`) for one to come back first (a caller
    that waits holds up whatever it dispatches, so only the buffers that are
    slow to allocate are worth waiting for)."""

    def __init__(self, wait_s: float = 2.0, wait_bytes: int = 64 << 20):
        import torch
        self.torch = torch
        self.wait_s = float(wait_s)
        self.wait_bytes = int(wait_bytes)
        self._free: dict = collections.defaultdict(list)
        self._owned: dict = collections.defaultdict(int)
        self._cv = threading.Condition()

    def _alloc(self, shape):
        t = self.torch.empty(shape, dtype=self.torch.float32, pin_memory=True)
        with self._cv:
            self._owned[shape] += 1
        return t

    def get(self, shape):
        shape = tuple(shape)
        big = 4 * int(np.prod(shape)) >= self.wait_bytes
        with self._cv:
            if not self._free[shape] and self._owned[shape] > 0 and big:
                self._cv.wait_for(lambda: bool(self._free[shape]), timeout=self.wait_s)
            if self._free[shape]:
                return self._free[shape].pop()
        return self._alloc(shape)

    def put(self, t) -> None:
        with self._cv:
            self._free[tuple(t.shape)].append(t)
            self._cv.notify_all()

    def reserve(self, shape, count: int) -> None:
        """Hold at least `count` buffers of this shape (allocated now)."""
        shape = tuple(shape)
        with self._cv:
            have = self._owned[shape]
        for _ in range(max(0, count - have)):
            self.put(self._alloc(shape))


class _Lane:
    def __init__(self, name, streams, max_batch, depth=None):
        self.name = name
        self.streams = streams
        self.max_batch = max_batch
        # batches in flight at once (several may queue on one stream)
        self.depth = len(streams) if depth is None else max(1, int(depth))
        self.queue = collections.deque()
        self.in_flight = 0
        self.next_stream = 0


@dataclass
class Request:
    sensor: int
    frame: object                 # host tensor [N][T] float32 (pinned for overlap)
    t_arrival: float              # time.perf_counter() seconds
    keep_image: bool = False
    t_admitted: float = 0.0
    t_done: float = 0.0
    batch_size: int = 0
    image: object = None          # device tensor when keep_image, host tensor with copy_back
    rejected: bool = False
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class Server:
    """fast_cost: frames with cost <= fast_cost use the fast lane (default:
    about 0.5 ms of GPU work, 1.3e9 mic x direction x samples).  `streams`
    is the fast lane's stream count, `bulk_streams` the bulk lane's (None:
    the same), `bulk_depth` the big-frame batches in flight at once (None:
    one per bulk stream; more queue on a stream, so the next big frame is
    enqueued while the previous one runs); `bulk_batch` frames per bulk
    batch.  Defaults measured on B300 with the 16-sensor mix at 200 frames/s:
    one big frame per batch on one low-priority stream, two in flight, keeps
    big frames first-in first-out as one stream does (three concurrent
    streams stretched each big frame by the others' work: overall p99 +2 ms)
    while the small frames overtake them on high-priority streams."""

    # the server thread's sleep between scans of the batches in flight
    poll_s = 50e-6

    def __init__(self, sensors, device=None, budget_bytes: int = 32 << 30,
                 max_batch: int = 64, streams: int = 2, copy_back: bool = False,
                 fast_cost: float = FAST_COST, bulk_batch: int = 1,
                 bulk_streams: int | None = 1, bulk_env_tile_cap: int = BULK_ENV_TILE_CAP,
                 pinned: PinnedPool | None = None, bulk_depth: int | None = 2):
        import torch
        self.torch = torch
        self.sensors = list(sensors)
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.budget = int(budget_bytes)
        self.copy_back = bool(copy_back)
        self.fast_cost = float(fast_cost)
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream,
                                                              "priority_range") else (0, -1)
        n_fast = max(1, streams)
        n_bulk = max(1, streams if bulk_streams is None else bulk_streams)
        self.fast = _Lane("fast", [torch.cuda.Stream(device=self.device, priority=hi)
                                   for _ in range(n_fast)], int(max_batch))
        self.bulk = _Lane("bulk", [torch.cuda.Stream(device=self.device, priority=lo)
                                   for _ in range(n_bulk)], max(1, int(bulk_batch)), bulk_depth)
        self._cv = threading.Condition()
        self._reserved = 0
        self._inflight_q: collections.deque = collections.deque()
        self._events: list = []      # completion events free for reuse
        self._ws_bytes: dict = {}    # batch workspace bytes by sensor tuple
        self._running = False
        self._threads = []
        self.batches = 0
        self.completed: list[Request] = []
        self.pinned = pinned if pinned is not None else (PinnedPool() if copy_back else None)
        if copy_back:
            # page-locking takes milliseconds per gigabyte: hold enough host
            # images now for the frames that can be in flight at once (the
            # bulk lane's depth of big frames, small ones in the fast lane's
            # batches), counted per sensor and pooled per shape
            want = collections.Counter()
            for sn in self.sensors:
                small = sn.cost <= self.fast_cost
                want[tuple(sn.image_shape)] += 4 if small else self.bulk.depth + 1
            for shape, n in want.items():
                self.pinned.reserve(shape, n)
        # big frames' envelopes retire their CTAs every few tiles, so the fast
        # lane's kernels reach the SMs without waiting for a whole envelope
        for sn in self.sensors:
            if sn.cost > self.fast_cost and hasattr(sn.plan, "set_envelope_tile_cap"):
                sn.plan.set_envelope_tile_cap(bulk_env_tile_cap)

    def _lane_of(self, sensor: int) -> _Lane:
        return self.fast if self.sensors[sensor].cost <= self.fast_cost else self.bulk

    # -- lifecycle -------------------------------------------------------
    def start(self):
        self._running = True
        self._threads = [threading.Thread(target=self._loop, daemon=True)]
        for t in self._threads:
            t.start()
        return self

    def stop(self):
        with self._cv:
            self._running = False
            self._cv.notify_all()
        for t in self._threads:
            t.join(timeout=60)

    def __enter__(self):
        return self.start()

    def __exit__(self, *exc):
        self.stop()

    def submit(self, sensor: int, frame, t_arrival: float | None = None,
               keep_image: bool = False) -> Request:
        req = Request(sensor, frame, time.perf_counter() if t_arrival is None else t_arrival,
                      keep_image)
        with self._cv:
            self._lane_of(sensor).queue.append(req)
            self._cv.notify_all()
        return req

    def drain(self, timeout: float = 600.0) -> bool:
        end = time.perf_counter() + timeout
        with self._cv:
            while (self.fast.queue or self.bulk.queue or self.fast.in_flight
                   or self.bulk.in_flight):
                left = end - time.perf_counter()
                if left <= 0:
                    return False
                self._cv.wait(timeout=min(left, 0.1))
        return True

    # -- the server's thread: completion, admission and batching ------------
    def _loop(self):
        """One thread completes finished batches, admits queued frames and
        launches batches: with no second thread to hand the interpreter lock
        to, a launch is not kept waiting behind a completion poll."""
        while True:
            self._reap()
            with self._cv:
                lane = next((ln for ln in (self.fast, self.bulk) if self._can_launch(ln)), None)
                if lane is None:
                    if not self._inflight_q and not self._running:
                        return                      # stopped, nothing in flight
                    # poll the batches in flight; otherwise sleep until a submit
                    self._cv.wait(timeout=self.poll_s if self._inflight_q else 0.05)
                    continue
                batch = []
                while lane.queue and len(batch) < lane.max_batch:
                    req = lane.queue[0]
                    need = self.sensors[req.sensor].device_bytes
                    if need > self.budget:          # can never fit: reject
                        lane.queue.popleft()
                        req.rejected = True
                        req.t_done = time.perf_counter()
                        req.done.set()
                        continue
                    if self._reserved + need > self.budget:
                        break
                    lane.queue.popleft()
                    self._reserved += need
                    batch.append(req)
                if not batch:
                    continue
                lane.in_flight += 1
                stream = lane.streams[lane.next_stream]
                lane.next_stream = (lane.next_stream + 1) % len(lane.streams)
            now = time.perf_counter()
            for r in batch:
                r.t_admitted = now
            self._launch(batch, stream, lane)

    def _can_launch(self, lane) -> bool:
        if not lane.queue or lane.in_flight >= lane.depth:
            return False
        head = self.sensors[lane.queue[0].sensor].device_bytes
        return head > self.budget or self._reserved + head <= self.budget

    def _event(self, stream):
        """A completion event from the free list (created by one record)."""
        if self._events:
            return self._events.pop()
        ev = self.torch.cuda.Event()
        ev.record(stream)
        return ev

    def _launch(self, batch, stream, lane):
        torch = self.torch
        with torch.cuda.stream(stream):
            plans = [self.sensors[r.sensor].plan for r in batch]
            key = tuple(r.sensor for r in batch)
            ws_bytes = self._ws_bytes.get(key)
            if ws_bytes is None:
                ws_bytes = self._ws_bytes[key] = batch_workspace_bytes(plans)
            frames = [torch.empty((p.n_mics, p.n_samples), device=self.device) for p in plans]
            images = [torch.empty((p.n_dirs, p.n_samples), device=self.device) for p in plans]
            ws = torch.empty(ws_bytes, device=self.device, dtype=torch.uint8)
            hosts = None
            if self.copy_back:
                ev = torch.cuda.Event()
                beamform_batch_upload(plans, [r.frame for r in batch], frames, images, ws,
                                      stream=stream)
                hosts = [self.pinned.get(im.shape) for im in images]
                for h, im in zip(hosts, images):
                    _copy_in_pieces(h, im)
                ev.record(stream)
            else:
                # uploads, the batch and its completion event in one library call
                ev = self._event(stream)
                beamform_batch_upload(plans, [r.frame for r in batch], frames, images, ws,
                                      stream=stream, done_event=ev)
        self.batches += 1
        with self._cv:
            self._inflight_q.append((ev, batch, frames, images, ws, hosts, lane))
            self._cv.notify_all()

    # -- completion: latency and memory release ----------------------------
    def _reap(self):
        """Every batch whose completion event has fired (fast lanes finish out
        of order with the bulk lane): record its requests' latency, hand back
        host buffers and release its share of the memory budget."""
        with self._cv:
            done = [x for x in self._inflight_q if x[0].query()]
            for item in done:
                self._inflight_q.remove(item)
        if not done:
            return
        t = time.perf_counter()
        for ev, batch, frames, images, ws, hosts, lane in done:
            for k, r in enumerate(batch):
                r.t_done = t
                r.batch_size = len(batch)
                if r.keep_image:
                    r.image = hosts[k] if hosts is not None else images[k]
                elif hosts is not None:
                    self.pinned.put(hosts[k])
        with self._cv:
            for ev, batch, frames, images, ws, hosts, lane in done:
                for r in batch:
                    self._reserved -= self.sensors[r.sensor].device_bytes
                    self.completed.append(r)
                    r.done.set()
                lane.in_flight -= 1
                if hosts is None:
                    self._events.append(ev)
            self._cv.notify_all()


def one_frame_per_launch(sensors, requests, device=None, copy_back: bool = False,
                         pinned: PinnedPool | None = None):
    """Baseline: every frame alone through dmas_beamform, in arrival order, on
    one stream.  Blocks until each frame's arrival time; returns the requests
    with t_done filled (the image resident on the device, or with copy_back
    copied to pinned host memory: one buffer per sensor from `pinned`, reused
    frame after frame since the one stream orders the copies, unless the
    request keeps its image)."""
    import torch
    dev = torch.device("cuda") if device is None else torch.device(device)
    stream = torch.cuda.Stream(device=dev)
    pending = collections.deque()
    if copy_back and pinned is None:
        pinned = PinnedPool()
    per_sensor = {}

    def finish(ev, q, h):
        q.t_done = time.perf_counter()

    with torch.cuda.stream(stream):
        for r in requests:
            while time.perf_counter() < r.t_arrival:
                while pending and pending[0][0].query():
                    finish(*pending.popleft())
                time.sleep(0.0002)
            p = sensors[r.sensor].plan
            f = torch.empty((p.n_mics, p.n_samples), device=dev)
            f.copy_(r.frame, non_blocking=True)
            img = p(f, stream=stream)
            h = None
            if copy_back:
                if r.keep_image:
                    h = pinned.get(img.shape)
                else:
                    h = per_sensor.get(r.sensor)
                    if h is None:
                        h = per_sensor[r.sensor] = pinned.get(img.shape)
                h.copy_(img, non_blocking=True)
                img = h
            ev = torch.cuda.Event()
            ev.record(stream)
            pending.append((ev, r, h))
            r.batch_size = 1
            if r.keep_image:
                r.image = img
    while pending:
        ev, q, h = pending.popleft()
        ev.synchronize()
        finish(ev, q, h)
    for h in per_sensor.values():
        pinned.put(h)
    return requests


def poisson_arrivals(rate_hz: float, duration_s: float, n_sensors: int, seed: int):
    """Scheduled arrival offsets (s) and sensor indices of a Poisson stream."""
    rng = np.random.default_rng(seed)
    t, times, which = 0.0, [], []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        times.append(t)
        which.append(int(rng.integers(n_sensors)))
    return np.array(times), np.array(which, dtype=np.int64)


def latency_summary(reqs, t_from: float = -np.inf) -> dict:
    """p50/p99/mean latency (ms) of requests that arrived at or after t_from."""
    lat = np.array([r.latency for r in reqs if not r.rejected and r.t_arrival >= t_from])
    if lat.size == 0:
        return {"frames": 0}
    return {"frames": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "max_ms": float(lat.max() * 1e3)}
