"""Continuous-batching server for sonar frames from several sensors.

Each sensor has a resident plan (delay tables and taps on the device).  Frames
arrive on the host at any time and are handed to the library's serving
runtime (dmas_server_* in the C ABI), whose native thread

  * admits a frame when the device-memory budget has room for its frame,
    image and scratch (otherwise it waits in its lane's FIFO queue; a frame
    that can never fit is rejected),
  * sorts frames into two lanes by their cost N * M * T: small frames go to a
    fast lane whose streams have high priority (the GPU schedules their CTAs
    ahead of waiting CTAs of big frames) and are batched generously (every
    waiting small frame, up to `max_batch`, in one batch: one launch per
    kernel stage and variant); big frames go one per batch to one
    low-priority stream with `bulk_depth` batches queued on it, so they run
    first in, first out while the small frames overtake them,
  * uploads a batch's frames, runs it and records its completion event in one
    library call, and notices completions by polling the events while
    batches are in flight,
  * records, per frame, the time from its arrival to the completion of its
    batch on the device (the image is then resident in device memory; with
    `copy_back` the image is also copied to host memory first).

Python only submits frames and collects completions: no interpreter lock sits
between a frame's arrival and its launch.  Results do not depend on the batch
a frame lands in: each entry uses its own scratch, so its image is bitwise
identical to a `dmas_beamform` of that frame alone.
"""
from __future__ import annotations

import collections
import ctypes
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import DmasError, load_library


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
# Tensor-core envelope tiles per CTA for the bulk lane's plans; 0: no cap
# (one persistent CTA per SM).  Measured on B300, 16-sensor mix at 200
# frames/s over four arrival seeds: without a cap the overall p99 is 0.04-0.4
# ms lower than with 16 tiles per CTA and the small frames' p99 is the same
# (1.1 ms): a capped envelope costs a big frame 0.03-0.06 ms of relaunched
# CTAs, more than the small frames gain from the earlier SM slots.
BULK_ENV_TILE_CAP = 0


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
    status: int = 0               # the library's status for this frame (0: done)
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class _ServerDesc(ctypes.Structure):
    _fields_ = [("n_plans", ctypes.c_int), ("plans", ctypes.c_void_p),
                ("fast_cost", ctypes.c_double), ("fast_streams", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("bulk_depth", ctypes.c_int),
                ("budget_bytes", ctypes.c_size_t)]


class _ServerDone(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("sensor", ctypes.c_int), ("status", ctypes.c_int),
                ("batch_size", ctypes.c_int), ("t_arrival", ctypes.c_double),
                ("t_admitted", ctypes.c_double), ("t_done", ctypes.c_double),
                ("d_image", ctypes.c_void_p)]


class _DeviceImage:
    """A device image the runtime handed over, exposed to torch through the
    CUDA array interface; freed (ordered on the legacy default stream) when
    the last tensor over it and this holder are gone."""

    def __init__(self, lib, ptr: int, shape):
        self._lib, self._ptr = lib, ptr
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4",
                                         "data": (ptr, False), "version": 2, "strides": None}

    def __del__(self):
        if self._ptr:
            self._lib.dmas_server_image_free(ctypes.c_void_p(self._ptr), None)
            self._ptr = 0


_ETIMEOUT, _ENOMEM = 5, 2


class Server:
    """Serving through the library's native runtime (dmas_server_*).

    fast_cost: frames with cost <= fast_cost use the fast lane (default:
    about 0.5 ms of GPU work, 1.3e9 mic x direction x samples), `streams`
    high-priority streams with one batch of up to `max_batch` frames in
    flight on each; big frames take the bulk lane, one frame per batch on one
    low-priority stream with up to `bulk_depth` batches queued on it.
    Defaults measured on B300 with the 16-sensor mix at 200 frames/s: big
    frames first in, first out, two in flight (three concurrent big-frame
    streams stretched each big frame by the others' work: overall p99 +2 ms).
    The runtime allocates each frame's image when it admits the frame; with
    keep_image the completed request's `image` is that device tensor (freed
    when the last reference goes), with `copy_back` a page-locked host buffer
    from `pinned` that the image was copied into before the frame
    completed."""

    def __init__(self, sensors, device=None, budget_bytes: int = 32 << 30,
                 max_batch: int = 64, streams: int = 2, copy_back: bool = False,
                 fast_cost: float = FAST_COST, bulk_depth: int = 2,
                 bulk_env_tile_cap: int = BULK_ENV_TILE_CAP, pinned: PinnedPool | None = None):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.sensors = list(sensors)
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.streams = int(streams)
        self.bulk_depth = int(bulk_depth)
        self.copy_back = bool(copy_back)
        self.fast_cost = float(fast_cost)
        self.pinned = pinned if pinned is not None else (PinnedPool() if copy_back else None)
        if copy_back:
            # page-locking takes milliseconds per gigabyte: hold enough host
            # images now for the frames that can be queued or in flight at
            # once (a small frame's few, the bulk lane's depth plus the ones
            # waiting for it), counted per sensor and pooled per shape
            want = collections.Counter()
            for sn in self.sensors:
                small = sn.cost <= self.fast_cost
                want[tuple(sn.image_shape)] += 4 if small else self.bulk_depth + 2
            for shape, n in want.items():
                self.pinned.reserve(shape, n)
        # with a cap, big frames' envelopes retire their CTAs every few tiles,
        # so the fast lane's kernels reach the SMs without waiting for a whole
        # envelope
        for sn in self.sensors:
            if sn.cost > self.fast_cost and hasattr(sn.plan, "set_envelope_tile_cap"):
                sn.plan.set_envelope_tile_cap(bulk_env_tile_cap)
        self._handle = ctypes.c_void_p()
        self._cv = threading.Condition()
        self._reqs: dict = {}          # ticket -> Request, until its completion is taken
        self._running = False
        self._waiter = None
        self._batches = 0.0
        self.completed: list[Request] = []

    @property
    def batches(self) -> int:
        """Batches completed (each frame counts 1 / its batch's size)."""
        return int(round(self._batches))

    # -- lifecycle -------------------------------------------------------
    def start(self):
        torch = self.torch
        plans = (ctypes.c_void_p * len(self.sensors))(*[sn.plan.handle.value for sn in self.sensors])
        desc = _ServerDesc(len(self.sensors), ctypes.cast(plans, ctypes.c_void_p), self.fast_cost,
                           self.streams, self.max_batch, self.bulk_depth, self.budget)
        with torch.cuda.device(self.device):
            st = self.lib.dmas_server_create(ctypes.byref(desc), ctypes.byref(self._handle))
        if st != 0:
            raise DmasError(st, "dmas_server_create")
        self._running = True
        self._waiter = threading.Thread(target=self._wait_loop, daemon=True)
        self._waiter.start()
        return self

    def stop(self):
        """Finish the frames submitted so far, then shut the runtime down."""
        if not self._handle:
            return
        self.drain(600.0)
        with self._cv:
            self._running = False
        self._waiter.join(timeout=60)
        self.lib.dmas_server_destroy(self._handle)
        self._handle = ctypes.c_void_p()

    def __enter__(self):
        return self.start()

    def __exit__(self, *exc):
        self.stop()

    def submit(self, sensor: int, frame, t_arrival: float | None = None,
               keep_image: bool = False) -> Request:
        """frame: host tensor [N][T] float32 (page-locked for an asynchronous
        upload), kept unchanged until the request completes."""
        torch = self.torch
        sn = self.sensors[sensor]
        if frame.device.type != "cpu" or not frame.is_contiguous() or \
                frame.dtype != torch.float32 or tuple(frame.shape) != tuple(sn.frame_shape):
            raise ValueError(f"frame must be a contiguous host float32 {tuple(sn.frame_shape)}")
        req = Request(sensor, frame, time.perf_counter() if t_arrival is None else t_arrival,
                      keep_image)
        req._host = self.pinned.get(sn.image_shape) if self.copy_back else None
        keep_device = keep_image and not self.copy_back
        ticket = ctypes.c_uint64()
        with self._cv:
            st = self.lib.dmas_server_submit(
                self._handle, int(sensor), ctypes.c_void_p(frame.data_ptr()),
                ctypes.c_void_p(req._host.data_ptr() if req._host is not None else 0),
                int(keep_device), float(req.t_arrival), ctypes.byref(ticket))
            if st != 0:
                raise DmasError(st, "dmas_server_submit")
            self._reqs[ticket.value] = req
        return req

    def drain(self, timeout: float = 600.0) -> bool:
        """Wait until every submitted frame has completed."""
        end = time.perf_counter() + timeout
        with self._cv:
            while self._reqs:
                left = end - time.perf_counter()
                if left <= 0:
                    return False
                self._cv.wait(timeout=min(left, 0.1))
        return True

    # -- completions ------------------------------------------------------
    def _wait_loop(self):
        """Take the runtime's completions (blocking in the library, outside the
        interpreter lock) and fill in the requests."""
        done = _ServerDone()
        while True:
            st = self.lib.dmas_server_wait(self._handle, 0.05, ctypes.byref(done))
            if st == _ETIMEOUT:
                with self._cv:
                    if not self._running and not self._reqs:
                        return
                continue
            with self._cv:
                req = self._reqs.get(done.ticket)
            if req is None:
                continue
            req.t_admitted = done.t_admitted
            req.t_done = done.t_done
            req.batch_size = done.batch_size
            req.rejected = done.status == _ENOMEM
            req.status = done.status
            if done.d_image:
                req._holder = _DeviceImage(self.lib, done.d_image, self.sensors[req.sensor].image_shape)
                req.image = self.torch.as_tensor(req._holder, device=self.device)
            elif req.keep_image and req._host is not None and done.status == 0:
                req.image = req._host
            elif req._host is not None:
                self.pinned.put(req._host)
            req._host = None
            with self._cv:
                del self._reqs[done.ticket]
                self._batches += 1.0 / max(1, done.batch_size)
                self.completed.append(req)
                req.done.set()
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
