"""Python binding of libdmas.so, the B300 (sm_103a) n-th order DMAS + CF
beamformer.

Argument marshalling only: every step of the beamforming path runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  If the
library has not been built, importing works but every call raises: there is no
fallback path.

    plan = Plan(mic_xyz=..., dir_azel=..., n_samples=4096, fs=450e3, order=5)
    image = plan(frame)          # frame: float32 CUDA tensor [N][T] -> [M][T]
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libdmas.so")
# the host-checked build: every kernel index tested before its access
CHECKED_LIB_PATH = os.path.join(_PKG, "_lib", "libdmas_checked.so")


def _default_lib_path() -> str:
    """libdmas.so, or with DMAS_LIBRARY=checked the host-checked build (any
    other value is taken as a path)."""
    v = os.environ.get("DMAS_LIBRARY", "")
    if v == "checked":
        return CHECKED_LIB_PATH
    return v or LIB_PATH

ROUND, LINEAR = 0, 1
CH_F32, CH_F16, CH_BF16 = 0, 1, 2
NG_CF32, NG_F64, NG_F32 = 0, 1, 2  # compensated FP32 is the default
F_CF, F_ENVELOPE = 1, 2
V_PLAIN, V_CF = 1, 2  # dmas_beamform_orders: images without / with the coherence factor

STATUS = {0: "DMAS_OK", 1: "DMAS_EINVAL", 2: "DMAS_ENOMEM", 3: "DMAS_ECUDA",
          4: "DMAS_EBUSY", 5: "DMAS_ETIMEOUT", 6: "DMAS_EBOUNDS"}

# Every symbol include/dmas.h declares.
EXPORTS = [
    "dmas_plan_create", "dmas_destroy", "dmas_beamform", "dmas_beamform_orders",
    "dmas_beamform_host",
    "dmas_beamform_batch", "dmas_beamform_batch_upload", "dmas_batch_workspace_bytes",
    "dmas_plan_workspace_bytes",
    "dmas_plan_get_info", "dmas_plan_get_delays", "dmas_plan_get_taps", "dmas_plan_check",
    "dmas_plan_last_error", "dmas_plan_set_profiling", "dmas_plan_stage_ms",
    "dmas_selftest_wait_timeout", "dmas_beamform_noalloc", "dmas_status_string",
    "dmas_plan_set_envelope_tile_cap", "dmas_server_create", "dmas_server_submit",
    "dmas_server_wait", "dmas_server_pending", "dmas_server_destroy", "dmas_server_image_free",
    "dmas_version",
]


class DmasError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        msg = f"{what}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("n_mics", ctypes.c_int), ("mic_xyz", ctypes.c_void_p),
        ("n_dirs", ctypes.c_int), ("dir_azel", ctypes.c_void_p),
        ("dir_unit", ctypes.c_void_p), ("delays_s", ctypes.c_void_p),
        ("n_samples", ctypes.c_int), ("fs", ctypes.c_double), ("c", ctypes.c_double),
        ("order", ctypes.c_int), ("delay_mode", ctypes.c_int), ("flags", ctypes.c_int),
        ("cf_eps", ctypes.c_double), ("env_cutoff_hz", ctypes.c_double),
        ("env_taps", ctypes.c_int), ("chan_prec", ctypes.c_int), ("ng_prec", ctypes.c_int),
        ("mf_signal", ctypes.c_void_p), ("mf_len", ctypes.c_int),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int) for name in (
        "n_mics", "n_dirs", "n_samples", "order", "delay_mode", "flags", "chan_prec",
        "ng_prec", "env_taps", "n_groups", "group_size", "window", "mic_chunk", "time_tile",
        "row")] + [
        ("workspace_bytes", ctypes.c_size_t), ("table_bytes", ctypes.c_size_t)]


_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None):
    """Load libdmas.so (raises if it is missing: no CPU fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _default_lib_path()
        if not os.path.exists(p):
            raise RuntimeError(
                f"{p} is missing; build it with `python -m paper_2511_09165_b300.build`")
        lib = ctypes.CDLL(p)
        vp, i, sz, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float
        fp = ctypes.POINTER(f)
        sig = {
            "dmas_plan_create": ([ctypes.POINTER(PlanDesc), ctypes.POINTER(vp)], i),
            "dmas_destroy": ([vp], i),
            "dmas_beamform": ([vp, vp, vp, vp, vp, vp], i),
            "dmas_beamform_host": ([vp, vp, vp, vp], i),
            "dmas_beamform_orders": ([vp, vp, ctypes.c_uint, i, vp, vp, vp], i),
            "dmas_beamform_batch": ([i, vp, vp, vp, vp, sz, vp], i),
            "dmas_beamform_batch_upload": ([i, vp, vp, vp, vp, vp, sz, vp, vp], i),
            "dmas_batch_workspace_bytes": ([i, vp], sz),
            "dmas_plan_workspace_bytes": ([vp], sz),
            "dmas_plan_get_info": ([vp, ctypes.POINTER(PlanInfo)], i),
            "dmas_plan_get_delays": ([vp, vp, vp], i),
            "dmas_plan_get_taps": ([vp, vp], i),
            "dmas_plan_check": ([vp], i),
            "dmas_plan_last_error": ([vp], ctypes.c_char_p),
            "dmas_plan_set_profiling": ([vp, i], i),
            "dmas_plan_set_envelope_tile_cap": ([vp, i], i),
            "dmas_plan_stage_ms": ([vp, fp, fp, fp], i),
            "dmas_selftest_wait_timeout": ([ctypes.c_double, vp], i),
            "dmas_beamform_noalloc": ([vp, vp, vp, vp], i),
            "dmas_status_string": ([i], ctypes.c_char_p),
            "dmas_server_create": ([vp, ctypes.POINTER(vp)], i),
            "dmas_server_submit": ([vp, i, vp, vp, i, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_uint64)], i),
            "dmas_server_image_free": ([vp, vp], i),
            "dmas_server_wait": ([vp, ctypes.c_double, vp], i),
            "dmas_server_pending": ([vp], i),
            "dmas_server_destroy": ([vp], i),
            "dmas_version": ([], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _f64(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _check_tensor(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


@dataclass
class Info:
    n_mics: int
    n_dirs: int
    n_samples: int
    order: int
    delay_mode: int
    flags: int
    chan_prec: int
    ng_prec: int
    env_taps: int
    n_groups: int
    group_size: int
    window: int
    mic_chunk: int
    time_tile: int
    row: int
    workspace_bytes: int
    table_bytes: int


class Plan:
    """A beamforming plan: geometry, delay table, taps and scratch, resident on
    the current CUDA device until close()."""

    def __init__(self, *, n_samples: int, fs: float, order: int = 5,
                 mic_xyz=None, dir_azel=None, dir_unit=None, delays_s=None,
                 c: float = 343.0, delay_mode: int = ROUND, cf: bool = True,
                 envelope: bool = True, cf_eps: float = 1e-30,
                 env_cutoff_hz: float = 5000.0, env_taps: int = 0,
                 chan_prec: int = CH_F32, ng_prec: int = NG_CF32, mf_signal=None):
        xyz, azel, unit, dly = _f64(mic_xyz), _f64(dir_azel), _f64(dir_unit), _f64(delays_s)
        if dly is not None:
            M, N = dly.shape
        else:
            if xyz is None:
                raise ValueError("mic_xyz is required without delays_s")
            N = xyz.reshape(-1, 3).shape[0]
            if unit is not None:
                M = unit.reshape(-1, 3).shape[0]
            elif azel is not None:
                M = azel.reshape(-1, 2).shape[0]
            else:
                raise ValueError("dir_azel or dir_unit is required")
        lib = load_library()
        self._lib = lib
        self._h = ctypes.c_void_p()
        flags = (F_CF if cf else 0) | (F_ENVELOPE if envelope else 0)
        mf = None if mf_signal is None else np.ascontiguousarray(mf_signal, dtype=np.float32)
        d = PlanDesc(int(N), _np_ptr(xyz), int(M), _np_ptr(azel), _np_ptr(unit), _np_ptr(dly),
                     int(n_samples), float(fs), float(c), int(order), int(delay_mode), flags,
                     float(cf_eps), float(env_cutoff_hz), int(env_taps), int(chan_prec),
                     int(ng_prec), _np_ptr(mf), 0 if mf is None else int(mf.size))
        st = lib.dmas_plan_create(ctypes.byref(d), ctypes.byref(self._h))
        if st != 0:
            self._h = None
            raise DmasError(st, "dmas_plan_create")
        self.n_mics, self.n_dirs, self.n_samples = int(N), int(M), int(n_samples)
        self.order = int(order)
        self.envelope = bool(envelope)

    # -- lifecycle ---------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.dmas_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise RuntimeError("plan is closed")
        return self._h

    def _raise(self, st: int, what: str):
        detail = self._lib.dmas_plan_last_error(self.handle).decode()
        raise DmasError(st, what, detail)

    # -- introspection -----------------------------------------------------
    def info(self) -> Info:
        pi = PlanInfo()
        st = self._lib.dmas_plan_get_info(self.handle, ctypes.byref(pi))
        if st != 0:
            self._raise(st, "dmas_plan_get_info")
        return Info(**{f: getattr(pi, f) for f, _ in PlanInfo._fields_})

    def delays(self):
        """(shift[M][N] int32, frac[M][N] float32) in the desc's direction order."""
        shift = np.empty((self.n_dirs, self.n_mics), dtype=np.int32)
        frac = np.empty((self.n_dirs, self.n_mics), dtype=np.float32)
        st = self._lib.dmas_plan_get_delays(self.handle, _np_ptr(shift), _np_ptr(frac))
        if st != 0:
            self._raise(st, "dmas_plan_get_delays")
        return shift, frac

    def taps(self) -> np.ndarray:
        L = self.info().env_taps
        h = np.empty(L, dtype=np.float32)
        if L:
            st = self._lib.dmas_plan_get_taps(self.handle, _np_ptr(h))
            if st != 0:
                self._raise(st, "dmas_plan_get_taps")
        return h

    def workspace_bytes(self) -> int:
        return int(self._lib.dmas_plan_workspace_bytes(self.handle))

    def check(self) -> None:
        """Synchronise and raise if a kernel's bounded wait expired."""
        st = self._lib.dmas_plan_check(self.handle)
        if st != 0:
            self._raise(st, "dmas_plan_check")

    def set_profiling(self, enable: bool = True) -> None:
        st = self._lib.dmas_plan_set_profiling(self.handle, int(bool(enable)))
        if st != 0:
            self._raise(st, "dmas_plan_set_profiling")

    def set_envelope_tile_cap(self, tiles_per_cta: int) -> None:
        """At most this many tensor-core envelope tiles per CTA (0: one CTA per
        SM over all tiles), so higher-priority streams reach the SMs sooner."""
        st = self._lib.dmas_plan_set_envelope_tile_cap(self.handle, int(tiles_per_cta))
        if st != 0:
            self._raise(st, "dmas_plan_set_envelope_tile_cap")

    def stage_ms(self):
        """(roots, beamform, envelope) milliseconds of the last profiled call."""
        a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        st = self._lib.dmas_plan_stage_ms(self.handle, ctypes.byref(a), ctypes.byref(b),
                                          ctypes.byref(c))
        if st != 0:
            self._raise(st, "dmas_plan_stage_ms")
        return a.value, b.value, c.value

    # -- compute -----------------------------------------------------------
    def __call__(self, frame, out=None, y=None, cf=None, stream=None):
        """Beamform one frame [N][T] (float32 CUDA) -> image [M][T]."""
        import torch
        _check_tensor(frame, (self.n_mics, self.n_samples), "frame")
        if out is None:
            out = torch.empty((self.n_dirs, self.n_samples), device=frame.device,
                              dtype=torch.float32)
        _check_tensor(out, (self.n_dirs, self.n_samples), "out")
        for t, name in ((y, "y"), (cf, "cf")):
            if t is not None:
                _check_tensor(t, (self.n_dirs, self.n_samples), name)
        st = self._lib.dmas_beamform(
            self.handle, ctypes.c_void_p(frame.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(y.data_ptr()) if y is not None else None,
            ctypes.c_void_p(cf.data_ptr()) if cf is not None else None,
            ctypes.c_void_p(_stream_handle(stream)))
        if st != 0:
            self._raise(st, "dmas_beamform")
        return out

    def beamform_orders(self, frame, orders=None, variants=V_PLAIN | V_CF, out=None, cf=None,
                        stream=None):
        """Every order at once: images [V][K][M][T] of the orders `orders`
        (default 1..order, ascending) for the variants V_PLAIN (E_k) and/or
        V_CF (E_k x CF), plain first, from one pass over the delayed samples."""
        import torch
        _check_tensor(frame, (self.n_mics, self.n_samples), "frame")
        orders = sorted(set(range(1, self.order + 1) if orders is None else orders))
        mask = 0
        for k in orders:
            if not 1 <= k <= 8:
                raise ValueError(f"order {k} out of range")
            mask |= 1 << (k - 1)
        n_v = bin(int(variants) & 3).count("1")
        shape = (n_v, len(orders), self.n_dirs, self.n_samples)
        if out is None:
            out = torch.empty(shape, device=frame.device, dtype=torch.float32)
        _check_tensor(out, shape, "out")
        if cf is not None:
            _check_tensor(cf, (self.n_dirs, self.n_samples), "cf")
        st = self._lib.dmas_beamform_orders(
            self.handle, ctypes.c_void_p(frame.data_ptr()), mask, int(variants),
            ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(cf.data_ptr()) if cf is not None else None,
            ctypes.c_void_p(_stream_handle(stream)))
        if st != 0:
            self._raise(st, "dmas_beamform_orders")
        return out

    def beamform_host(self, frame: np.ndarray, out: np.ndarray | None = None, stream=None):
        """Host buffers in and out (copies inside the call; synchronises)."""
        frame = np.ascontiguousarray(frame, dtype=np.float32)
        if frame.shape != (self.n_mics, self.n_samples):
            raise ValueError("frame shape mismatch")
        if out is None:
            out = np.empty((self.n_dirs, self.n_samples), dtype=np.float32)
        if out.shape != (self.n_dirs, self.n_samples) or out.dtype != np.float32 \
                or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float32 [M][T] array")
        self.beamform_host_ptr(frame.ctypes.data, out.ctypes.data, stream)
        return out

    def beamform_host_ptr(self, frame_ptr: int, out_ptr: int, stream=None) -> None:
        """Host-buffer call on raw pointers (e.g. pinned torch tensors)."""
        st = self._lib.dmas_beamform_host(self.handle, ctypes.c_void_p(frame_ptr),
                                          ctypes.c_void_p(out_ptr),
                                          ctypes.c_void_p(_stream_handle(stream)))
        if st != 0:
            self._raise(st, "dmas_beamform_host")


def batch_workspace_bytes(plans) -> int:
    lib = load_library()
    arr = (ctypes.c_void_p * len(plans))(*[p.handle.value for p in plans])
    return int(lib.dmas_batch_workspace_bytes(len(plans), arr))


def beamform_batch(plans, frames, images=None, workspace=None, stream=None):
    """Beamform frames[k] with plans[k]; returns the list of images."""
    import torch
    lib = load_library()
    n = len(plans)
    if n != len(frames):
        raise ValueError("plans and frames differ in length")
    if images is None:
        images = [torch.empty((p.n_dirs, p.n_samples), device=f.device, dtype=torch.float32)
                  for p, f in zip(plans, frames)]
    for p, f, im in zip(plans, frames, images):
        _check_tensor(f, (p.n_mics, p.n_samples), "frame")
        _check_tensor(im, (p.n_dirs, p.n_samples), "image")
    need = batch_workspace_bytes(plans)
    if workspace is None:
        workspace = torch.empty(need, device=frames[0].device, dtype=torch.uint8)
    ph = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in frames])
    ip = (ctypes.c_void_p * n)(*[im.data_ptr() for im in images])
    st = lib.dmas_beamform_batch(n, ph, fp, ip, ctypes.c_void_p(workspace.data_ptr()),
                                 workspace.numel() * workspace.element_size(),
                                 ctypes.c_void_p(_stream_handle(stream)))
    if st != 0:
        raise DmasError(st, "dmas_beamform_batch")
    return images


def beamform_batch_upload(plans, host_frames, frames, images, workspace, stream=None,
                          done_event=None):
    """beamform_batch for frames in (page-locked) host memory, in one call into
    the library: host_frames[k] is copied into the device tensor frames[k] on
    the stream, the batch runs, and `done_event` (a recorded-once
    torch.cuda.Event, or None) is recorded after it."""
    lib = load_library()
    n = len(plans)
    if not (n == len(host_frames) == len(frames) == len(images)):
        raise ValueError("plans, host frames, frames and images differ in length")
    import torch
    for p, h, f, im in zip(plans, host_frames, frames, images):
        if h.device.type != "cpu" or not h.is_contiguous() or h.dtype != torch.float32 \
                or tuple(h.shape) != (p.n_mics, p.n_samples):
            raise ValueError(f"host frame must be a contiguous CPU float32 {(p.n_mics, p.n_samples)}")
        _check_tensor(f, (p.n_mics, p.n_samples), "frame")
        _check_tensor(im, (p.n_dirs, p.n_samples), "image")
    ph = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    hp = (ctypes.c_void_p * n)(*[h.data_ptr() for h in host_frames])
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in frames])
    ip = (ctypes.c_void_p * n)(*[im.data_ptr() for im in images])
    ev = ctypes.c_void_p(done_event.cuda_event if done_event is not None else 0)
    st = lib.dmas_beamform_batch_upload(n, ph, hp, fp, ip, ctypes.c_void_p(workspace.data_ptr()),
                                        workspace.numel() * workspace.element_size(),
                                        ctypes.c_void_p(_stream_handle(stream)), ev)
    if st != 0:
        raise DmasError(st, "dmas_beamform_batch_upload")
    return images


def selftest_wait_timeout(limit_ms: float = 50.0, stream=None) -> int:
    """Run the bounded-wait self-test; returns the status (5 = timed out as designed)."""
    lib = load_library()
    return int(lib.dmas_selftest_wait_timeout(float(limit_ms),
                                              ctypes.c_void_p(_stream_handle(stream))))
