"""FP64 CPU oracle for n-th order DMAS + Coherence Factor beamforming.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import this package.  The CUDA library
never imports it, and it imports nothing from the CUDA library.

The arithmetic lives in ``dmas_oracle.c`` (plain C, double precision, compiled
with ``-ffp-contract=off`` and without fast-math).  This module compiles it
with gcc on first use and wraps it with numpy arrays.  Section and equation
names below refer to the DMAS paper (Jansen, Daems, Steckel, "Delay-Multiply-
And-Sum Beamforming for Real-Time In-Air Acoustic Imaging").

Parity status of each function (what pins it is in tests/test_oracle_pins.py):
  unit_vectors, geometric_delays, round_shifts  pinned (closed forms, plane wave)
  esym_product                                  pinned (brute-force subsets, Eq. dmasn)
  esym_newton_girard                            pinned (explicit Eqs. dmas2..5 from
                                                the paper, brute force, product form)
  signed_root                                   pinned (closed forms)
  fir_taps / envelope                           pinned to its own design (DC gain,
                                                impulse, cutoff); the paper does not
                                                give its filter, so agreement with
                                                the authors' envelope is unpinned
  dmas                                          pinned (n = 1 DAS, n = 2 Eq. dmas,
                                                brute force, closed forms, invariants)
  matched_filter                                pinned (impulse response = the emitted
                                                signal reversed, numpy.correlate,
                                                linearity, frame end); the authors'
                                                emitted signal and alignment are not
                                                given, so agreement with their
                                                matched filter is unpinned
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmas_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "libdmas_oracle.so")
_lock = threading.Lock()
_lib = None

ROUND = 0
LINEAR = 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc; returns its path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.oracle_set_threads.argtypes = [i]
        lib.oracle_set_threads.restype = i
        lib.oracle_unit_vectors.argtypes = [i, p, p]
        lib.oracle_unit_vectors.restype = None
        lib.oracle_geometric_delays.argtypes = [i, p, i, p, d, p]
        lib.oracle_geometric_delays.restype = None
        lib.oracle_round_shift.argtypes = [d, d]
        lib.oracle_round_shift.restype = ctypes.c_longlong
        lib.oracle_esym_product.argtypes = [i, p, i]
        lib.oracle_esym_product.restype = d
        lib.oracle_esym_newton_girard.argtypes = [i, p]
        lib.oracle_esym_newton_girard.restype = d
        lib.oracle_signed_root.argtypes = [d, i]
        lib.oracle_signed_root.restype = d
        lib.oracle_fir_length.argtypes = [d, d]
        lib.oracle_fir_length.restype = i
        lib.oracle_fir_taps.argtypes = [d, d, i, p]
        lib.oracle_fir_taps.restype = i
        lib.oracle_envelope.argtypes = [i, p, i, p, p]
        lib.oracle_envelope.restype = None
        lib.oracle_matched_filter.argtypes = [i, i, p, i, p, p]
        lib.oracle_matched_filter.restype = None
        lib.oracle_dmas.argtypes = [i, i, p, i, p, d, i, i, i, d, i, p, i, i, p, p, p]
        lib.oracle_dmas.restype = i
        lib.oracle_linear_esym_ld.argtypes = [i, i, p, p, d, i, i]
        lib.oracle_linear_esym_ld.restype = d
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int = 0) -> int:
    """Set (n > 0) and return the number of OpenMP threads the oracle uses."""
    return int(_load().oracle_set_threads(int(n)))


def unit_vectors(azel) -> np.ndarray:
    """[M][2] (azimuth, elevation) radians -> [M][3] unit vectors (Fig. 1 axes)."""
    azel = _f64(azel).reshape(-1, 2)
    u = np.empty((azel.shape[0], 3))
    _load().oracle_unit_vectors(azel.shape[0], _ptr(azel), _ptr(u))
    return u


def geometric_delays(xyz, u, c: float) -> np.ndarray:
    """Delay look-up table tau[M][N] in seconds (Sec. II)."""
    xyz = _f64(xyz).reshape(-1, 3)
    u = _f64(u).reshape(-1, 3)
    tau = np.empty((u.shape[0], xyz.shape[0]))
    _load().oracle_geometric_delays(xyz.shape[0], _ptr(xyz), u.shape[0], _ptr(u),
                                    float(c), _ptr(tau))
    return tau


def round_shifts(tau, fs: float) -> np.ndarray:
    """Nearest-sample shifts llround(tau * fs) as int64, same shape as tau."""
    lib = _load()
    tau = _f64(tau)
    out = np.empty(tau.shape, dtype=np.int64)
    flat_in, flat_out = tau.reshape(-1), out.reshape(-1)
    for k in range(flat_in.size):
        flat_out[k] = lib.oracle_round_shift(float(flat_in[k]), float(fs))
    return out


def esym_product(r, n: int) -> float:
    """E_n(r) via the coefficients of prod_i (1 + r_i z) (Eq. dmasn)."""
    r = _f64(r).reshape(-1)
    return float(_load().oracle_esym_product(r.size, _ptr(r), int(n)))


def esym_newton_girard(P, n: int) -> float:
    """E_n from power sums P[1..n] (P[0] ignored) by Eq. girard_newton_general."""
    P = _f64(P).reshape(-1)
    if P.size < n + 1:
        raise ValueError("P must hold P[0..n]")
    return float(_load().oracle_esym_newton_girard(int(n), _ptr(P)))


def signed_root(x: float, n: int) -> float:
    return float(_load().oracle_signed_root(float(x), int(n)))


def fir_length(fs: float, fc: float) -> int:
    return int(_load().oracle_fir_length(float(fs), float(fc)))


def fir_taps(fs: float, fc: float, L: int | None = None) -> np.ndarray:
    """Envelope low-pass taps h[-H..H] (stored 0..L-1), unit DC gain."""
    if L is None:
        L = fir_length(fs, fc)
    h = np.empty(int(L))
    if _load().oracle_fir_taps(float(fs), float(fc), int(L), _ptr(h)) != 0:
        raise ValueError("FIR length must be odd and positive")
    return h


def envelope(y, h) -> np.ndarray:
    """|y| filtered by h along the last axis, zero padded at both ends."""
    y = _f64(y)
    h = _f64(h)
    out = np.empty_like(y)
    rows_in, rows_out = y.reshape(-1, y.shape[-1]), out.reshape(-1, y.shape[-1])
    for k in range(rows_in.shape[0]):
        rin = np.ascontiguousarray(rows_in[k])
        rout = np.empty_like(rin)
        _load().oracle_envelope(rin.size, _ptr(rin), h.size, _ptr(h), _ptr(rout))
        rows_out[k] = rout
    return out


def matched_filter(frame, e) -> np.ndarray:
    """Each row of frame [N][T] correlated with the emitted signal e [L]:
    out[i][t] = sum_k e[k] frame[i][t + k], zero past the frame end."""
    frame = _f64(frame)
    e = _f64(e)
    if frame.ndim != 2 or e.ndim != 1 or e.size < 1:
        raise ValueError("frame must be [N][T] and e a non-empty vector")
    out = np.empty_like(frame)
    _load().oracle_matched_filter(frame.shape[0], frame.shape[1], _ptr(frame), e.size, _ptr(e),
                                  _ptr(out))
    return out


def dmas(frame, tau, fs: float, order: int, delay_mode: int = ROUND,
         use_cf: bool = True, cf_eps: float = 1e-30, taps=None,
         dir_range: tuple[int, int] | None = None) -> dict:
    """Full DMAS(-CF) image.

    frame : [N][T] samples; tau : [M][N] seconds.  Returns a dict with
    ``y`` (E_n or E_n * CF), ``cf`` and, when taps are given, ``img`` (the
    envelope), each [D][T] for the D directions of ``dir_range``.
    """
    frame = _f64(frame)
    tau = _f64(tau)
    N, T = frame.shape
    M = tau.shape[0]
    if tau.shape[1] != N:
        raise ValueError("tau must be [M][N]")
    b, e = (0, M) if dir_range is None else dir_range
    D = e - b
    y = np.empty((D, T))
    cf = np.empty((D, T))
    img = None
    L = 0
    hp = None
    if taps is not None:
        taps = _f64(taps)
        L = taps.size
        hp = _ptr(taps)
        img = np.empty((D, T))
    rc = _load().oracle_dmas(N, T, _ptr(frame), M, _ptr(tau), float(fs), int(order),
                             int(delay_mode), int(bool(use_cf)), float(cf_eps), L, hp,
                             int(b), int(e), _ptr(y), _ptr(cf),
                             _ptr(img) if img is not None else None)
    if rc != 0:
        raise ValueError("oracle_dmas rejected its arguments")
    out = {"y": y, "cf": cf}
    if img is not None:
        out["img"] = img
    return out


def linear_esym_ld(frame, tau_row, fs: float, order: int, t: int) -> float:
    """Long-double E_n of one LINEAR-mode pixel (spot check of FP64 rounding)."""
    frame = _f64(frame)
    tau_row = _f64(tau_row).reshape(-1)
    N, T = frame.shape
    return float(_load().oracle_linear_esym_ld(N, T, _ptr(frame), _ptr(tau_row),
                                               float(fs), int(order), int(t)))
