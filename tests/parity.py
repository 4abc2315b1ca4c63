"""Helpers shared by the GPU parity tests: run a scene through the CUDA
library and through the oracle on the same seeded inputs, and compare.

Error measures (per-pixel relative error is meaningless where E_n crosses
zero, so errors are taken relative to the image peak):
  eps_peak = max |gpu - ref| / max |ref|
  db_err   = |20 log10(|gpu| / |ref|)| over pixels within `floor_db` of the peak
"""
from __future__ import annotations

import numpy as np

import oracle

# FP32 path (FP32 channels and sums): peak-relative tolerance on y and on the
# envelope image.
TOL_F32 = 1e-5


def eps_peak(gpu, ref) -> float:
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    peak = float(np.max(np.abs(ref)))
    if peak == 0.0:
        return float(np.max(np.abs(gpu)))
    return float(np.max(np.abs(gpu - ref)) / peak)


def db_error(gpu, ref, floor_db: float = 60.0):
    gpu = np.abs(np.asarray(gpu, dtype=np.float64))
    ref = np.abs(np.asarray(ref, dtype=np.float64))
    peak = ref.max()
    mask = ref > peak * 10.0 ** (-floor_db / 20.0)
    with np.errstate(divide="ignore"):
        d = np.abs(20.0 * np.log10(np.maximum(gpu[mask], 1e-300) / ref[mask]))
    return float(d.max()), float(d.mean())


def scene_tau(scene) -> np.ndarray:
    """Oracle delay table for a scene's geometry."""
    u = scene.dir_unit if scene.dir_unit is not None else oracle.unit_vectors(scene.dir_azel)
    return oracle.geometric_delays(scene.mic_xyz, u, scene.c)


def oracle_run(scene, order, delay_mode, cf=True, envelope=True, dir_range=None,
               env_cutoff_hz=5000.0, env_taps=None, tau=None):
    if tau is None:
        tau = scene_tau(scene)
    taps = None
    if envelope:
        taps = oracle.fir_taps(scene.fs, env_cutoff_hz, env_taps)
    return oracle.dmas(scene.frame.astype(np.float64), tau, scene.fs, order, delay_mode,
                       use_cf=cf, taps=taps, dir_range=dir_range)


def gpu_plan(dm, scene, order, delay_mode, **kw):
    return dm.Plan(mic_xyz=scene.mic_xyz, dir_azel=scene.dir_azel, dir_unit=scene.dir_unit,
                   n_samples=scene.n_samples, fs=scene.fs, c=scene.c, order=order,
                   delay_mode=delay_mode, **kw)
