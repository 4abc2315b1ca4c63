"""Seeded synthetic sonar scenes and direction grids.

This module feeds both the CUDA library and the oracle with the same inputs.
It holds none of the beamforming arithmetic: it only synthesises microphone
signals from point reflectors or sources (spherical propagation, one-way path
length d, amplitude 1/d) and lists the direction grids to image.  Directions
are returned either as (azimuth, elevation) pairs in radians or, for the
Fibonacci grid, as unit vectors in the array frame (array in the z = 0 plane,
broadside along +z, x horizontal, y vertical).

The paper's recorded eRTIS dataset is not available; these scenes stand in
for it with its array size (32 microphones), sample rate (450 kHz) and the
frame lengths of the benchmark configurations.

Recipes (all draws from numpy.random.default_rng(seed)):

  small_2d   32 mics area-uniform in a 12 cm disc, fs 450 kHz, T 4096, three
             reflectors (azimuth U(-60, 60) deg, elevation 0, range U(0.5, 3) m,
             amplitude 1), Gaussian-windowed 40 kHz echo (sigma 50 us),
             white noise at 20 dB SNR, 91 azimuths -90..90 deg, elevation 0.
  hemi_3d    the same array, T 16384, 2048 directions on a frontal-hemisphere
             Fibonacci grid, eight reflectors (area-uniform on the hemisphere,
             range U(0.3, 6) m, amplitude log-uniform over 40 dB), 10 dB SNR.
  passive    N in {64, 256} mics uniform in a 0.4 m square, fs 400 kHz,
             T 32768, four broadband sources (white noise band-passed to
             20-80 kHz, unit RMS, azimuth/elevation U(-60, 60) deg, range
             U(1, 5) m, exact frequency-domain fractional delay, amplitude 1/d)
             plus uncorrelated sensor noise at 0 dB SNR; 128 x 64 az/el grid
             over [-60, 60] deg.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SOUND_SPEED = 343.0


@dataclass
class Scene:
    """One synthetic frame with the geometry needed to image it."""
    name: str
    mic_xyz: np.ndarray            # [N][3] float64 metres
    frame: np.ndarray              # [N][T] float32 samples
    fs: float
    c: float
    dir_azel: np.ndarray | None    # [M][2] float64 radians, or None
    dir_unit: np.ndarray | None    # [M][3] float64, or None
    meta: dict = field(default_factory=dict)

    @property
    def n_mics(self) -> int:
        return int(self.frame.shape[0])

    @property
    def n_samples(self) -> int:
        return int(self.frame.shape[1])

    @property
    def n_dirs(self) -> int:
        if self.dir_unit is not None:
            return int(self.dir_unit.shape[0])
        return int(self.dir_azel.shape[0])


# --------------------------------------------------------------------------
# arrays
# --------------------------------------------------------------------------
def disc_array(rng: np.random.Generator, n: int, radius: float) -> np.ndarray:
    """n positions area-uniform in a disc of the given radius, z = 0."""
    rad = radius * np.sqrt(rng.random(n))
    ang = 2.0 * np.pi * rng.random(n)
    return np.stack([rad * np.cos(ang), rad * np.sin(ang), np.zeros(n)], axis=1)


def square_array(rng: np.random.Generator, n: int, side: float) -> np.ndarray:
    """n positions uniform in a side x side square centred on 0, z = 0."""
    xy = (rng.random((n, 2)) - 0.5) * side
    return np.concatenate([xy, np.zeros((n, 1))], axis=1)


# --------------------------------------------------------------------------
# direction grids
# --------------------------------------------------------------------------
def azimuth_fan(start_deg: float = -90.0, stop_deg: float = 90.0,
                step_deg: float = 2.0) -> np.ndarray:
    """Azimuths start..stop (inclusive) at elevation 0 -> [M][2] radians."""
    count = int(round((stop_deg - start_deg) / step_deg)) + 1
    az = np.deg2rad(start_deg + step_deg * np.arange(count))
    return np.stack([az, np.zeros_like(az)], axis=1)


def azel_grid(n_az: int, n_el: int, lim_deg: float = 60.0) -> np.ndarray:
    """n_az x n_el grid uniform over [-lim, lim] in both angles -> [M][2]."""
    az = np.deg2rad(np.linspace(-lim_deg, lim_deg, n_az))
    el = np.deg2rad(np.linspace(-lim_deg, lim_deg, n_el))
    A, E = np.meshgrid(az, el, indexing="xy")
    return np.stack([A.reshape(-1), E.reshape(-1)], axis=1)


def fibonacci_hemisphere(m: int) -> np.ndarray:
    """m unit vectors on the frontal (+z) hemisphere, Fibonacci spiral."""
    k = np.arange(m, dtype=np.float64)
    z = (k + 0.5) / m
    rho = np.sqrt(1.0 - z * z)
    ang = k * np.pi * (3.0 - math.sqrt(5.0))
    return np.stack([rho * np.cos(ang), rho * np.sin(ang), z], axis=1)


def _point(az: float, el: float, rng_m: float) -> np.ndarray:
    """Scene position at azimuth/elevation/range (x horizontal, y up, z ahead)."""
    return rng_m * np.array([math.sin(az) * math.cos(el), math.sin(el),
                             math.cos(az) * math.cos(el)])


# --------------------------------------------------------------------------
# signals
# --------------------------------------------------------------------------
def lfm_chirp(fs: float, f0: float = 25e3, f1: float = 50e3, duration: float = 2.5e-3,
              tau=None) -> np.ndarray:
    """Linear FM chirp sin(2 pi (f0 tau + (f1 - f0) tau^2 / (2 D))) for 0 <= tau < D,
    zero elsewhere; sampled at k / fs (k < round(D fs)) when tau is None.  The
    defaults are the eRTIS call: 2.5 ms from 25 to 50 kHz."""
    if tau is None:
        tau = np.arange(int(round(duration * fs))) / fs
    tau = np.asarray(tau, dtype=np.float64)
    phase = 2.0 * np.pi * (f0 * tau + 0.5 * (f1 - f0) / duration * tau * tau)
    return np.where((tau >= 0.0) & (tau < duration), np.sin(phase), 0.0)


def _echo_frame(rng, mic_xyz, positions, amps, fs, T, c, f0, sigma, noise_eta, pulse="tone"):
    """Echo of each point at one-way delay d/c, amplitude a/d: the Gaussian-
    windowed tone at f0 (pulse "tone") or the eRTIS chirp (pulse "chirp",
    evaluated at the exact delayed time)."""
    N = mic_xyz.shape[0]
    t = np.arange(T) / fs
    sig = np.zeros((N, T))
    for p, a in zip(positions, amps):
        d = np.linalg.norm(mic_xyz - p[None, :], axis=1)
        for i in range(N):
            tt = t - d[i] / c
            if pulse == "chirp":
                sig[i] += a / d[i] * lfm_chirp(fs, tau=tt)
            else:
                sig[i] += a / d[i] * np.exp(-tt * tt / (2.0 * sigma * sigma)) * \
                    np.cos(2.0 * np.pi * f0 * tt)
    sig += noise_eta * rng.standard_normal((N, T))
    return sig


def small_2d(seed: int = 1, n_mics: int = 32, n_samples: int = 4096,
             n_reflectors: int = 3, snr_db: float = 20.0, n_dirs: int = 91,
             pulse: str = "tone") -> Scene:
    """2-D scene: 12 cm disc, n_dirs azimuths evenly spaced over -90..90 degrees
    at elevation 0 (91: every 2 degrees); echoes of the Gaussian tone or, with
    pulse="chirp", of the eRTIS chirp."""
    rng = np.random.default_rng(seed)
    fs, c = 450e3, SOUND_SPEED
    mic = disc_array(rng, n_mics, 0.06)
    pos, amps = [], []
    for _ in range(n_reflectors):
        az = math.radians(rng.uniform(-60.0, 60.0))
        rg = rng.uniform(0.5, 3.0)
        pos.append(_point(az, 0.0, rg))
        amps.append(1.0)
    eta = 10.0 ** (-snr_db / 20.0)
    frame = _echo_frame(rng, mic, pos, amps, fs, n_samples, c, 40e3, 50e-6, eta, pulse)
    dirs = azimuth_fan() if n_dirs == 91 else np.stack(
        [np.deg2rad(np.linspace(-90.0, 90.0, n_dirs)), np.zeros(n_dirs)], axis=1)
    return Scene("small_2d", mic, frame.astype(np.float32), fs, c,
                 dirs, None,
                 {"seed": seed, "reflectors": np.array(pos), "snr_db": snr_db})


def point_target(snr_db: float, seed: int = 11, n_samples: int = 2048,
                 range_m: float = 1.0, az_step_deg: float = 1.0) -> Scene:
    """Image-quality scene: the small_2d array (12 cm disc), one reflector at
    broadside at range_m whose echo has amplitude 1 at the microphones, white
    Gaussian noise of standard deviation 10^(-snr_db/20), azimuths -90..90 deg
    every az_step_deg at elevation 0."""
    mic = disc_array(np.random.default_rng(1), 32, 0.06)
    rng = np.random.default_rng(seed)
    fs, c = 450e3, SOUND_SPEED
    eta = 10.0 ** (-snr_db / 20.0)
    pos = _point(0.0, 0.0, range_m)
    # amplitude a/d with a = range_m: 1 at the array (d differs from range_m by
    # under 0.2 % across a 12 cm aperture at 1 m)
    frame = _echo_frame(rng, mic, [pos], [range_m], fs, n_samples, c, 40e3, 50e-6, eta)
    return Scene("point_target", mic, frame.astype(np.float32), fs, c,
                 azimuth_fan(-90.0, 90.0, az_step_deg), None,
                 {"seed": seed, "snr_db": snr_db, "range_m": range_m})


def hemi_3d(seed: int = 2, n_samples: int = 16384, n_dirs: int = 2048,
            n_reflectors: int = 8, snr_db: float = 10.0, array_seed: int = 1,
            pulse: str = "tone") -> Scene:
    """3-D scene: the small_2d array, Fibonacci hemisphere of directions."""
    mic = disc_array(np.random.default_rng(array_seed), 32, 0.06)
    rng = np.random.default_rng(seed)
    fs, c = 450e3, SOUND_SPEED
    pos, amps = [], []
    for _ in range(n_reflectors):
        z = rng.random()
        ang = 2.0 * np.pi * rng.random()
        rho = math.sqrt(1.0 - z * z)
        u = np.array([rho * math.cos(ang), rho * math.sin(ang), z])
        rg = rng.uniform(0.3, 6.0)
        pos.append(rg * u)
        amps.append(10.0 ** (-2.0 * rng.random()))
    eta = 10.0 ** (-snr_db / 20.0)
    frame = _echo_frame(rng, mic, pos, amps, fs, n_samples, c, 40e3, 50e-6, eta, pulse)
    return Scene("hemi_3d", mic, frame.astype(np.float32), fs, c, None,
                 fibonacci_hemisphere(n_dirs),
                 {"seed": seed, "reflectors": np.array(pos), "amps": np.array(amps),
                  "snr_db": snr_db})


def passive(seed: int = 4, n_mics: int = 64, n_samples: int = 32768,
            n_az: int = 128, n_el: int = 64, n_sources: int = 4) -> Scene:
    """Large passive array: broadband sources, 0 dB sensor noise."""
    rng = np.random.default_rng(seed)
    fs, c = 400e3, SOUND_SPEED
    mic = square_array(rng, n_mics, 0.4)
    T = n_samples
    freqs = np.fft.rfftfreq(T, 1.0 / fs)
    band = (freqs >= 20e3) & (freqs <= 80e3)
    sig = np.zeros((n_mics, T))
    pos = []
    for _ in range(n_sources):
        w = rng.standard_normal(T)
        W = np.fft.rfft(w)
        W[~band] = 0.0
        s = np.fft.irfft(W, T)
        s /= np.sqrt(np.mean(s * s))
        S = np.fft.rfft(s)
        az = math.radians(rng.uniform(-60.0, 60.0))
        el = math.radians(rng.uniform(-60.0, 60.0))
        rg = rng.uniform(1.0, 5.0)
        p = _point(az, el, rg)
        pos.append(p)
        d = np.linalg.norm(mic - p[None, :], axis=1)
        for i in range(n_mics):
            shift = np.exp(-2j * np.pi * freqs * d[i] / c)
            sig[i] += np.fft.irfft(S * shift, T) / d[i]
    rms = float(np.mean(np.sqrt(np.mean(sig * sig, axis=1))))
    sig += rms * rng.standard_normal((n_mics, T))
    return Scene("passive", mic, sig.astype(np.float32), fs, c,
                 azel_grid(n_az, n_el), None,
                 {"seed": seed, "sources": np.array(pos)})


@dataclass
class SensorSpec:
    """One sensor of the serving mix: its array, direction grid and frames."""
    name: str
    mic_xyz: np.ndarray
    n_samples: int
    order: int
    fs: float
    c: float
    dir_azel: np.ndarray | None
    dir_unit: np.ndarray | None
    frames: list  # seeded frames [N][T] float32

    @property
    def n_mics(self) -> int:
        return int(self.mic_xyz.shape[0])

    @property
    def n_dirs(self) -> int:
        return int((self.dir_unit if self.dir_unit is not None else self.dir_azel).shape[0])


def serving_mix(seed: int = 5, n_sensors: int = 16, frames_per_sensor: int = 4,
                mics=(32, 64, 128), dirs=(91, 2048, 8192), samples=(4096, 16384, 32768),
                orders=(3, 5)) -> list:
    """Sensors of the serving workload: each draws its microphone count, direction
    grid (the 91-azimuth fan, the 2048-point hemisphere, the 128 x 64 az/el
    grid), frame length and order; its array is a 12 cm disc of that many
    microphones and its frames are small_2d-style echo scenes (3 reflectors,
    20 dB SNR)."""
    rng = np.random.default_rng(seed)
    out = []
    for s_i in range(n_sensors):
        N = int(rng.choice(mics))
        M = int(rng.choice(dirs))
        T = int(rng.choice(samples))
        n = int(rng.choice(orders))
        fs, c = 450e3, SOUND_SPEED
        mic = disc_array(rng, N, 0.06)
        azel = unit = None
        if M == 91:
            azel = azimuth_fan()
        elif M == 2048:
            unit = fibonacci_hemisphere(2048)
        else:
            azel = azel_grid(128, 64)
        frames = []
        for _ in range(frames_per_sensor):
            pos = []
            for _ in range(3):
                az = math.radians(rng.uniform(-60.0, 60.0))
                pos.append(_point(az, 0.0, rng.uniform(0.5, 3.0)))
            frames.append(_echo_frame(rng, mic, pos, [1.0] * 3, fs, T, c, 40e3, 50e-6,
                                      0.1).astype(np.float32))
        out.append(SensorSpec(f"sensor{s_i}", mic, T, n, fs, c, azel, unit, frames))
    return out


def plane_wave(n_mics: int, n_samples: int, az_deg: float, el_deg: float = 0.0,
               fs: float = 450e3, c: float = SOUND_SPEED, seed: int = 7,
               radius: float = 0.06, t0: float = 2e-3) -> Scene:
    """Far-field pulse from one direction, sampled with its exact arrival times.

    Mic i receives the pulse at t0 - (p_i - p_bar).u / c: microphones further
    along the arrival direction u hear it earlier.
    """
    rng = np.random.default_rng(seed)
    mic = disc_array(rng, n_mics, radius)
    u = _point(math.radians(az_deg), math.radians(el_deg), 1.0)
    proj = (mic - mic.mean(axis=0)) @ u
    t = np.arange(n_samples) / fs
    frame = np.zeros((n_mics, n_samples))
    for i in range(n_mics):
        tt = t - (t0 - proj[i] / c)
        frame[i] = np.exp(-tt * tt / (2.0 * (50e-6) ** 2)) * np.cos(2.0 * np.pi * 40e3 * tt)
    return Scene("plane_wave", mic, frame.astype(np.float32), fs, c,
                 azimuth_fan(-90.0, 90.0, 1.0), None, {"az_deg": az_deg})


def random_frame(seed: int, n_mics: int, n_samples: int, scale: float = 1.0,
                 zero_fraction: float = 0.0) -> np.ndarray:
    """Gaussian frame [N][T] float32, optionally with exact zeros sprinkled in."""
    rng = np.random.default_rng(seed)
    f = scale * rng.standard_normal((n_mics, n_samples))
    if zero_fraction > 0.0:
        f[rng.random(f.shape) < zero_fraction] = 0.0
    return f.astype(np.float32)
