"""Image-quality measures of an acoustic image (post-processing only).

The image SNR follows the paper's simulation analysis (Sec. III-A, Table I):
the image is normalised to a maximum of one, E_off is the mean over the
off-target pixels, and SNR_image = 20 log10(1 / E_off).  Which pixels count
as on target is not stated there; here it is the window within max_az_deg of
the target's azimuth and within max_range_m of its range (one-way range
c t).  The peak-to-sidelobe ratio is 20 log10(1 / max over the same
off-target pixels) of the normalised image.

The directional point-spread function (Sec. III-A, the noise-free point
target) is the image's maximum over t per direction, normalised to one; its
dynamic range is read here as 20 log10(1 / median over the directions outside
the main lobe), the depth of its typical side-lobe floor (the paper reads the
range off a plot and gives no formula).
"""
from __future__ import annotations

import numpy as np


def off_target_mask(az_rad: np.ndarray, n_samples: int, fs: float, c: float,
                    target_az_rad: float, target_range_m: float,
                    max_az_deg: float = 10.0, max_range_m: float = 0.15) -> np.ndarray:
    """Boolean [M][T]: True for pixels outside the target window."""
    az_off = np.abs(np.degrees(az_rad - target_az_rad)) > max_az_deg
    rng = c * np.arange(n_samples) / fs
    r_off = np.abs(rng - target_range_m) > max_range_m
    return az_off[:, None] | r_off[None, :]


def image_snr_db(image: np.ndarray, off: np.ndarray) -> float:
    img = np.abs(np.asarray(image, dtype=np.float64))
    img = img / img.max()
    return float(20.0 * np.log10(1.0 / img[off].mean()))


def peak_sidelobe_db(image: np.ndarray, off: np.ndarray) -> float:
    img = np.abs(np.asarray(image, dtype=np.float64))
    img = img / img.max()
    return float(20.0 * np.log10(1.0 / img[off].max()))


def directional_psf(image: np.ndarray) -> np.ndarray:
    """[M]: max over t of |image|, normalised to a maximum of one."""
    p = np.abs(np.asarray(image, dtype=np.float64)).max(axis=1)
    return p / p.max()


def psf_dynamic_range_db(image: np.ndarray, az_rad: np.ndarray, target_az_rad: float,
                         main_lobe_deg: float = 10.0) -> float:
    p = directional_psf(image)
    side = np.abs(np.degrees(az_rad - target_az_rad)) > main_lobe_deg
    return float(20.0 * np.log10(1.0 / np.median(p[side])))
