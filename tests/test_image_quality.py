"""The paper's qualitative image-quality claims (Sec. III-A, Table I), checked
on a seeded point-target scene: at 0 dB microphone SNR the image SNR (mean
off-target level of the normalised image) rises with the DMAS order and the
coherence factor raises it at every order; without noise, the dynamic range
of the directional point-spread function does the same.  The absolute values
depend on details the paper does not give (array, pulse, target window) and
are not pinned.

CPU: the FP64 oracle shows the trends.  GPU: the CUDA path shows them; its
image SNR agrees with the oracle's to 0.01 dB and its PSF dynamic range (all
ten images from one every-order pass) to 0.5 dB.
"""
import functools

import numpy as np
import pytest

import oracle
from parity import gpu_plan, oracle_run
from workloads import image_quality as iq
from workloads import scenes

ORDERS = (1, 2, 3, 4, 5)


@functools.lru_cache(maxsize=None)
def _scene():
    sc = scenes.point_target(0.0)
    off = iq.off_target_mask(sc.dir_azel[:, 0], sc.n_samples, sc.fs, sc.c, 0.0, 1.0)
    return sc, off


@functools.lru_cache(maxsize=None)
def _oracle_snr():
    sc, off = _scene()
    return {(n, cf): iq.image_snr_db(oracle_run(sc, n, oracle.LINEAR, cf=cf)["img"], off)
            for n in ORDERS for cf in (False, True)}


def _assert_trend(snr):
    for cf in (False, True):
        vals = [snr[(n, cf)] for n in ORDERS]
        assert all(b > a + 1.0 for a, b in zip(vals, vals[1:])), (cf, vals)
    for n in ORDERS:
        assert snr[(n, True)] > snr[(n, False)] + 3.0, n


def test_oracle_image_snr_rises_with_order_and_cf():
    _assert_trend(_oracle_snr())


def test_oracle_cf_gain_shrinks_with_order_only_under_an_image_floor():
    """Table I's coherence-factor gain shrinks with the order (+23 dB for DAS,
    +7 dB for DMAS5) while its no-CF column rises to 71 dB.  On the oracle, at
    20 dB microphone SNR (where the no-CF column lands within 3 dB of Table
    I's: 31, 45, 57, 66, 74 dB) the CF gain grows with the order as long as
    the normalised image keeps its full range, and shrinks from DAS to DMAS5
    once the image is floored at -80 dB relative to its peak (the CF images
    then saturate near 80 dB, as Table I's do at 78 dB): the reading that
    reproduces the paper's trend is a finite image dynamic range of about
    80 dB, with an effective SNR about 20 dB above this scene's definition."""
    sc = scenes.point_target(20.0)
    off = iq.off_target_mask(sc.dir_azel[:, 0], sc.n_samples, sc.fs, sc.c, 0.0, 1.0)
    imgs = {(n, cf): oracle_run(sc, n, oracle.LINEAR, cf=cf)["img"]
            for n in (1, 5) for cf in (False, True)}

    def snr(img, floor_db=None):
        a = np.abs(img) / np.abs(img).max()
        if floor_db is not None:
            a = np.maximum(a, 10.0 ** (-floor_db / 20.0))
        return iq.image_snr_db(a, off)

    gain_full = [snr(imgs[(n, True)]) - snr(imgs[(n, False)]) for n in (1, 5)]
    gain_floor = [snr(imgs[(n, True)], 80.0) - snr(imgs[(n, False)], 80.0) for n in (1, 5)]
    assert gain_full[1] > gain_full[0]                  # full range: grows with the order
    assert gain_floor[1] < gain_floor[0] - 10.0         # -80 dB floor: shrinks, as in Table I
    assert 70.0 < snr(imgs[(5, False)]) < 78.0          # DMAS5 no CF near Table I's 71 dB


@pytest.mark.gpu
def test_gpu_image_snr_matches_oracle_and_trend():
    torch = pytest.importorskip("torch")
    dm = pytest.importorskip("paper_2511_09165_b300")
    sc, off = _scene()
    x = torch.from_numpy(sc.frame).cuda()
    got = {}
    for n in ORDERS:
        for cf in (False, True):
            plan = gpu_plan(dm, sc, n, dm.LINEAR, cf=cf)
            got[(n, cf)] = iq.image_snr_db(plan(x).cpu().numpy(), off)
            plan.check()
            plan.close()
    _assert_trend(got)
    ref = _oracle_snr()
    for k, v in got.items():
        assert abs(v - ref[k]) < 0.01, (k, v, ref[k])


@functools.lru_cache(maxsize=None)
def _psf_scene():
    return scenes.point_target(float("inf"))


@functools.lru_cache(maxsize=None)
def _oracle_psf():
    sc = _psf_scene()
    az = sc.dir_azel[:, 0]
    return {(n, cf): iq.psf_dynamic_range_db(oracle_run(sc, n, oracle.LINEAR, cf=cf)["img"],
                                             az, 0.0)
            for n in ORDERS for cf in (False, True)}


def _assert_psf_trend(dr):
    for cf in (False, True):
        vals = [dr[(n, cf)] for n in ORDERS]
        assert all(b > a + 3.0 for a, b in zip(vals, vals[1:])), (cf, vals)
    for n in ORDERS:
        assert dr[(n, True)] > dr[(n, False)] + 3.0, n


def test_oracle_psf_dynamic_range_rises_with_order_and_cf():
    _assert_psf_trend(_oracle_psf())


@pytest.mark.gpu
def test_gpu_psf_dynamic_range_matches_oracle_and_trend():
    torch = pytest.importorskip("torch")
    dm = pytest.importorskip("paper_2511_09165_b300")
    sc = _psf_scene()
    az = sc.dir_azel[:, 0]
    plan = gpu_plan(dm, sc, 5, dm.LINEAR)
    imgs = plan.beamform_orders(torch.from_numpy(sc.frame).cuda()).cpu().numpy()
    plan.check()
    plan.close()
    got = {(n, cf): iq.psf_dynamic_range_db(imgs[int(cf), n - 1], az, 0.0)
           for n in ORDERS for cf in (False, True)}
    _assert_psf_trend(got)
    ref = _oracle_psf()
    for k, v in got.items():
        assert abs(v - ref[k]) < 0.5, (k, v, ref[k])
