"""Every order at once (dmas_beamform_orders): DAS and DMAS-2..n, with and
without the coherence factor, from one pass, against the FP64 oracle run once
per (order, CF) on the same seeded frame.

FP32 gate as for the single-order path: eps_peak <= 1e-5 on every image (the
envelope, or E_k (x CF) without it) and |CF error| <= 1e-5.
"""
import dataclasses
import functools

import numpy as np
import pytest

import oracle
from parity import TOL_F32, eps_peak, gpu_plan, oracle_run, scene_tau
from workloads import scenes

torch = pytest.importorskip("torch")
dm = pytest.importorskip("paper_2511_09165_b300")

pytestmark = pytest.mark.gpu

MODES = {"round": (dm.ROUND, oracle.ROUND), "linear": (dm.LINEAR, oracle.LINEAR)}


@functools.lru_cache(maxsize=None)
def small_2d(T=4096):
    return scenes.small_2d(seed=1, n_samples=T)


@functools.lru_cache(maxsize=None)
def hemi(T=2048, M=256):
    return scenes.hemi_3d(seed=2, n_samples=T, n_dirs=M)


def run_orders(sc, nmax, mode, orders=None, variants=dm.V_PLAIN | dm.V_CF, **kw):
    plan = gpu_plan(dm, sc, nmax, MODES[mode][0], **kw)
    x = torch.from_numpy(sc.frame).cuda()
    cf = torch.empty((sc.n_dirs, sc.n_samples), device="cuda")
    img = plan.beamform_orders(x, orders=orders, variants=variants, cf=cf)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    return img.cpu().numpy(), cf.cpu().numpy()


def check_against_oracle(sc, img, cf, orders, variants, mode, envelope=True, tau=None,
                         dir_range=None):
    tau = scene_tau(sc) if tau is None else tau
    vs = [v for v in (dm.V_PLAIN, dm.V_CF) if variants & v]
    for vi, v in enumerate(vs):
        for ki, k in enumerate(orders):
            r = oracle_run(sc, k, MODES[mode][1], cf=(v == dm.V_CF), envelope=envelope,
                           tau=tau, dir_range=dir_range)
            ref = r["img"] if envelope else r["y"]
            got = img[vi, ki] if dir_range is None else img[vi, ki, dir_range[0]:dir_range[1]]
            e = eps_peak(got, ref)
            assert e <= TOL_F32, (k, v, e)
            if vi == 0 and ki == 0:
                gcf = cf if dir_range is None else cf[dir_range[0]:dir_range[1]]
                assert float(np.max(np.abs(gcf - r["cf"]))) <= 1e-5


@pytest.mark.parametrize("mode", ["round", "linear"])
@pytest.mark.parametrize("envelope", [True, False])
def test_all_orders_2d(mode, envelope):
    """The 2-D frame (32 mics, 91 directions, 4096 samples): all ten images."""
    sc = small_2d()
    img, cf = run_orders(sc, 5, mode, envelope=envelope)
    assert img.shape == (2, 5, sc.n_dirs, sc.n_samples)
    check_against_oracle(sc, img, cf, [1, 2, 3, 4, 5], dm.V_PLAIN | dm.V_CF, mode, envelope)


@pytest.mark.parametrize("nmax", [1, 2, 3, 4])
@pytest.mark.parametrize("mode", ["round", "linear"])
def test_lower_highest_orders(nmax, mode):
    """Plans of order 1..4: their passes keep fewer running sums."""
    sc = hemi(T=1500, M=100)
    img, cf = run_orders(sc, nmax, mode, envelope=False)
    check_against_oracle(sc, img, cf, list(range(1, nmax + 1)), dm.V_PLAIN | dm.V_CF, mode,
                         envelope=False)


@pytest.mark.parametrize("ng", ["f64", "cf32"])
def test_newton_girard_precisions(ng):
    sc = hemi()
    prec = {"f64": dm.NG_F64, "cf32": dm.NG_CF32}[ng]
    img, cf = run_orders(sc, 5, "linear", ng_prec=prec)
    check_against_oracle(sc, img, cf, [1, 2, 3, 4, 5], dm.V_PLAIN | dm.V_CF, "linear")


def test_selected_orders_and_variants_are_the_full_pass_images():
    """A mask and a variant choice only decide which images are written: each
    one is bitwise the full pass's."""
    sc = hemi()
    full, cf_full = run_orders(sc, 5, "linear")
    sub, cf_sub = run_orders(sc, 5, "linear", orders=[2, 5], variants=dm.V_CF)
    assert sub.shape == (1, 2, sc.n_dirs, sc.n_samples)
    assert np.array_equal(sub[0, 0], full[1, 1])
    assert np.array_equal(sub[0, 1], full[1, 4])
    assert np.array_equal(cf_sub, cf_full)
    plain, _ = run_orders(sc, 5, "round", orders=[3], variants=dm.V_PLAIN)
    full_r, _ = run_orders(sc, 5, "round", variants=dm.V_PLAIN)
    assert np.array_equal(plain[0, 0], full_r[0, 2])


@pytest.mark.parametrize("mode", ["round", "linear"])
def test_each_image_matches_the_single_order_path(mode):
    """Same frame through dmas_beamform with plans of order k, CF on and off."""
    sc = hemi()
    img, _ = run_orders(sc, 5, mode)
    x = torch.from_numpy(sc.frame).cuda()
    for k in range(1, 6):
        for vi, use_cf in enumerate((False, True)):
            plan = gpu_plan(dm, sc, k, MODES[mode][0], cf=use_cf)
            single = plan(x).cpu().numpy()
            plan.close()
            assert eps_peak(img[vi, k - 1], single) <= TOL_F32, (k, use_cf)


def test_matched_filter_plan():
    sc = scenes.small_2d(seed=1, n_samples=4096, pulse="chirp")
    e = scenes.lfm_chirp(sc.fs).astype(np.float32)
    img, cf = run_orders(sc, 5, "round", mf_signal=e)
    filt = dataclasses.replace(sc, frame=oracle.matched_filter(sc.frame, e.astype(np.float64)))
    check_against_oracle(filt, img, cf, [1, 2, 3, 4, 5], dm.V_PLAIN | dm.V_CF, "round",
                         tau=scene_tau(sc))


def test_ragged_and_chunked():
    """A frame that ends inside a tile, a direction count that leaves empty
    warps, and an array large enough to need several microphone stages."""
    sc = scenes.passive(seed=4, n_mics=100, n_samples=700, n_az=16, n_el=8)
    for mode in ("round", "linear"):
        plan = gpu_plan(dm, sc, 5, MODES[mode][0])
        assert plan.info().n_mics == 100
        plan.close()
        img, cf = run_orders(sc, 5, mode, orders=[1, 3, 5])
        check_against_oracle(sc, img, cf, [1, 3, 5], dm.V_PLAIN | dm.V_CF, mode)


@pytest.mark.parametrize("mode", ["round", "linear"])
def test_frame_length_not_a_multiple_of_four(mode):
    """T % 4 != 0: the envelope of the ten images takes its plain-load path and
    the last time tile is ragged."""
    sc = hemi(T=1501, M=100)
    img, cf = run_orders(sc, 5, mode)
    check_against_oracle(sc, img, cf, [1, 2, 3, 4, 5], dm.V_PLAIN | dm.V_CF, mode)


def test_full_size_hemisphere_sampled_rows():
    """The 3-D frame in its benchmark size (2048 directions, 16384 samples,
    interpolated delays): rows sampled across the direction range."""
    sc = scenes.hemi_3d(seed=2)
    img, cf = run_orders(sc, 5, "linear")
    tau = scene_tau(sc)
    M = sc.n_dirs
    for b in (0, M // 3 + 5, M - 8):
        check_against_oracle(sc, img, cf, [1, 2, 3, 4, 5], dm.V_PLAIN | dm.V_CF, "linear",
                             tau=tau, dir_range=(b, b + 8))


def test_rejected_calls():
    sc = hemi(T=512, M=16)
    x = torch.from_numpy(sc.frame).cuda()
    plan = gpu_plan(dm, sc, 5, dm.ROUND)
    for orders, variants in (([], 3), ([6], 3), ([1], 0), ([1], 4)):
        with pytest.raises(dm.DmasError):
            plan.beamform_orders(x, orders=orders, variants=variants)
    plan.close()
    for kw, order in (({"chan_prec": dm.CH_F16}, 5), ({}, 6)):
        plan = gpu_plan(dm, sc, order, dm.ROUND, **kw)
        with pytest.raises(dm.DmasError):
            plan.beamform_orders(x, orders=[1])
        plan.close()
