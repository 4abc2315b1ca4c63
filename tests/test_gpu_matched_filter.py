"""Matched filter (pulse compression, Sec. II step 1) on the GPU against the
oracle: the frame is correlated with the emitted signal before the roots.
Oracle side: oracle.matched_filter in FP64, then the FP64 beamformer on its
output.  FP32 gate as for the rest of the path (eps_peak <= 1e-5 on y and the
image, |CF error| <= 1e-5)."""
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


@functools.lru_cache(maxsize=None)
def chirp_2d(T=4096):
    return scenes.small_2d(seed=1, n_samples=T, pulse="chirp")


def _filtered(sc, e):
    return dataclasses.replace(sc, frame=oracle.matched_filter(sc.frame, e))


def _run(sc, e, order, mode, **kw):
    plan = gpu_plan(dm, sc, order, mode, mf_signal=e, **kw)
    x = torch.from_numpy(sc.frame).cuda()
    y = torch.empty((sc.n_dirs, sc.n_samples), device="cuda")
    cf = torch.empty_like(y)
    img = plan(x, y=y, cf=cf)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    return {"y": y.cpu().numpy(), "cf": cf.cpu().numpy(), "img": img.cpu().numpy()}


def _check(g, r):
    assert eps_peak(g["y"], r["y"]) <= TOL_F32, eps_peak(g["y"], r["y"])
    assert float(np.max(np.abs(g["cf"] - r["cf"]))) <= 1e-5
    assert eps_peak(g["img"], r["img"]) <= TOL_F32, eps_peak(g["img"], r["img"])


@pytest.mark.parametrize("order,mode", [(5, "round"), (3, "round"), (5, "linear"), (2, "linear")])
def test_matched_filter_chirp_scene(order, mode):
    sc = chirp_2d()
    e = scenes.lfm_chirp(sc.fs).astype(np.float32)
    gm, om = (dm.ROUND, oracle.ROUND) if mode == "round" else (dm.LINEAR, oracle.LINEAR)
    _check(_run(sc, e, order, gm), oracle_run(_filtered(sc, e.astype(np.float64)), order, om))


@pytest.mark.parametrize("T,L", [(2305, 37), (3000, 8192), (700, 1), (5000, 1126)])
def test_matched_filter_lengths_and_ragged_frames(T, L):
    """Tile edges (2304 outputs per CTA, 9 per thread), a filter longer than
    the frame, a one-sample filter, a length that is not a multiple of 18."""
    sc = chirp_2d(T)
    e = np.random.default_rng(L).standard_normal(L).astype(np.float32)
    _check(_run(sc, e, 3, dm.ROUND),
           oracle_run(_filtered(sc, e.astype(np.float64)), 3, oracle.ROUND))


def test_matched_filter_in_batches_and_host_path_is_bitwise_the_same():
    sc = chirp_2d()
    big = scenes.hemi_3d(seed=2, n_samples=8192, n_dirs=1024, pulse="chirp")
    e = scenes.lfm_chirp(sc.fs).astype(np.float32)
    p1 = gpu_plan(dm, sc, 5, dm.ROUND, mf_signal=e)
    p2 = gpu_plan(dm, big, 5, dm.LINEAR, mf_signal=e[:600])
    p3 = gpu_plan(dm, sc, 3, dm.ROUND)                      # no filter, in the same batch
    f1, f2 = torch.from_numpy(sc.frame).cuda(), torch.from_numpy(big.frame).cuda()
    a1, a2, a3 = p1(f1).clone(), p2(f2).clone(), p3(f1).clone()
    b = dm.beamform_batch([p1, p2, p3, p2], [f1, f2, f1, f2])
    torch.cuda.synchronize()
    assert torch.equal(b[0], a1) and torch.equal(b[1], a2) and torch.equal(b[2], a3)
    assert torch.equal(b[3], a2)
    h2 = p2.beamform_host(big.frame)          # 1024 x 8192: the chunked host path
    assert np.array_equal(h2, a2.cpu().numpy())
    for p in (p1, p2, p3):
        p.check()
        p.close()


def test_matched_filter_full_size_sampled_rows():
    """The hemisphere frame with chirp echoes and the eRTIS call as the
    matched filter (2048 x 16384, linear delays, n = 5)."""
    sc = scenes.hemi_3d(seed=2, pulse="chirp")
    e = scenes.lfm_chirp(sc.fs).astype(np.float32)
    plan = gpu_plan(dm, sc, 5, dm.LINEAR, mf_signal=e)
    x = torch.from_numpy(sc.frame).cuda()
    y = torch.empty((sc.n_dirs, sc.n_samples), device="cuda")
    img = plan(x, y=y)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    fsc = _filtered(sc, e.astype(np.float64))
    tau = scene_tau(sc)
    peak_row = int(torch.argmax(torch.amax(torch.abs(y), dim=1)).item())
    starts = sorted({0, 700, 1500, 2040, min(max(peak_row - 4, 0), 2040)})
    peak_y = peak_i = err_y = err_i = 0.0
    for b in starts:
        r = oracle_run(fsc, 5, oracle.LINEAR, dir_range=(b, b + 8), tau=tau)
        gy, gi = y[b:b + 8].cpu().numpy(), img[b:b + 8].cpu().numpy()
        peak_y, peak_i = max(peak_y, np.abs(r["y"]).max()), max(peak_i, np.abs(r["img"]).max())
        err_y = max(err_y, np.abs(gy - r["y"]).max())
        err_i = max(err_i, np.abs(gi - r["img"]).max())
    assert err_y <= TOL_F32 * peak_y, err_y / peak_y
    assert err_i <= TOL_F32 * peak_i, err_i / peak_i
