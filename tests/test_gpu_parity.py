"""CUDA path against the FP64 oracle on the same seeded inputs.

FP32 gate: eps_peak <= 1e-5 on E_n*CF (y) and on the envelope image, |CF err|
<= 1e-5.  Cases span several direction groups and time tiles with ragged
tails, every order 1..8, both delay modes, all Newton-Girard precisions, the
reduced-precision channels, microphone chunking, and the degenerate cases.
"""
import functools
import math

import numpy as np
import pytest

import oracle
from workloads import scenes
from parity import TOL_F32, db_error, eps_peak, gpu_plan, oracle_run, scene_tau

torch = pytest.importorskip("torch")
dm = pytest.importorskip("paper_2511_09165_b300")

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def small_2d(T=4096):
    return scenes.small_2d(seed=1, n_samples=T)


@functools.lru_cache(maxsize=None)
def hemi(T=2048, M=256):
    return scenes.hemi_3d(seed=2, n_samples=T, n_dirs=M)


@functools.lru_cache(maxsize=None)
def passive(N=100, T=700, n_az=16, n_el=8):
    return scenes.passive(seed=4, n_mics=N, n_samples=T, n_az=n_az, n_el=n_el)


# Newton-Girard arithmetic: compensated FP32 (the default), FP64, plain FP32
NG = {"cf32": "NG_CF32", "f64": "NG_F64", "f32": "NG_F32"}


def ng_prec(name):
    return getattr(dm, NG[name])


def run_gpu(scene, order, mode, want_y=True, want_cf=True, **kw):
    plan = gpu_plan(dm, scene, order, mode, **kw)
    frame = torch.from_numpy(scene.frame).cuda()
    M, T = scene.n_dirs, scene.n_samples
    y = torch.empty((M, T), device="cuda") if want_y else None
    cf = torch.empty((M, T), device="cuda") if want_cf else None
    img = plan(frame, y=y, cf=cf)
    torch.cuda.synchronize()
    plan.check()
    out = {"img": img.cpu().numpy()}
    if want_y:
        out["y"] = y.cpu().numpy()
    if want_cf:
        out["cf"] = cf.cpu().numpy()
    plan.close()
    return out


def assert_parity(g, r, tol=TOL_F32, envelope=True):
    assert eps_peak(g["y"], r["y"]) <= tol, eps_peak(g["y"], r["y"])
    assert float(np.max(np.abs(g["cf"] - r["cf"]))) <= max(tol, 1e-5)
    if envelope:
        assert eps_peak(g["img"], r["img"]) <= tol, eps_peak(g["img"], r["img"])


# ---------------------------------------------------------------------------
# plan tables and bounded waits
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["small_2d", "hemi", "passive"])
def test_delay_table_matches_oracle(which):
    sc = {"small_2d": small_2d, "hemi": hemi, "passive": passive}[which]()
    tau = scene_tau(sc)
    for mode in (dm.ROUND, dm.LINEAR):
        plan = gpu_plan(dm, sc, 3, mode)
        shift, frac = plan.delays()
        plan.close()
        delta = tau * sc.fs
        if mode == dm.ROUND:
            assert np.array_equal(shift, oracle.round_shifts(tau, sc.fs))
            assert np.all(frac == 0)
        else:
            assert np.array_equal(shift, np.floor(delta).astype(np.int64))
            np.testing.assert_allclose(frac, delta - np.floor(delta), rtol=0, atol=2 ** -24)


def test_taps_match_oracle():
    sc = small_2d(512)
    plan = gpu_plan(dm, sc, 5, dm.ROUND)
    h = plan.taps()
    plan.close()
    ref = oracle.fir_taps(sc.fs, 5000.0)
    assert h.size == ref.size == 181
    np.testing.assert_allclose(h, ref, rtol=1e-7, atol=1e-12)


def test_bounded_wait_reports_timeout_and_context_survives():
    assert dm.selftest_wait_timeout(20.0) == 5   # DMAS_ETIMEOUT, by design
    x = torch.ones(4, device="cuda")
    assert float((x * 2).sum()) == 8.0           # the context is still usable


def test_stage_profiling_events():
    sc = small_2d(2048)
    plan = gpu_plan(dm, sc, 5, dm.ROUND)
    plan.set_profiling(True)
    plan(torch.from_numpy(sc.frame).cuda())
    r, b, e = plan.stage_ms()
    plan.close()
    assert r > 0 and b > 0 and e > 0


# ---------------------------------------------------------------------------
# FP32 path against the oracle
# ---------------------------------------------------------------------------
def test_small_2d_order5_full_frame():
    """32 mics, 91 azimuths, 4096 samples, n = 5, nearest-sample delays, CF,
    envelope: the whole small 2-D workload."""
    sc = small_2d()
    g = run_gpu(sc, 5, dm.ROUND)
    r = oracle_run(sc, 5, oracle.ROUND)
    assert_parity(g, r)


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6, 7, 8])
def test_every_order_round(order):
    sc = small_2d(1000)  # 4 time tiles, the last one ragged; 12 groups, last ragged
    g = run_gpu(sc, order, dm.ROUND)
    r = oracle_run(sc, order, oracle.ROUND)
    assert_parity(g, r)


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
def test_wide_tile_round(order):
    """Nearest-sample frames with enough work take more than two pixel pairs per
    lane (a wider tile): 2047 directions (256 groups, the last with 7) x 1537
    samples (ragged last tile), against a small frame that keeps two pairs
    (128-sample tiles)."""
    sc = hemi(1537, 2047)
    plan = gpu_plan(dm, sc, order, dm.ROUND)
    assert plan.info().time_tile > 128
    plan.close()
    small = gpu_plan(dm, small_2d(1000), order, dm.ROUND)
    assert small.info().time_tile == 128
    small.close()
    g = run_gpu(sc, order, dm.ROUND)
    r = oracle_run(sc, order, oracle.ROUND)
    assert_parity(g, r)


def test_wide_delay_spread_keeps_the_narrow_tile():
    """A nearest-sample frame with enough work for the wide tile but delay
    spreads too long for its staging budget (8 microphones, 2048 directions,
    delays of 0..8900 samples) falls back to two pixel pairs per lane and still
    matches the oracle."""
    rng = np.random.default_rng(11)
    N, T, M, fs = 8, 4096, 2048, 1000.0
    frame = rng.standard_normal((N, T)).astype(np.float32)
    tau = rng.integers(0, 8901, size=(M, N)) / fs
    plan = dm.Plan(delays_s=tau, n_samples=T, fs=fs, order=3, delay_mode=dm.ROUND,
                   env_cutoff_hz=100.0, env_taps=15)
    assert plan.info().time_tile == 128
    plan.close()
    g = _explicit(frame, tau, fs, 3, dm.ROUND, env_cutoff_hz=100.0, env_taps=15)
    r = oracle.dmas(frame.astype(np.float64), tau, fs, 3, oracle.ROUND, use_cf=True,
                    taps=oracle.fir_taps(fs, 100.0, 15))
    assert_parity(g, r)


@pytest.mark.parametrize("ng", ["cf32", "f64", "f32"])
@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
def test_every_order_linear(order, ng):
    """The interpolated-delay pair kernel (the benchmark's) at every order it
    serves, with each Newton-Girard arithmetic: 1500 samples (ragged last
    tile) x 200 directions (ragged last group)."""
    sc = hemi(1500, 200)
    g = run_gpu(sc, order, dm.LINEAR, ng_prec=ng_prec(ng))
    r = oracle_run(sc, order, oracle.LINEAR)
    assert_parity(g, r)


@pytest.mark.parametrize("ng", ["cf32", "f64", "f32"])
@pytest.mark.parametrize("order", [2, 3, 4, 5, 7])
def test_newton_girard_precisions(ng, order):
    sc = small_2d(1000)
    g = run_gpu(sc, order, dm.ROUND, ng_prec=ng_prec(ng))
    r = oracle_run(sc, order, oracle.ROUND)
    assert_parity(g, r)


def test_microphone_chunks_and_wide_delays():
    sc = passive()  # 100 mics in a 0.4 m square
    plan = gpu_plan(dm, sc, 3, dm.ROUND)
    info = plan.info()
    plan.close()
    assert info.window > 256
    for mode in (dm.ROUND, dm.LINEAR):
        g = run_gpu(sc, 3, mode)
        r = oracle_run(sc, 3, mode)
        assert_parity(g, r)


@pytest.mark.parametrize("mode", ["round", "linear"])
def test_several_staging_passes(mode):
    """Directions spread over the whole field in one group force a wide window,
    so fewer microphones fit per staging pass than the array has; 301
    microphones leave a last pass whose count is not a multiple of 4."""
    rng = np.random.default_rng(9)
    N, T, M, fs = 301, 600, 16, 1000.0
    frame = rng.standard_normal((N, T)).astype(np.float32)
    tau = rng.integers(-60, 61, size=(M, N)) / fs
    if mode == "linear":
        tau = tau + rng.uniform(0.0, 1.0, size=(M, N)) / fs
    dmode, omode = {"round": (dm.ROUND, oracle.ROUND), "linear": (dm.LINEAR, oracle.LINEAR)}[mode]
    plan = dm.Plan(delays_s=tau, n_samples=T, fs=fs, order=3, delay_mode=dmode,
                   env_cutoff_hz=100.0, env_taps=15)
    info = plan.info()
    plan.close()
    assert info.mic_chunk < N and N % info.mic_chunk != 0
    g = _explicit(frame, tau, fs, 3, dmode, env_cutoff_hz=100.0, env_taps=15)
    r = oracle.dmas(frame.astype(np.float64), tau, fs, 3, omode, use_cf=True,
                    taps=oracle.fir_taps(fs, 100.0, 15))
    assert_parity(g, r)


def test_cf_and_envelope_flags():
    sc = small_2d(700)
    for cf in (False, True):
        for env in (False, True):
            g = run_gpu(sc, 4, dm.ROUND, cf=cf, envelope=env)
            r = oracle_run(sc, 4, oracle.ROUND, cf=cf, envelope=env)
            assert eps_peak(g["y"], r["y"]) <= TOL_F32
            if env:
                assert eps_peak(g["img"], r["img"]) <= TOL_F32
            else:
                assert np.array_equal(g["img"], g["y"])


def test_generic_envelope_length():
    sc = small_2d(900)
    g = run_gpu(sc, 3, dm.ROUND, env_cutoff_hz=12000.0, env_taps=45)
    r = oracle_run(sc, 3, oracle.ROUND, env_cutoff_hz=12000.0, env_taps=45)
    assert_parity(g, r)


@pytest.mark.parametrize("T,M,taps", [(6001, 1200, None), (6000, 1201, None), (6004, 1200, 33),
                                     (4096, 300, 209), (4096, 300, 211), (4096, 300, 1023)])
def test_tensor_core_envelope_ragged_tiles(T, M, taps):
    """Frames beyond 2e7 tap products (M T L) take the tensor-core FIR
    (smaller ones the CUDA-core FIR): ragged last row block and time tile,
    T % 4 != 0 (copy fallback) and T % 4 == 0 (TMA), another tap count, the
    longest filter whose Toeplitz block matrix still fits beside four stages
    (209 taps), the shortest that takes the phase arrays instead (211), and the
    longest filter (1023 taps)."""
    sc = hemi(T, M)
    kw = {} if taps is None else {"env_cutoff_hz": 1000.0 if taps > 500 else 20000.0,
                                  "env_taps": taps}
    g = run_gpu(sc, 3, dm.LINEAR, **kw)
    r = oracle_run(sc, 3, oracle.LINEAR, **kw)
    assert_parity(g, r)


# ---------------------------------------------------------------------------
# reduced-precision channels (measured bounds)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("chan,tol", [("f16", 3e-3), ("bf16", 3e-2)])
@pytest.mark.parametrize("order", [3, 5])
def test_reduced_precision_channels(chan, tol, order):
    sc = small_2d()
    cp = {"f16": dm.CH_F16, "bf16": dm.CH_BF16}[chan]
    g = run_gpu(sc, order, dm.ROUND, chan_prec=cp)
    r = oracle_run(sc, order, oracle.ROUND)
    ey, ei = eps_peak(g["y"], r["y"]), eps_peak(g["img"], r["img"])
    print(f"{chan} n={order}: eps_peak y {ey:.3e} img {ei:.3e} "
          f"dB(60) {db_error(g['img'], r['img'])}")
    assert ey <= tol and ei <= tol


# ---------------------------------------------------------------------------
# degenerate inputs
# ---------------------------------------------------------------------------
def _explicit(frame, tau, fs, order, mode=dm.ROUND, **kw):
    N, T = frame.shape
    plan = dm.Plan(delays_s=tau, n_samples=T, fs=fs, order=order, delay_mode=mode, **kw)
    x = torch.from_numpy(np.ascontiguousarray(frame, dtype=np.float32)).cuda()
    y = torch.empty((tau.shape[0], T), device="cuda")
    cf = torch.empty((tau.shape[0], T), device="cuda")
    img = plan(x, y=y, cf=cf)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    return {"img": img.cpu().numpy(), "y": y.cpu().numpy(), "cf": cf.cpu().numpy()}


@pytest.mark.parametrize("ng", ["cf32", "f64"])
@pytest.mark.parametrize("frac", [1e-4, 0.5, 0.9999])
@pytest.mark.parametrize("order", [3, 5])
def test_interpolation_weights_near_the_ends(frac, order, ng):
    """Interpolated delays whose fractions all sit near 0, at 1/2 or near 1: the
    kernel forms the (1 - f)-weighted sums as plain minus f-weighted ones, which
    near f = 1 is a difference of nearly equal sums."""
    rng = np.random.default_rng(int(frac * 1e4) + order)
    N, T, M, fs = 32, 1500, 24, 1000.0
    frame = rng.standard_normal((N, T)).astype(np.float32)
    tau = (rng.integers(-20, 21, size=(M, N)) + frac) / fs
    g = _explicit(frame, tau, fs, order, dm.LINEAR, env_cutoff_hz=100.0, env_taps=15,
                  ng_prec=ng_prec(ng))
    r = oracle.dmas(frame.astype(np.float64), tau, fs, order, oracle.LINEAR, use_cf=True,
                    taps=oracle.fir_taps(fs, 100.0, 15))
    assert_parity(g, r)


@pytest.mark.parametrize("T", [1, 2, 37, 255, 256, 257])
def test_short_frames(T):
    rng = np.random.default_rng(T)
    frame = rng.standard_normal((9, T)).astype(np.float32)
    fs = 1000.0
    tau = rng.integers(-5, 6, size=(11, 9)) / fs
    for mode in (dm.ROUND, dm.LINEAR):
        t = tau + (0.3 / fs if mode == dm.LINEAR else 0.0)
        g = _explicit(frame, t, fs, 3, mode, env_cutoff_hz=100.0, env_taps=9)
        r = oracle.dmas(frame.astype(np.float64), t, fs, 3, mode, use_cf=True,
                        taps=oracle.fir_taps(fs, 100.0, 9))
        assert_parity(g, r)


def test_single_mic_and_single_direction():
    rng = np.random.default_rng(3)
    frame = rng.standard_normal((1, 300)).astype(np.float32)
    tau = np.array([[2.0 / 1000.0]])
    g = _explicit(frame, tau, 1000.0, 1, cf=False, envelope=False)
    want = np.zeros(300, dtype=np.float32)
    want[:298] = frame[0, 2:]
    np.testing.assert_array_equal(g["y"][0], want)
    g2 = _explicit(frame, tau, 1000.0, 2, cf=False, envelope=False)
    assert np.all(np.abs(g2["y"]) <= 1e-6 * np.max(np.abs(frame)))  # E_2 of one value is 0


def test_order_above_mic_count_is_zero():
    rng = np.random.default_rng(4)
    frame = rng.standard_normal((3, 400)).astype(np.float32)
    tau = np.zeros((8, 3))
    g = _explicit(frame, tau, 1000.0, 5, cf=False, envelope=False)
    roots = np.abs(frame.astype(np.float64)) ** 0.2
    scale = np.sum(roots, axis=0) ** 5          # magnitude of the largest NG term
    assert np.all(np.abs(g["y"]) <= 1e-5 * scale[None, :])


def test_zero_frame_and_out_of_range_delays_give_exact_zero():
    frame = np.zeros((6, 500), dtype=np.float32)
    env = dict(env_cutoff_hz=100.0, env_taps=9)
    g = _explicit(frame, np.zeros((10, 6)), 1000.0, 5, **env)
    assert np.all(g["img"] == 0) and np.all(g["y"] == 0) and np.all(g["cf"] == 0)
    rng = np.random.default_rng(5)
    frame = rng.standard_normal((6, 500)).astype(np.float32)
    tau = np.full((10, 6), 900.0 / 1000.0)   # every delayed sample beyond the frame
    g = _explicit(frame, tau, 1000.0, 3, **env)
    assert np.all(g["img"] == 0) and np.all(g["y"] == 0)


def test_sign_flip_is_exact_for_odd_orders():
    sc = small_2d(800)
    plan = gpu_plan(dm, sc, 5, dm.ROUND)
    x = torch.from_numpy(sc.frame).cuda()
    y1 = torch.empty((sc.n_dirs, sc.n_samples), device="cuda")
    y2 = torch.empty_like(y1)
    a = plan(x, y=y1).clone()
    b = plan(-x, y=y2)
    torch.cuda.synchronize()
    plan.close()
    assert torch.equal(y1, -y2)
    assert torch.equal(a, b)


@pytest.mark.parametrize("mode", ["round", "linear"])
def test_image_is_one_homogeneous_in_the_frame(mode):
    """E_n of n-th roots has degree 1 in the samples, CF degree 0 and the
    envelope is linear, so scaling the frame by a scales y and the image by a
    (up to FP32 rounding of the roots)."""
    sc = hemi(1500, 200)
    dmode = dm.LINEAR if mode == "linear" else dm.ROUND
    plan = gpu_plan(dm, sc, 5, dmode)
    x = torch.from_numpy(sc.frame).cuda()
    y1 = torch.empty((sc.n_dirs, sc.n_samples), device="cuda")
    y2 = torch.empty_like(y1)
    a = plan(x, y=y1).cpu().numpy()
    b = plan(3.7 * x, y=y2).cpu().numpy()
    plan.check()
    plan.close()
    assert eps_peak(y2.cpu().numpy(), 3.7 * y1.cpu().numpy()) <= TOL_F32
    assert eps_peak(b, 3.7 * a) <= TOL_F32


def test_microphone_order_does_not_change_the_image():
    """The sums run over the microphones, so listing them in another order
    changes the image only by FP32 rounding."""
    sc = hemi(1500, 200)
    tau = scene_tau(sc)
    perm = np.random.default_rng(3).permutation(sc.mic_xyz.shape[0])
    kw = dict(n_samples=sc.n_samples, fs=sc.fs, c=sc.c, order=5, delay_mode=dm.LINEAR)
    p1 = dm.Plan(delays_s=tau, **kw)
    p2 = dm.Plan(delays_s=np.ascontiguousarray(tau[:, perm]), **kw)
    x = torch.from_numpy(sc.frame).cuda()
    a = p1(x).cpu().numpy()
    b = p2(x[torch.from_numpy(perm).cuda()].contiguous()).cpu().numpy()
    p1.check()
    p2.check()
    p1.close()
    p2.close()
    assert eps_peak(b, a) <= TOL_F32


def test_explicit_delays_equal_geometry():
    sc = small_2d(600)
    tau = scene_tau(sc)
    g1 = run_gpu(sc, 5, dm.ROUND)
    g2 = _explicit(sc.frame, tau, sc.fs, 5)
    np.testing.assert_array_equal(g1["y"], g2["y"])


# ---------------------------------------------------------------------------
# other entry points
# ---------------------------------------------------------------------------
def test_host_buffers_and_batch_equal_device_path():
    sc1, sc2 = small_2d(1000), hemi(1200, 64)
    p1 = gpu_plan(dm, sc1, 5, dm.ROUND)
    p2 = gpu_plan(dm, sc2, 3, dm.LINEAR)
    f1 = torch.from_numpy(sc1.frame).cuda()
    f2 = torch.from_numpy(sc2.frame).cuda()
    a1, a2 = p1(f1).clone(), p2(f2).clone()
    h1 = p1.beamform_host(sc1.frame)
    b1, b2, b3 = dm.beamform_batch([p1, p2, p1], [f1, f2, f1])
    torch.cuda.synchronize()
    assert np.array_equal(h1, a1.cpu().numpy())
    assert torch.equal(b1, a1) and torch.equal(b2, a2) and torch.equal(b3, a1)
    p1.close()
    p2.close()


def sampled_rows_parity(sc, order, gpu_mode, oracle_mode, cf=True, **kw):
    """Whole frame on the GPU in the benchmark's launch configuration; blocks
    of 8 rows sampled across the direction range, plus the rows around the
    image peak, compared with the oracle."""
    plan = gpu_plan(dm, sc, order, gpu_mode, cf=cf, **kw)
    x = torch.from_numpy(sc.frame).cuda()
    y = torch.empty((sc.n_dirs, sc.n_samples), device="cuda")
    img = plan(x, y=y)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    M = sc.n_dirs
    peak_row = int(torch.argmax(torch.amax(torch.abs(y), dim=1)).item())
    last = M - 8
    starts = sorted({0, M // 4 + 5, M // 2, (3 * M) // 4 - 3, last,
                     min(max(peak_row - 4, 0), last)})
    tau = scene_tau(sc)
    peak_y = peak_i = err_y = err_i = 0.0
    for b in starts:
        r = oracle_run(sc, order, oracle_mode, cf=cf, dir_range=(b, b + 8), tau=tau)
        gy, gi = y[b:b + 8].cpu().numpy(), img[b:b + 8].cpu().numpy()
        peak_y = max(peak_y, np.max(np.abs(r["y"])))
        peak_i = max(peak_i, np.max(np.abs(r["img"])))
        err_y = max(err_y, np.max(np.abs(gy - r["y"])))
        err_i = max(err_i, np.max(np.abs(gi - r["img"])))
    assert peak_y > 0 and peak_i > 0
    assert err_y <= TOL_F32 * peak_y, err_y / peak_y
    assert err_i <= TOL_F32 * peak_i, err_i / peak_i


@pytest.mark.parametrize("mode,kw,M", [
    ("linear", {}, 2048),                          # tensor-core envelope
    ("round", {"envelope": False}, 2048),          # image = E_n x CF
    ("round", {"env_taps": 31}, 256),              # CUDA-core envelope
])
def test_host_path_in_time_chunks_equals_device_path(mode, kw, M):
    """dmas_beamform_host runs a large frame in time chunks whose image columns
    download while the next chunk computes; the image is bitwise the device
    path's."""
    sc = scenes.hemi_3d(seed=2, n_dirs=M)
    plan = gpu_plan(dm, sc, 5, dm.LINEAR if mode == "linear" else dm.ROUND, **kw)
    x = torch.from_numpy(sc.frame).cuda()
    ref = plan(x).cpu().numpy()
    got = plan.beamform_host(sc.frame)
    plan.check()
    plan.close()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("ng", ["cf32", "f64"])
def test_full_size_hemisphere_sampled_rows(ng):
    """The timed workload: 2048 directions x 16384 samples, linear delays,
    n = 5, CF, envelope; compensated FP32 (the benchmark's) and FP64
    Newton-Girard."""
    sampled_rows_parity(scenes.hemi_3d(seed=2), 5, dm.LINEAR, oracle.LINEAR,
                        ng_prec=ng_prec(ng))


def test_full_size_hemisphere_nearest_sampled_rows():
    """The same frame with nearest-sample delays (the persistent kernel: 32768
    work items over 4096 CTAs drawing on one counter)."""
    sampled_rows_parity(scenes.hemi_3d(seed=2), 5, dm.ROUND, oracle.ROUND)


def test_full_size_paper_timing_configuration_sampled_rows():
    """The paper's timing configuration: 1000 azimuths x 163840 samples, n = 5
    without CF."""
    sampled_rows_parity(scenes.small_2d(seed=1, n_samples=163840, n_dirs=1000), 5,
                        dm.ROUND, oracle.ROUND, cf=False)


@pytest.mark.parametrize("n_mics,order,mode", [(64, 5, "round"), (64, 3, "linear"),
                                               (256, 5, "round"), (256, 3, "round")])
def test_full_size_passive_sampled_rows(n_mics, order, mode):
    """Passive arrays at full size: N = 64 or 256, 8192 directions x 32768
    samples at 400 kHz (161-tap envelope)."""
    sc = scenes.passive(seed=4, n_mics=n_mics)
    gm, om = (dm.ROUND, oracle.ROUND) if mode == "round" else (dm.LINEAR, oracle.LINEAR)
    sampled_rows_parity(sc, order, gm, om)
