"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here calls the CUDA library.  Each test checks the oracle against an
independent source: brute-force subset sums (Eq. dmasn), the pairwise DMAS of
Eq. dmas, the paper's pre-expanded Newton-Girard equations (Eqs. dmas2_impl to
dmas5_impl, transcribed in tests/golden), a hand-worked example, closed forms
and invariances.  The tests are sized so that a dropped term, a wrong sign, a
wrong index or a transposed operand in the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from workloads import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_esym(r, n):
    """Eq. dmasn: sum over all n-subsets of the product of their members."""
    return math.fsum(math.prod(c) for c in itertools.combinations(list(r), n))


def signed_root_np(x, n):
    return np.sign(x) * np.abs(x) ** (1.0 / n)


def load_expansions():
    terms = {}
    with open(os.path.join(GOLDEN, "ng_expansions.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x) for x in line.split()]
            n, den, coef, expo = v[0], v[1], v[2], v[3:]
            assert len(expo) == n
            terms.setdefault(n, []).append((den, coef, expo))
    return terms


def eval_expansion(terms, P):
    den = terms[0][0]
    acc = 0.0
    for d, coef, expo in terms:
        assert d == den
        acc += coef * math.prod(P[k + 1] ** e for k, e in enumerate(expo))
    return acc / den


def delayed(frame, shifts):
    """x[i][t] = frame[i][t + shifts[i]], zero outside the frame (numpy slicing)."""
    N, T = frame.shape
    x = np.zeros_like(frame, dtype=np.float64)
    for i in range(N):
        s = int(shifts[i])
        if s >= 0:
            if s < T:
                x[i, :T - s] = frame[i, s:]
        else:
            if -s < T:
                x[i, -s:] = frame[i, :T + s]
    return x


# ---------------------------------------------------------------------------
# elementary symmetric polynomials
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 5, 7, 10])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_product_form_equals_subset_sums(N, n):
    rng = np.random.default_rng(100 + 10 * N + n)
    for _ in range(5):
        r = rng.standard_normal(N) * rng.choice([1e-3, 1.0, 30.0])
        want = brute_esym(r, n) if n <= N else 0.0
        got = oracle.esym_product(r, n)
        scale = brute_esym(np.abs(r), n) if n <= N else 1.0
        assert abs(got - want) <= 1e-12 * max(scale, 1e-300)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_partition_formula_equals_paper_expansions(n):
    terms = load_expansions()[n]
    rng = np.random.default_rng(7 + n)
    for _ in range(20):
        P = np.concatenate([[0.0], rng.standard_normal(n) * 3.0])
        want = eval_expansion(terms, P)
        got = oracle.esym_newton_girard(P, n)
        scale = sum(abs(c) * math.prod(abs(P[k + 1]) ** e for k, e in enumerate(x))
                    for _, c, x in terms) / terms[0][0]
        assert abs(got - want) <= 1e-13 * scale


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_partition_formula_equals_subset_sums(n):
    rng = np.random.default_rng(50 + n)
    for N in (n, n + 1, 9):
        r = rng.standard_normal(N)
        P = np.array([0.0] + [np.sum(r ** k) for k in range(1, n + 1)])
        want = brute_esym(r, n)
        got = oracle.esym_newton_girard(P, n)
        assert abs(got - want) <= 1e-10 * max(1.0, brute_esym(np.abs(r), n))


def test_hand_worked_example():
    with open(os.path.join(GOLDEN, "hand_example.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    vals = np.array([float(x) for x in rows[0]])
    E = [float(x) for x in rows[1]]
    P = [0.0] + [float(x) for x in rows[2]]
    for n in range(1, 5):
        assert oracle.esym_product(vals, n) == E[n - 1]
        assert abs(oracle.esym_newton_girard(np.array(P), n) - E[n - 1]) < 1e-9
    # the power sums in the file are the values' own
    for k in range(1, 5):
        assert np.sum(vals ** k) == P[k]


def test_fewer_than_n_nonzero_is_exactly_zero():
    r = np.zeros(12)
    r[[2, 7]] = [1.7, -0.3]
    for n in (3, 4, 5):
        assert oracle.esym_product(r, n) == 0.0
        P = np.array([0.0] + [np.sum(r ** k) for k in range(1, n + 1)])
        assert abs(oracle.esym_newton_girard(P, n)) < 1e-15


def test_signed_root_closed_forms():
    assert oracle.signed_root(-8.0, 3) == pytest.approx(-2.0, rel=1e-15)
    assert oracle.signed_root(16.0, 4) == pytest.approx(2.0, rel=1e-15)
    assert oracle.signed_root(-16.0, 4) == pytest.approx(-2.0, rel=1e-15)
    assert oracle.signed_root(0.0, 5) == 0.0
    assert oracle.signed_root(-0.0, 5) == 0.0
    assert oracle.signed_root(-0.37, 1) == -0.37
    assert oracle.signed_root(32.0, 5) == pytest.approx(2.0, rel=1e-15)


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
def test_unit_vectors_axes():
    azel = np.deg2rad([[0.0, 0.0], [90.0, 0.0], [-90.0, 0.0], [0.0, 90.0], [30.0, 20.0]])
    u = oracle.unit_vectors(azel)
    np.testing.assert_allclose(u[0], [0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(u[1], [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(u[2], [-1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(u[3], [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-15)
    th, ph = np.deg2rad(30.0), np.deg2rad(20.0)
    np.testing.assert_allclose(u[4], [np.sin(th) * np.cos(ph), np.sin(ph),
                                      np.cos(th) * np.cos(ph)], atol=1e-15)


def test_delays_broadside_and_endfire():
    rng = np.random.default_rng(3)
    mic = scenes.disc_array(rng, 16, 0.06)
    u = oracle.unit_vectors(np.deg2rad([[0.0, 0.0], [90.0, 0.0], [0.0, 90.0]]))
    tau = oracle.geometric_delays(mic, u, 343.0)
    assert np.all(tau[0] == 0.0)
    cen = mic.mean(axis=0)
    np.testing.assert_allclose(tau[1], -(mic[:, 0] - cen[0]) / 343.0, atol=1e-18)
    np.testing.assert_allclose(tau[2], -(mic[:, 1] - cen[1]) / 343.0, atol=1e-18)
    # centroid reference: delays over the array sum to zero
    assert abs(tau[1].sum()) < 1e-17


def test_round_shift_half_away_from_zero():
    fs = 1024.0
    taus = np.array([2.5, -2.5, 0.49 / fs * fs, 1.5]) / fs
    assert list(oracle.round_shifts(taus, fs)) == [3, -3, 0, 2]


@pytest.mark.parametrize("az_true", [-41.0, 0.0, 30.0])
def test_plane_wave_peaks_at_its_azimuth(az_true):
    """A wrong delay sign would put the peak at -az_true."""
    sc = scenes.plane_wave(24, 2048, az_true)
    u = oracle.unit_vectors(sc.dir_azel)
    tau = oracle.geometric_delays(sc.mic_xyz, u, sc.c)
    out = oracle.dmas(sc.frame, tau, sc.fs, 1, use_cf=False)
    peak_dir = np.argmax(np.max(np.abs(out["y"]), axis=1))
    assert abs(np.rad2deg(sc.dir_azel[peak_dir, 0]) - az_true) <= 1.0


# ---------------------------------------------------------------------------
# the beamformer against definitions
# ---------------------------------------------------------------------------
def _tiny_case(seed, N, T, M, span, fs=1000.0):
    rng = np.random.default_rng(seed)
    frame = rng.standard_normal((N, T))
    frame[rng.random((N, T)) < 0.05] = 0.0
    shifts = rng.integers(-span, span + 1, size=(M, N))
    tau = shifts / fs
    return frame, shifts, tau, fs


def test_order1_is_delay_and_sum():
    frame, shifts, tau, fs = _tiny_case(11, 9, 64, 5, 7)
    out = oracle.dmas(frame, tau, fs, 1, use_cf=False)
    for p in range(5):
        x = delayed(frame, shifts[p])
        np.testing.assert_allclose(out["y"][p], x.sum(axis=0), rtol=0, atol=1e-12)


def test_round_mode_takes_the_nearest_sample():
    """Fractional delays in ROUND mode pick the nearest sample (half away from 0)."""
    frame, shifts, tau, fs = _tiny_case(13, 8, 50, 4, 6, fs=1024.0)
    frac = np.random.default_rng(5).uniform(-0.45, 0.45, size=shifts.shape)
    frac[0, :4] = [0.5, -0.5, 0.49, -0.49]
    tot = shifts + frac
    # nearest integer, exact halves away from zero (only the +-0.5 entries differ
    # from shifts)
    want_shift = (np.sign(tot) * np.floor(np.abs(tot) + 0.5)).astype(int)
    out = oracle.dmas(frame, tot / fs, fs, 1, use_cf=False)
    for p in range(4):
        x = delayed(frame, want_shift[p])
        np.testing.assert_allclose(out["y"][p], x.sum(axis=0), rtol=0, atol=1e-12)


def test_order2_is_pairwise_dmas():
    frame, shifts, tau, fs = _tiny_case(12, 7, 40, 4, 5)
    out = oracle.dmas(frame, tau, fs, 2, use_cf=False)
    for p in range(4):
        x = delayed(frame, shifts[p])
        want = np.zeros(frame.shape[1])
        for i in range(7):
            for j in range(i + 1, 7):
                prod = x[i] * x[j]
                want += np.sign(prod) * np.sqrt(np.abs(prod))
        np.testing.assert_allclose(out["y"][p], want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_higher_order_brute_force_with_cf(n):
    N, T, M = 8, 24, 3
    frame, shifts, tau, fs = _tiny_case(20 + n, N, T, M, 4)
    eps = 1e-30
    out = oracle.dmas(frame, tau, fs, n, use_cf=True, cf_eps=eps)
    for p in range(M):
        x = delayed(frame, shifts[p])
        r = signed_root_np(x, n)
        for t in range(T):
            E = brute_esym(r[:, t], n)
            cf = x[:, t].sum() ** 2 / (N * np.sum(x[:, t] ** 2) + eps)
            assert abs(out["cf"][p, t] - cf) <= 1e-13 * max(1.0, cf)
            assert abs(out["y"][p, t] - E * cf) <= 1e-11 * max(
                1.0, brute_esym(np.abs(r[:, t]), n))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_all_equal_closed_form(n):
    """All delayed samples equal s: E_n = C(N,n) sgn(s)^n |s|, CF ~ 1."""
    N, T = 32, 50
    s = np.linspace(-2.0, 2.0, T)
    frame = np.tile(s, (N, 1))
    tau = np.zeros((2, N))
    out = oracle.dmas(frame, tau, 1000.0, n, use_cf=False)
    want = math.comb(N, n) * np.sign(s) ** n * np.abs(s)
    np.testing.assert_allclose(out["y"][0], want, rtol=1e-12, atol=1e-300)
    outcf = oracle.dmas(frame, tau, 1000.0, n, use_cf=True)
    nz = s != 0
    np.testing.assert_allclose(outcf["cf"][0][nz], 1.0, rtol=1e-14)


def test_cf_bounds_and_single_active_mic():
    frame, shifts, tau, fs = _tiny_case(30, 10, 80, 6, 9)
    out = oracle.dmas(frame, tau, fs, 3, use_cf=True)
    assert np.all(out["cf"] >= 0.0) and np.all(out["cf"] <= 1.0 + 1e-15)
    single = np.zeros((10, 30))
    single[4] = np.linspace(0.1, 3.0, 30)
    o2 = oracle.dmas(single, np.zeros((1, 10)), fs, 3, use_cf=True)
    np.testing.assert_allclose(o2["cf"][0], 0.1, rtol=1e-14)
    z = oracle.dmas(np.zeros((10, 30)), np.zeros((1, 10)), fs, 3, use_cf=True)
    assert np.all(z["cf"] == 0.0) and np.all(z["y"] == 0.0)


def test_invariances():
    frame, shifts, tau, fs = _tiny_case(40, 9, 70, 4, 6)
    taps = oracle.fir_taps(1000.0, 50.0, 21)
    for n in (2, 3, 5):
        base = oracle.dmas(frame, tau, fs, n, use_cf=True, taps=taps)
        perm = np.random.default_rng(n).permutation(9)
        pm = oracle.dmas(frame[perm], tau[:, perm], fs, n, use_cf=True, taps=taps)
        np.testing.assert_allclose(pm["y"], base["y"], rtol=1e-11, atol=1e-11)
        alpha = 3.7
        sc = oracle.dmas(alpha * frame, tau, fs, n, use_cf=True, taps=taps)
        np.testing.assert_allclose(sc["y"], alpha * base["y"], rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(sc["img"], alpha * base["img"], rtol=1e-11, atol=1e-11)
        fl = oracle.dmas(-frame, tau, fs, n, use_cf=True, taps=taps)
        np.testing.assert_allclose(fl["y"], (-1) ** n * base["y"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(fl["img"], base["img"], rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# linear interpolation of every channel
# ---------------------------------------------------------------------------
def test_linear_with_integer_delays_equals_round():
    frame, shifts, tau, fs = _tiny_case(50, 8, 60, 4, 5, fs=1024.0)
    for n in (1, 3, 5):
        a = oracle.dmas(frame, tau, fs, n, delay_mode=oracle.ROUND)
        b = oracle.dmas(frame, tau, fs, n, delay_mode=oracle.LINEAR)
        scale = np.max(np.abs(a["y"]))
        np.testing.assert_allclose(b["y"], a["y"], rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(b["cf"], a["cf"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_linear_against_interpolated_power_sums(n):
    rng = np.random.default_rng(60 + n)
    N, T, M, fs = 7, 48, 3, 1000.0
    frame = rng.standard_normal((N, T))
    tau = rng.uniform(-6.0, 6.0, size=(M, N)) / fs
    out = oracle.dmas(frame, tau, fs, n, delay_mode=oracle.LINEAR, use_cf=True)
    terms = load_expansions()[n]
    r = signed_root_np(frame, n)
    for p in range(M):
        delta = tau[p] * fs
        j = np.floor(delta).astype(int)
        f = delta - j
        for t in range(T):
            P = [0.0] * (n + 1)
            A = B = 0.0
            for i in range(N):
                def at(v, s):
                    return v[i, s] if 0 <= s < T else 0.0
                s0 = t + j[i]
                for k in range(1, n + 1):
                    P[k] += (1 - f[i]) * at(r ** k, s0) + f[i] * at(r ** k, s0 + 1)
                A += (1 - f[i]) * at(frame, s0) + f[i] * at(frame, s0 + 1)
                B += (1 - f[i]) * at(frame ** 2, s0) + f[i] * at(frame ** 2, s0 + 1)
            E = eval_expansion(terms, P)
            cf = A * A / (N * B + 1e-30)
            assert abs(out["y"][p, t] - E * cf) <= 1e-10 * max(1.0, abs(E))
            assert cf <= 1.0 + 1e-12


def test_linear_constant_signal_closed_form():
    """Interpolating constant channels is exact: E_n = C(N,n) s for odd n."""
    N, T, fs = 12, 80, 1000.0
    frame = np.full((N, T), 0.8)
    tau = np.random.default_rng(1).uniform(-3.0, 3.0, size=(2, N)) / fs
    for n in (3, 5):
        out = oracle.dmas(frame, tau, fs, n, delay_mode=oracle.LINEAR, use_cf=True)
        inner = slice(8, T - 8)
        np.testing.assert_allclose(out["y"][:, inner], math.comb(N, n) * 0.8, rtol=1e-12)
        np.testing.assert_allclose(out["cf"][:, inner], 1.0, rtol=1e-13)


def test_linear_fp64_against_long_double():
    sc = scenes.small_2d(seed=1, n_samples=512)
    u = oracle.unit_vectors(sc.dir_azel)
    tau = oracle.geometric_delays(sc.mic_xyz, u, sc.c) * 1.0001  # force fractions
    frame = sc.frame.astype(np.float64)
    out = oracle.dmas(frame, tau, sc.fs, 5, delay_mode=oracle.LINEAR, use_cf=False,
                      dir_range=(40, 45))
    peak = np.max(np.abs(out["y"]))
    for p in range(5):
        for t in range(0, 512, 37):
            ld = oracle.linear_esym_ld(frame, tau[40 + p], sc.fs, 5, t)
            assert abs(out["y"][p, t] - ld) <= 1e-12 * peak


# ---------------------------------------------------------------------------
# envelope low-pass
# ---------------------------------------------------------------------------
def test_fir_design():
    fs, fc = 450e3, 5e3
    L = oracle.fir_length(fs, fc)
    assert L == 181
    assert oracle.fir_length(400e3, 5e3) == 161
    h = oracle.fir_taps(fs, fc)
    assert abs(h.sum() - 1.0) < 1e-14
    np.testing.assert_allclose(h, h[::-1], rtol=0, atol=1e-18)
    k = np.arange(L) - (L - 1) // 2

    def gain(f):
        return abs(np.sum(h * np.exp(-2j * np.pi * f * k / fs)))

    assert abs(gain(0.0) - 1.0) < 1e-14
    assert abs(gain(fc) - 0.5) < 0.02          # windowed-sinc cutoff is the -6 dB point
    assert gain(20e3) < 10 ** (-50 / 20)       # Hamming stop band
    assert gain(40e3) < 10 ** (-50 / 20)       # the echo carrier is removed


def test_envelope_impulse_constant_and_ends():
    h = oracle.fir_taps(450e3, 5e3)
    L, H, T = h.size, (h.size - 1) // 2, 600
    y = np.zeros(T)
    y[300] = -1.0  # |y| is filtered
    env = oracle.envelope(y, h)
    np.testing.assert_allclose(env[300 - H:300 + H + 1], h, rtol=0, atol=1e-17)
    assert np.all(env[:300 - H] == 0.0) and np.all(env[300 + H + 1:] == 0.0)
    c = oracle.envelope(np.full(T, 2.0), h)
    np.testing.assert_allclose(c[H:T - H], 2.0, rtol=1e-14)
    assert abs(c[0] - 2.0 * h[H:].sum()) < 1e-14


def test_dmas_envelope_matches_separate_envelope():
    frame, shifts, tau, fs = _tiny_case(70, 6, 90, 3, 4)
    h = oracle.fir_taps(1000.0, 40.0, 15)
    out = oracle.dmas(frame, tau, fs, 3, use_cf=True, taps=h)
    np.testing.assert_allclose(out["img"], oracle.envelope(out["y"], h), rtol=0, atol=0)


# ---------------------------------------------------------------------------
# matched filter (Sec. II step 1): mf[t] = sum_k e[k] m[t + k]
# ---------------------------------------------------------------------------
def test_matched_filter_impulse_response_is_the_reversed_signal():
    rng = np.random.default_rng(31)
    e = rng.standard_normal(37)
    T, t0 = 200, 120
    frame = np.zeros((1, T))
    frame[0, t0] = 1.0
    mf = oracle.matched_filter(frame, e)[0]
    want = np.zeros(T)
    for t in range(t0 - e.size + 1, t0 + 1):
        want[t] = e[t0 - t]
    assert np.array_equal(mf, want)


def test_matched_filter_equals_numpy_correlate():
    rng = np.random.default_rng(32)
    frame = rng.standard_normal((3, 500))
    e = rng.standard_normal(61)
    mf = oracle.matched_filter(frame, e)
    for i in range(3):
        full = np.correlate(frame[i], e, "full")
        assert np.allclose(mf[i], full[e.size - 1:e.size - 1 + frame.shape[1]],
                           rtol=1e-12, atol=1e-12)


def test_matched_filter_linear_and_zero_past_the_frame():
    rng = np.random.default_rng(33)
    a, b = rng.standard_normal((2, 1, 300))
    e = rng.standard_normal(45)
    lhs = oracle.matched_filter(2.0 * a - 0.5 * b, e)
    rhs = 2.0 * oracle.matched_filter(a, e) - 0.5 * oracle.matched_filter(b, e)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    mf = oracle.matched_filter(a, e)[0]
    assert mf[-1] == e[0] * a[0, -1]
    assert np.isclose(mf[-3], e[0] * a[0, -3] + e[1] * a[0, -2] + e[2] * a[0, -1], rtol=1e-14)


def test_matched_filter_compresses_the_chirp_echo():
    """A chirp echo arriving at t0 peaks at t0 after the matched filter."""
    fs = 450e3
    e = scenes.lfm_chirp(fs)
    T, t0 = 4096, 1500
    frame = np.zeros((1, T))
    frame[0, t0:t0 + e.size] = e
    mf = oracle.matched_filter(frame, e)[0]
    assert int(np.argmax(mf)) == t0
    assert np.isclose(mf[t0], float(np.sum(e * e)), rtol=1e-12)
