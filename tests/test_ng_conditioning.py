"""Why the Newton-Girard step needs more than FP32 (Sec. II-C, Eqs.
dmas2_impl..dmas5_impl): the pre-expanded equations are alternating sums whose
terms can exceed E_n by many orders of magnitude, so evaluating them in FP32
loses digits even when the power sums themselves are exact.  These CPU tests pin that reading on a set of 32 roots (signed
powers of two, so every power sum is exact in FP32) against the oracle's
E_n, which expands the product of Eq. dmasn with no cancellation."""
import numpy as np

import oracle

# 32 signed powers of two: E_5 = 480, terms of Eq. dmas5_impl up to 9.2e9
ROOTS = [4, -8, 4, -4, -2, -4, -16, -16, -4, 16, 8, 1, 8, 8, 0, 8, 0, 8, 2, -4, -2, 0, 2, 0,
         -8, -16, -16, -16, 1, -16, 8, -16]


def _power_sums(r, n):
    return [0.0] + [float(np.sum(np.asarray(r, dtype=np.float64) ** k)) for k in range(1, n + 1)]


def _eq_dmas5_terms(P, dtype):
    """The seven terms of Eq. dmas5_impl (times 120) in the given precision."""
    p1, p2, p3, p4, p5 = (dtype(v) for v in P[1:6])
    return [p1 ** 5, -dtype(10) * p1 ** 3 * p2, dtype(15) * p1 * p2 ** 2,
            dtype(20) * p1 ** 2 * p3, -dtype(20) * p2 * p3, -dtype(30) * p1 * p4,
            dtype(24) * p5]


def test_power_sums_are_exact_in_fp32():
    P = _power_sums(ROOTS, 5)
    for k in range(1, 6):
        assert float(np.float32(P[k])) == P[k]


def test_oracle_e5_of_the_set():
    assert oracle.esym_product(np.asarray(ROOTS, dtype=np.float64), 5) == 480.0
    # the oracle's FP64 Newton-Girard: the cancellation costs FP64 digits too,
    # far below the gate
    assert abs(oracle.esym_newton_girard(_power_sums(ROOTS, 5), 5) - 480.0) <= 1e-9 * 480.0


def test_fp32_evaluation_misses_the_gate_fp64_meets_it():
    P = _power_sums(ROOTS, 5)
    t64 = _eq_dmas5_terms(P, np.float64)
    assert max(abs(v) for v in t64) > 9e9            # terms ~1.9e7 times E_5
    e64 = float(sum(t64)) / 120.0
    assert abs(e64 - 480.0) <= 1e-5 * 480.0
    acc = np.float32(0.0)
    for v in _eq_dmas5_terms(P, np.float32):
        acc = np.float32(acc + v)
    e32 = float(acc) / 120.0
    assert abs(e32 - 480.0) > 1e-3 * 480.0           # FP32 alone: the gate is missed
