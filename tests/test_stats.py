"""Reporting helpers pinned to independent references (CPU): the Wilson interval that the FER
parity tests accept against, the FER-ratio interval, and the stabilizer test of the Monte
Carlo protocol."""
import math

import numpy as np
import pytest

from paper_2605_10433_gb300.stats import log_ratio_interval, logical_ok, wilson_interval


@pytest.mark.parametrize("k,n", [(0, 10), (1, 10), (5, 10), (10, 10), (3, 1_000_000), (31, 8_388_608),
                                 (4117, 100_000), (999_999, 1_000_000)])
def test_wilson_interval_matches_scipy(k, n):
    stats = pytest.importorskip("scipy.stats")
    ci = stats.binomtest(k, n).proportion_ci(confidence_level=0.95, method="wilson")
    lo, hi = wilson_interval(k, n)
    assert abs(lo - ci.low) < 1e-12 and abs(hi - ci.high) < 1e-12


def test_wilson_interval_edges():
    assert wilson_interval(0, 0) == (0.0, 1.0)
    lo, hi = wilson_interval(0, 100)
    assert abs(lo) < 1e-15 and 0 < hi < 0.05           # no failures: an upper bound only
    lo, hi = wilson_interval(100, 100)
    assert abs(hi - 1.0) < 1e-15 and 0.95 < lo < 1
    lo, hi = wilson_interval(50, 100)
    assert abs((lo + hi) / 2 - 0.5) < 1e-15             # symmetric at one half


def test_log_ratio_interval():
    lo, hi = log_ratio_interval(100, 10_000, 100, 10_000)
    assert abs(math.log(lo) + math.log(hi)) < 1e-12     # equal rates: symmetric about ratio 1 in log
    se = math.sqrt(2 * (1 / 100 - 1 / 10_000))
    assert abs(hi - math.exp(1.959963984540054 * se)) < 1e-12
    lo, hi = log_ratio_interval(50, 10_000, 200, 10_000)
    assert lo < 0.25 < hi                                # contains the point ratio
    assert log_ratio_interval(0, 10, 5, 10) == (0.0, math.inf)


def test_logical_ok_on_the_steane_code():
    """H_Z = the Hamming(7,4) checks: residuals in their row space (the [7,3] simplex code:
    weights 0 and 4) are stabilizers; a single flip or the all-ones vector is not."""
    rows = [[3, 4, 5, 6], [1, 2, 5, 6], [0, 2, 4, 6]]
    hz = [sum(1 << j for j in r) for r in rows]
    R = np.zeros((6, 7), dtype=np.uint8)
    R[1, rows[0]] = 1                                   # a stabilizer
    R[2, rows[0]] ^= 1
    R[2, rows[1]] ^= 1                                  # a sum of two
    R[3, 2] = 1                                         # one flip
    R[4, :] = 1                                         # all ones (weight 7)
    R[5, rows[2]] = 1
    R[5, 0] ^= 1                                        # a stabilizer plus one flip
    assert logical_ok(hz, R).tolist() == [True, True, True, False, False, False]


def test_mcnemar_exact_p_matches_the_binomial_test():
    """The paired FER check's exact McNemar p-value equals scipy's two-sided binomial test of the
    discordant shots at 1/2."""
    scipy_stats = pytest.importorskip("scipy.stats")
    import numpy as np
    from tests.gpu_helpers import mcnemar_p
    rng = np.random.default_rng(3)
    for b, c in [(0, 0), (0, 1), (5, 0), (3, 9), (17, 11), (40, 70)]:
        conv_g = np.ones(200, dtype=np.uint8)
        conv_o = np.ones(200, dtype=np.uint8)
        idx = rng.permutation(200)
        conv_g[idx[:b]] = 0                    # GPU-only failures
        conv_o[idx[b:b + c]] = 0               # oracle-only failures
        conv_g[idx[b + c:b + c + 7]] = 0       # shared failures: not discordant
        conv_o[idx[b + c:b + c + 7]] = 0
        want = 1.0 if b + c == 0 else scipy_stats.binomtest(min(b, c), b + c, 0.5).pvalue
        assert abs(mcnemar_p(conv_g, conv_o) - min(1.0, want)) < 1e-12
