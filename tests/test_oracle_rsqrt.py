"""Pins of the oracle's version of the paper's inverse square root (Sec. II-A:
an estimate y0 of 1/sqrt(x) refined by h0 = 1 - x y0^2,
y1 = y0 (1 + h0/2 + 3 h0^2/8)): the step against its exact error polynomial,
the estimate and the refined value against their error bounds over many
binades, and the force variant against the exact-root force."""
import numpy as np

import oracle


def test_third_order_step_has_the_exact_error_polynomial():
    # y0 = (1 + e)/sqrt(x) gives y1 sqrt(x) - 1 = 5/2 e^3 + 15/8 e^4 + 3/8 e^5 exactly
    for x in (4.0, 0.25, 1.0, 64.0):
        r = 1.0 / np.sqrt(x)
        for e in (-2.7e-2, -1e-2, -3e-3, -1e-3, 1e-3, 3e-3, 1e-2, 2.7e-2):
            y1 = oracle.rsqrt_third_order(x, (1.0 + e) * r)
            want = 2.5 * e ** 3 + 1.875 * e ** 4 + 0.375 * e ** 5
            assert abs(y1 / r - 1.0 - want) <= 4e-16 + 1e-9 * abs(want), (x, e, y1 / r - 1.0, want)


def test_estimate_and_refinement_error_bounds_over_many_binades():
    rng = np.random.default_rng(3)
    xs = np.concatenate([np.logspace(-30, 30, 2001), rng.uniform(0.5, 2.0, 5000) * 2.0 ** rng.integers(-60, 60, 5000)])
    e0 = np.array([oracle.rsqrt_seed(x) * np.sqrt(x) - 1.0 for x in xs])
    e1 = np.array([oracle.rsqrt_refined(x) * np.sqrt(x) - 1.0 for x in xs])
    assert np.abs(e0).max() <= 1.8e-3, np.abs(e0).max()
    assert np.abs(e0).max() >= 1e-3                      # the estimate alone is ~9 bits, not full precision
    assert np.abs(e1).max() <= 1.5e-8, np.abs(e1).max()
    # the step turns e into 5/2 e^3 + O(e^4): the refined errors follow the estimate's
    assert np.allclose(e1, 2.5 * e0 ** 3, rtol=0.02, atol=1e-15)


def test_force_variant_stays_within_the_refinement_error():
    rng = np.random.default_rng(5)
    G, eps, rc = 1.0, 1e-3, 0.1
    worst, moved = 0.0, 0
    for _ in range(500):
        d = rng.uniform(-0.06, 0.06, 3)
        a = oracle.pair(d, 0.7, G, eps, rc)
        b = oracle.pair(d, 0.7, G, eps, rc, rsqrt_refined=True)
        if np.linalg.norm(a) > 0:
            rel = np.linalg.norm(b - a) / np.linalg.norm(a)
            worst = max(worst, rel)
            moved += rel > 0
    assert worst <= 4.5e-8 and moved > 100
