"""The synthetic input recipe that stands in for the paper's cosmological
box, checked against closed forms rather than against its own code: NFW
radii against the enclosed-mass profile M(<r) ~ ln(1+s) - s/(1+s) with
s = r/r_s, r_s = r_200/c and r_200 = (3 M / (800 pi))^(1/3) (200 times the
mean density of the unit box); the 70 / 30 split between halos and the
uniform background; the log-uniform box sizes of the batched workload;
seeding and the value ranges."""
import math

import numpy as np
import pytest

from paper_1211_4406_gb300 import inputs

stats = pytest.importorskip("scipy.stats")


def _nfw_cdf(s, c):
    mu = lambda t: np.log1p(t) - t / (1.0 + t)
    return mu(np.minimum(s, c)) / mu(c)


def _halo_radii(pos):
    """Minimum-image distances from the circular-mean centre of a compact halo."""
    ang = 2.0 * np.pi * pos
    centre = (np.arctan2(np.sin(ang).mean(0), np.cos(ang).mean(0)) / (2.0 * np.pi)) % 1.0
    d = pos - centre
    d -= np.round(d)
    return np.linalg.norm(d, axis=1)


def test_single_halo_follows_the_nfw_profile():
    n, conc = 40000, 10.0
    pos, mass = inputs.clustered_box(n, 1, seed=5, frac=1.0, conc=conc)
    r200 = (3.0 * 1.0 / (800.0 * math.pi)) ** (1.0 / 3.0)   # the whole box mass in the halo
    r = _halo_radii(pos)
    # truncated at r_200 (up to the centre estimate's error, ~ r_200 / sqrt(n))
    assert r.max() <= r200 * (1 + 0.01)
    s = r / (r200 / conc)
    d, p = stats.kstest(s, lambda x: _nfw_cdf(np.asarray(x), conc))
    assert d < 0.012, (d, p)
    # the half-mass radius of a c = 10 NFW halo, solved from the closed form
    from scipy.optimize import brentq
    s_half = brentq(lambda t: _nfw_cdf(np.array(t), conc) - 0.5, 1e-6, conc)
    assert abs(np.median(s) / s_half - 1.0) < 0.02, (np.median(s), s_half)


def test_seventy_percent_of_particles_are_in_the_halo():
    n = 50000
    pos, _ = inputs.clustered_box(n, 1, seed=9)               # frac = 0.7 by default
    r200 = (3.0 * 0.7 / (800.0 * math.pi)) ** (1.0 / 3.0)     # the halo holds 0.7 of the mass
    # the circular mean is pulled towards the box centre by the background:
    # find the halo centre from the densest particles instead
    r_all = _halo_radii(pos)
    core = pos[np.argsort(r_all)[: n // 10]]
    ang = 2.0 * np.pi * core
    centre = (np.arctan2(np.sin(ang).mean(0), np.cos(ang).mean(0)) / (2.0 * np.pi)) % 1.0
    d = pos - centre
    d -= np.round(d)
    inside = np.linalg.norm(d, axis=1) <= r200 * (1 + 1e-6)
    expect = 0.7 + 0.3 * (4.0 / 3.0) * math.pi * r200 ** 3    # halo + background in that sphere
    sigma = math.sqrt(0.3 * n * (4.0 / 3.0) * math.pi * r200 ** 3) / n + 1e-4
    assert abs(inside.mean() - expect) < 5 * sigma + 2e-4, (inside.mean(), expect)


def test_boxes_are_seeded_and_in_range():
    a, ma = inputs.clustered_box(4096, 12, seed=71)
    b, mb = inputs.clustered_box(4096, 12, seed=71)
    c, _ = inputs.clustered_box(4096, 12, seed=72)
    assert np.array_equal(a, b) and np.array_equal(ma, mb) and not np.array_equal(a, c)
    assert a.dtype == np.float64 and a.shape == (4096, 3) and a.min() >= 0.0 and a.max() < 1.0
    assert np.all(ma == 1.0 / 4096)
    u, mu = inputs.uniform_box(8192, 3)
    assert u.min() >= 0.0 and u.max() < 1.0 and np.all(mu == 1.0 / 8192)
    assert np.allclose(u.mean(0), 0.5, atol=0.02) and np.allclose(u.var(0), 1.0 / 12.0, atol=0.01)
    w = inputs.cotangent(1000, 4)
    assert w.dtype == np.float32 and w.shape == (1000, 3) and np.array_equal(w, inputs.cotangent(1000, 4))


def test_input_order_carries_no_spatial_structure():
    pos, _ = inputs.clustered_box(20000, 50, seed=13)
    # consecutive particles are no closer than random pairs
    d = pos[1:] - pos[:-1]
    d -= np.round(d)
    mean_step = np.linalg.norm(d, axis=1).mean()
    rng = np.random.default_rng(0)
    i, j = rng.integers(0, len(pos), (2, 20000))
    e = pos[i] - pos[j]
    e -= np.round(e)
    assert abs(mean_step / np.linalg.norm(e, axis=1).mean() - 1.0) < 0.03


def test_batched_sizes_are_log_uniform_in_range():
    sizes = np.asarray(inputs.batched_sizes(64))
    lo, hi = 16 ** 3, 96 ** 3
    assert sizes.size == 64 and sizes.min() >= lo and sizes.max() <= hi
    x = (np.log(sizes) - math.log(lo)) / (math.log(hi) - math.log(lo))
    assert stats.kstest(x, "uniform").pvalue > 1e-3
