"""Pins of the oracle's cutoff function (Eq. 3) and pair term (Eq. 2).

Independent pins: the force between two S2 clouds (the PM density of Eq. 1)
computed by a Fourier integral, which Eq. 3 must reproduce as
g = 1 - r^2 F_S2S2 / (G m^2); exact rational values of the printed formula;
factored closed forms; smoothness; numerical derivatives.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.integrate import quad

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def s2_hat(k, a=1.0):
    """Fourier transform of the unit-mass S2 cloud of radius a (Eq. 1)."""
    x = k * a
    if x < 0.2:
        return 1 - x ** 2 / 15 + x ** 4 / 560 - x ** 6 / 37800
    return 12.0 / x ** 4 * (2 - 2 * np.cos(x) - x * np.sin(x))


def s2_hat_by_quadrature(k, a=1.0):
    rho = lambda r: 3 / (np.pi * a ** 3) * (1 - r / a)          # Eq. 1, m = 1
    return 4 * np.pi / k * quad(lambda r: r * rho(r) * np.sin(k * r), 0, a,
                                epsabs=1e-14, epsrel=1e-13)[0]


def cloud_force(r, a=1.0):
    """Attractive force between two unit-mass S2 clouds of radius a at
    separation r (G = 1): F = (2/pi) int S^2 [sin(kr)/(kr^2) - cos(kr)/r] dk."""
    f = lambda k: s2_hat(k, a) ** 2 * (np.sin(k * r) / (k * r * r) - np.cos(k * r) / r)
    edges = np.linspace(0.0, 400.0 / a, 201)
    tot = sum(quad(f, lo, hi, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
              for lo, hi in zip(edges[:-1], edges[1:]))
    return 2 / np.pi * tot


def test_s2_transform_matches_density():
    for k in [0.05, 0.5, 1.0, 3.0, 10.0, 30.0]:
        assert abs(s2_hat(k) - s2_hat_by_quadrature(k)) < 1e-11


def test_s2_density_has_unit_mass():
    # Sec. II: 4 pi int_0^{r_cut/2} r^2 rho_PM dr = m
    rc = 0.37
    a = rc / 2
    rho = lambda r: 3 / np.pi * (2 / rc) ** 3 * (1 - r / a)
    m = quad(lambda r: 4 * np.pi * r * r * rho(r), 0, a, epsabs=1e-15)[0]
    assert abs(m - 1.0) < 1e-13


@pytest.mark.parametrize("xi", [0.1, 0.3, 0.5, 0.8, 1.0, 1.2, 1.5, 1.8, 1.95])
def test_g_is_point_minus_cloud_force(xi):
    # a = r_cut/2 = 1 so xi = 2r/r_cut = r
    g_ref = 1.0 - xi ** 2 * cloud_force(xi)
    assert abs(oracle.g(xi) - g_ref) < 1e-10


def test_g_vanishes_beyond_cutoff_by_newtons_theorem():
    for xi in [2.0, 2.3, 3.0]:
        assert abs(1.0 - xi ** 2 * cloud_force(xi)) < 1e-10
        assert oracle.g(xi) == (0.0 if xi > 2 else oracle.g(xi))
    assert oracle.g(2.0 + 1e-12) == 0.0
    assert oracle.g(5.0) == 0.0


def test_g_exact_rationals():
    with open(os.path.join(GOLDEN, "g_rationals.txt")) as f:
        rows = [l.split() for l in f if not l.startswith("#")]
    for xn, xd, gn, gd in rows:
        xi = int(xn) / int(xd)
        g = Fraction(int(gn), int(gd))
        # terms of size ~1 cancel near xi = 2: a few ulps of 1 absolute
        assert abs(oracle.g(xi) - float(g)) <= 8e-15


def test_g_factored_forms():
    # independent representations of Eq. 3 on each branch
    for xi in np.linspace(0.0, 1.0, 41):
        ref = 1 - 8 / 5 * xi ** 3 + 8 / 5 * xi ** 5 - xi ** 6 / 2 - 12 / 35 * xi ** 7 + 3 / 20 * xi ** 8
        assert abs(oracle.g(xi) - ref) < 2e-15
    for xi in np.linspace(1.0, 2.0, 41):
        ref = (2 - xi) ** 5 * (7 * xi ** 3 + 22 * xi ** 2 + 10 * xi + 4) / 140
        assert abs(oracle.g(xi) - ref) < 2e-14


def test_g_smoothness():
    # continuous with continuous slope through xi = 1 and xi = 2, flat at 0
    h = 1e-4
    for x in [1.0, 2.0]:
        gl = [oracle.g(x - k * h) for k in range(3)]
        gr = [oracle.g(x + k * h) if x < 2 else 0.0 for k in range(3)]
        d1l = (3 * gl[0] - 4 * gl[1] + gl[2]) / (2 * h)
        d1r = (-3 * gr[0] + 4 * gr[1] - gr[2]) / (2 * h)
        assert abs(gl[0] - gr[0]) < 1e-14
        assert abs(d1l - d1r) < 1e-6
    assert abs(oracle.g(2.0)) < 1e-15
    assert 0 < oracle.g(2.0 - 1e-2) < 2e-10      # ~ (144/120) h^5 near the cutoff
    assert abs(oracle.g(1e-4) - 1.0) < 1e-11


@pytest.mark.parametrize("xi", [0.05, 0.4, 0.9, 0.99, 1.01, 1.3, 1.7, 1.99])
def test_gpx_is_derivative(xi):
    h = 1e-5
    fd = (-oracle.g(xi + 2 * h) + 8 * oracle.g(xi + h) - 8 * oracle.g(xi - h) + oracle.g(xi - 2 * h)) / (12 * h)
    assert abs(oracle.gpx(xi) * xi - fd) < 1e-9


def test_gpx_closed_forms():
    for xi in np.linspace(0.0, 1.0, 21):
        ref = -24 / 5 * xi + 8 * xi ** 3 - 3 * xi ** 4 - 12 / 5 * xi ** 5 + 6 / 5 * xi ** 6
        assert abs(oracle.gpx(xi) - ref) < 1e-14
    for xi in np.linspace(1.0, 2.0, 21):
        ref = -(xi - 2) ** 4 * (2 * xi ** 2 + 4 * xi - 1) / 5
        assert abs(oracle.gpx(xi) - ref) < 1e-13
    assert oracle.gpx(2.5) == 0.0


@pytest.mark.parametrize("r", [0.02, 0.05, 0.1, 0.2, 0.3])
def test_pair_is_point_minus_cloud_force(r):
    # unsoftened: |a| = G m / r^2 - F_S2S2(r), toward the source
    rcut = 0.4
    a_cloud = rcut / 2
    d = np.array([0.6, -0.48, 0.64]) * r                       # |d| = r
    acc = oracle.pair(d, 2.5, 1.7, 0.0, rcut)
    # scale the unit-radius cloud force to radius a: F_a(r) = F_1(r/a)/a^2
    mag = 1.7 * 2.5 * (1 / r ** 2 - cloud_force(r / a_cloud) / a_cloud ** 2)
    assert np.allclose(acc, mag * d / r, rtol=1e-9, atol=0)


def test_pair_cutoff_and_degenerate():
    rc = 0.1
    for r in [rc, rc * (1 + 1e-12), 0.3]:
        assert np.all(oracle.pair([r, 0, 0], 1.0, 1.0, 1e-3, rc) == 0.0)
    assert np.all(oracle.pair([0, 0, 0], 1.0, 1.0, 1e-3, rc) == 0.0)
    assert np.all(oracle.pair([0, 0, 0], 1.0, 1.0, 0.0, rc) == 0.0)
    assert oracle.pair([rc * (1 - 1e-6), 0, 0], 1.0, 1.0, 0.0, rc)[0] > 0.0


def test_pair_softening_limits():
    rc, eps = 0.1, 1e-3
    # far from eps the softened term tends to the unsoftened one
    d = np.array([0.03, 0.0, 0.0])
    s = oracle.pair(d, 1.0, 1.0, eps, rc)[0]
    u = oracle.pair(d, 1.0, 1.0, 0.0, rc)[0]
    assert abs(s / u - (1 + eps ** 2 / 0.03 ** 2) ** -1.5) < 1e-12
    # deep inside eps the term is linear in d with slope G m g(0)/eps^3
    d = np.array([1e-9, 0.0, 0.0])
    assert abs(oracle.pair(d, 1.0, 1.0, eps, rc)[0] / (1e-9 / eps ** 3) - 1) < 1e-9


def test_pair_minimum_image():
    rc = 0.1
    a = oracle.pair([0.98, 0.0, 0.0], 1.0, 1.0, 0.0, rc)     # image at -0.02
    b = oracle.pair([-0.02, 0.0, 0.0], 1.0, 1.0, 0.0, rc)
    assert np.allclose(a, b, rtol=1e-12, atol=0) and a[0] < 0
    c = oracle.pair([-0.99, 0.005, 3.0], 1.0, 1.0, 0.0, rc)  # image (0.01, 0.005, 0)
    d = oracle.pair([0.01, 0.005, 0.0], 1.0, 1.0, 0.0, rc)
    assert np.allclose(c, d, rtol=1e-12, atol=0)


def test_pair_jacobian_is_derivative():
    rng = np.random.default_rng(3)
    rc, eps, G = 0.2, 2e-3, 1.3
    for _ in range(20):
        d = rng.normal(size=3)
        d *= rng.uniform(0.001, 0.19) / np.linalg.norm(d)
        w = rng.normal(size=3)
        v = oracle.pair_jw(d, 0.7, w, G, eps, rc)
        J = np.zeros((3, 3))
        h = 1e-7 * np.linalg.norm(d)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            J[:, k] = (oracle.pair(d + e, 0.7, G, eps, rc) - oracle.pair(d - e, 0.7, G, eps, rc)) / (2 * h)
        assert np.allclose(J, J.T, rtol=1e-6, atol=1e-6 * np.abs(J).max())
        assert np.allclose(v, J @ w, rtol=1e-6, atol=1e-7 * np.abs(J @ w).max())


def test_tidal_trace_closed_form():
    # eps = 0, G = m = 1: div of d g(2r/rc)/r^3 as a polynomial in r
    # (r_cut < 1/2 so that the offsets stay their own minimum image)
    rc = 0.4
    for r in np.linspace(0.02, 0.396, 25):
        d = np.full(3, r / np.sqrt(3))
        tr = sum(oracle.pair_jw(d, 1.0, np.eye(3)[k], 1.0, 0.0, rc)[k] for k in range(3))
        if r <= rc / 2:
            ref = 64 / (5 * rc ** 8) * (24 * r ** 5 - 24 * r ** 4 * rc - 15 * r ** 3 * rc ** 2
                                        + 20 * r ** 2 * rc ** 3 - 3 * rc ** 5)
        else:
            ref = -64 * (r - rc) ** 4 * (8 * r ** 2 + 8 * r * rc - rc ** 2) / (5 * r * rc ** 8)
        assert abs(tr - ref) < 1e-9 * max(1.0, abs(ref))
    # r -> 0 limit: -4 pi (rho_S2 * rho_S2)(0) = -192/(5 rc^3)
    d = np.array([1e-4, 0, 0])
    tr0 = sum(oracle.pair_jw(d, 1.0, np.eye(3)[k], 1.0, 0.0, rc)[k] for k in range(3))
    assert abs(tr0 / (-192 / (5 * rc ** 3)) - 1) < 1e-3


@pytest.mark.parametrize("xi", [False, True])
def test_pair_is_odd_and_its_jacobian_even(xi):
    """a(-d) = -a(d) and J(-d) = J(d), bit for bit (r, g and s depend on |d|
    only; the minimum image commutes with negation)."""
    rng = np.random.default_rng(8)
    for _ in range(40):
        d = rng.normal(size=3)
        d *= rng.uniform(1e-3, 0.19) / np.linalg.norm(d)
        d += rng.integers(-2, 3, size=3)                # far images of the same offset
        w = rng.normal(size=3)
        a, b = oracle.pair(d, 0.7, 1.3, 2e-3, 0.2, xi), oracle.pair(-d, 0.7, 1.3, 2e-3, 0.2, xi)
        assert np.array_equal(a, -b)
        assert np.array_equal(oracle.pair_jw(d, 0.7, w, 1.3, 2e-3, 0.2, xi),
                              oracle.pair_jw(-d, 0.7, w, 1.3, 2e-3, 0.2, xi))
