"""Pins of the oracle's photon physics and line integrals against closed forms,
limits and independent numerical integration (CPU only)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

E0 = 159.0
MEC2 = 510.99895


def test_compton_endpoints():
    # no deflection keeps the energy; backscatter gives E0 / (1 + 2 E0/mc^2)
    assert oracle.compton_energy(E0, 1.0) == pytest.approx(E0, rel=1e-15)
    eb = oracle.compton_energy(E0, -1.0)
    assert eb == pytest.approx(E0 / (1 + 2 * E0 / MEC2), rel=1e-15)
    assert eb == pytest.approx(98.01, abs=0.01)   # 159 keV backscatter peak
    # 90 degrees: E0 / (1 + E0/mc^2)
    assert oracle.compton_energy(E0, 0.0) == pytest.approx(E0 / (1 + E0 / MEC2), rel=1e-15)


def test_kn_shape_forward_and_thomson_limit():
    assert oracle.kn_shape(E0, 1.0) == pytest.approx(1.0, rel=1e-15)
    for c in np.linspace(-1, 1, 11):
        # E -> 0: Thomson (1 + cos^2)/2
        assert oracle.kn_shape(1e-7, c) == pytest.approx(0.5 * (1 + c * c), rel=1e-8)
    # the shape decreases with energy at every non-zero angle
    for c in (0.5, 0.0, -1.0):
        assert oracle.kn_shape(300.0, c) < oracle.kn_shape(159.0, c) < oracle.kn_shape(50.0, c)


def test_kn_total_cross_section_matches_integral_of_shape():
    # sigma / (2 pi r_e^2) = int_0^pi K(theta) sin(theta) d theta  (3-D KN);
    # the closed form and the shape are pinned against each other
    for e in (20.0, 98.0, 140.0, 159.0, 364.0):
        num, _ = integrate.quad(lambda t: oracle.kn_shape(e, math.cos(t)) * math.sin(t), 0, math.pi,
                                epsabs=1e-14, epsrel=1e-13)
        assert oracle.sigma_kn(e) == pytest.approx(num, rel=1e-11)
    # Thomson limit: 8 pi r_e^2 / 3 (1 - 2k + O(k^2)) -> 4/3 (1 - 2k) in these
    # units (k = E / m_e c^2 small, but not so small that the closed form cancels)
    k = 0.5 / MEC2
    assert oracle.sigma_kn(0.5) == pytest.approx(4.0 / 3.0 * (1 - 2 * k), rel=1e-5)


def test_kn_mean_normalises_in_plane_density():
    for e in (50.0, 159.0, 300.0):
        num, _ = integrate.quad(lambda p: oracle.kn_shape(e, math.cos(p)), 0, 2 * math.pi,
                                epsabs=1e-14, epsrel=1e-13, limit=200)
        assert oracle.kn_mean(e) == pytest.approx(num / (2 * math.pi), rel=1e-12)
    # Thomson: mean of (1 + cos^2)/2 over the circle is 3/4
    assert oracle.kn_mean(1e-7) == pytest.approx(0.75, rel=1e-8)


# ---------------------------------------------------------------- line integrals

def clip_line_integral(mu, dpx, p0, p1):
    """Independent exact line integral: clip the segment against every pixel
    square (Liang-Barsky) and sum mu times the clipped length."""
    ny, nx = mu.shape
    x0, y0 = p0
    dx, dy = p1[0] - p0[0], p1[1] - p0[1]
    L = math.hypot(dx, dy)
    xs = (np.arange(nx) - 0.5 * nx) * dpx
    ys = (np.arange(ny) - 0.5 * ny) * dpx
    X0, Y0 = np.meshgrid(xs, ys)
    X1, Y1 = X0 + dpx, Y0 + dpx
    t0 = np.zeros_like(X0)
    t1 = np.ones_like(X0)
    for p, qlo, qhi in ((dx, X0 - x0, X1 - x0), (dy, Y0 - y0, Y1 - y0)):
        if p == 0.0:
            bad = (qlo > 0) | (qhi < 0)
            t1 = np.where(bad, -1.0, t1)
        else:
            a, b = qlo / p, qhi / p
            t0 = np.maximum(t0, np.minimum(a, b))
            t1 = np.minimum(t1, np.maximum(a, b))
    seg = np.clip(t1 - t0, 0.0, None) * L
    return float(np.sum(seg * mu))


def midpoint_line_integral(mu, dpx, p0, p1, n=1_000_000):
    ny, nx = mu.shape
    t = (np.arange(n) + 0.5) / n
    x = p0[0] + t * (p1[0] - p0[0])
    y = p0[1] + t * (p1[1] - p0[1])
    ix = np.floor(x / dpx + 0.5 * nx).astype(int)
    iy = np.floor(y / dpx + 0.5 * ny).astype(int)
    ok = (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny)
    vals = np.zeros(n)
    vals[ok] = mu[iy[ok], ix[ok]]
    return float(vals.sum() * math.hypot(p1[0] - p0[0], p1[1] - p0[1]) / n)


def test_axis_aligned_ray_sums_pixels():
    rng = np.random.default_rng(3)
    mu = rng.uniform(0, 0.03, (8, 8))
    d = 4.0
    # from the centre of pixel (ix=2, iy=5) towards +x: half of it plus the rest of the row
    x = (2 + 0.5 - 4) * d
    y = (5 + 0.5 - 4) * d
    want = 0.5 * d * mu[5, 2] + d * mu[5, 3:].sum()
    assert oracle.ray_to_edge(mu, d, (x, y), (1.0, 0.0)) == pytest.approx(want, rel=1e-14)
    want = 0.5 * d * mu[5, 2] + d * mu[:5, 2].sum()       # towards -y
    assert oracle.ray_to_edge(mu, d, (x, y), (0.0, -1.0)) == pytest.approx(want, rel=1e-14)


def test_line_integral_random_maps():
    rng = np.random.default_rng(11)
    for trial in range(20):
        n = int(rng.integers(3, 12))
        mu = rng.uniform(0, 0.03, (n, n)) * (rng.uniform(0, 1, (n, n)) > 0.2)
        d = float(rng.uniform(1, 8))
        ext = 0.5 * n * d
        p0 = rng.uniform(-1.3 * ext, 1.3 * ext, 2)
        p1 = rng.uniform(-1.3 * ext, 1.3 * ext, 2)
        v = oracle.line_integral(mu, d, p0, p1)
        assert v == pytest.approx(clip_line_integral(mu, d, p0, p1), rel=1e-12, abs=1e-14)
        assert v == pytest.approx(oracle.line_integral(mu, d, p1, p0), rel=1e-13, abs=1e-15)
        if trial < 5:
            assert v == pytest.approx(midpoint_line_integral(mu, d, p0, p1), rel=1e-5, abs=1e-9)


def test_disk_chord_converges():
    # centre-to-edge integral through an area-rasterised uniform disk tends to
    # mu * rho at first order in the pixel size
    rho, m = 50.0, 0.015
    errs = []
    for n in (16, 32, 64):
        d = 128.0 / n
        sub = 16
        k = ((np.arange(n * sub) + 0.5) / sub - 0.5 * n) * d
        X, Y = np.meshgrid(k, k)
        mu = (np.hypot(X, Y) <= rho).astype(float).reshape(n, sub, n, sub).mean(axis=(1, 3)) * m
        th = 0.3
        got = oracle.ray_to_edge(mu, d, (0.0, 0.0), (math.cos(th), math.sin(th)))
        errs.append(abs(got - m * rho))
    assert errs[-1] < 0.02 * m * rho
    assert errs[2] < errs[0]
