"""Pins of the oracle's detector-line attenuation (the two line inputs of the
scatter surrogate) against closed forms: a uniform square, where the
integral from depth s to the detector is mu times the distance to the exit
side, and a uniform disk, whose whole-line integral is mu times the chord
(CPU only)."""
import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S


def _problem(mu, n_angles=8, n_bins=16, bin_mm=8.0, pixel_mm=8.0):
    g = dict(S.workload("tiny16")[1])
    g.update(n_angles=n_angles, n_bins=n_bins, bin_mm=bin_mm, pixel_mm=pixel_mm)
    return oracle.Problem(g, mu)


def test_uniform_square_distance_to_exit_at_axis_angles():
    # mu uniform over the whole 16 x 16 grid (half side A = 64 mm): along the
    # line {s omega + u t}, |u| < A, the integral from s in [-A, A] to the
    # detector is mu (A - s) at the four axis angles; bilinear interpolation
    # of a function linear in s and constant in u is exact away from |u| = A
    mu0 = 0.0153
    P = _problem(np.full((16, 16), mu0))
    A = 64.0
    rng = np.random.default_rng(3)
    for a in (0, 2, 4, 6):      # theta = 0, 90, 180, 270 degrees of 8 angles
        u = rng.uniform(-A + 6.0, A - 6.0, 40)
        s = rng.uniform(-A + 6.0, A - 6.0, 40)
        got = P.line_attenuation(np.full(40, a), u, s)
        np.testing.assert_allclose(got, mu0 * (A - s), rtol=1e-12, atol=1e-12)
        # the whole line (from before the grid) is the full side
        whole = P.line_attenuation(np.full(40, a), u, np.full(40, P.line_start()))
        np.testing.assert_allclose(whole, mu0 * 2 * A, rtol=1e-12)
    # beyond the grid along omega nothing is left
    far = P.line_attenuation(np.zeros(5), np.linspace(-30, 30, 5), np.full(5, A + 8.0))
    np.testing.assert_allclose(far, 0.0, atol=1e-15)


def test_uniform_square_oblique_line_from_a_depth():
    # theta = 45 degrees: for a point inside the square whose exit lies on the
    # side x = A (u < 0 here), the distance to the exit is (A - x) / cos 45
    mu0 = 0.011
    P = _problem(np.full((16, 16), mu0))
    A = 64.0
    th = np.pi / 4
    rng = np.random.default_rng(4)
    for _ in range(20):
        u = rng.uniform(-40.0, -12.0)
        s = rng.uniform(-20.0, 20.0)
        x = s * np.cos(th) - u * np.sin(th)
        y = s * np.sin(th) + u * np.cos(th)
        assert abs(x) < A and abs(y) < A
        got = float(P.line_attenuation(np.array([1]), np.array([u]), np.array([s]))[0])
        assert got == pytest.approx(mu0 * (A - x) / np.cos(th), rel=1e-9)


def test_whole_line_through_a_disk_is_the_chord():
    # a uniform disk of radius R on a fine grid: the whole-line integral at
    # lateral offset u is 2 mu sqrt(R^2 - u^2), up to the pixelisation of the
    # disk edge (a band of one pixel: 2 mu dpx at most, less off the rim)
    n, dpx, R, mu0 = 128, 1.0, 40.0, 0.02
    c = (np.arange(n) + 0.5 - n / 2) * dpx
    xx, yy = np.meshgrid(c, c)
    P = _problem(np.where(xx ** 2 + yy ** 2 <= R * R, mu0, 0.0), n_angles=12, n_bins=128, bin_mm=1.0,
                 pixel_mm=dpx)
    u = np.linspace(-30.0, 30.0, 13)
    for a in (0, 1, 5):
        whole = P.line_attenuation(np.full(u.shape, a), u, np.full(u.shape, P.line_start()))
        np.testing.assert_allclose(whole, 2 * mu0 * np.sqrt(R * R - u * u), atol=2 * mu0 * dpx)


def _pin_holds(P, mu0, A=64.0):
    """theta = 0, lines y = u < 0 inside the filled part: mu0 (A - s)."""
    rng = np.random.default_rng(5)
    u = rng.uniform(-40.0, -12.0, 20)
    s = rng.uniform(-50.0, 50.0, 20)
    return bool(np.allclose(P.line_attenuation(np.zeros(20, dtype=int), u, s), mu0 * (A - s),
                            rtol=1e-12, atol=1e-12))


def test_planted_line_mistakes_fail_the_closed_form(monkeypatch):
    """The closed forms have teeth: integrating away from the detector
    (-omega) fails the uniform square's; placing the line on the wrong side
    of the origin (t -> -t) fails that of a map filled only below y = 0."""
    mu0 = 0.0153
    full = np.full((16, 16), mu0)
    half = full.copy()
    half[8:, :] = 0.0     # rows with y > 0 empty
    assert _pin_holds(_problem(full), mu0) and _pin_holds(_problem(half), mu0)
    orig = oracle.ray_to_edge
    monkeypatch.setattr(oracle, "ray_to_edge", lambda mu, dpx, p0, d: orig(mu, dpx, p0, (-d[0], -d[1])))
    assert not _pin_holds(_problem(full), mu0)

    def mirrored(mu, dpx, p0, d):
        u = -d[1] * p0[0] + d[0] * p0[1]           # p0 = s omega + u t  ->  s omega - u t
        return orig(mu, dpx, (p0[0] + 2 * u * d[1], p0[1] - 2 * u * d[0]), d)
    monkeypatch.setattr(oracle, "ray_to_edge", mirrored)
    assert not _pin_holds(_problem(half), mu0)
