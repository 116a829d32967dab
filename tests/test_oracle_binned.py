"""Pins of the support initialiser's FP64 reference (CPU only): its detector
geometry against closed forms at the axis angles, the bin-integrated
projector against numerical quadrature of the collimator response, the sinogram against a brute-force count, the EM count identity of
every sub-iteration, likelihood ascent and point-source recovery on noiseless
data, and the threshold/dilation on hand-made images."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import binned
from paper_2002_12471_gb300 import synthetic as S


@pytest.fixture(scope="module")
def small():
    g = S.geometry(8, 12, 6.0, 60.0)
    return g, 8, 8, 7.0


def test_projector_matches_quadrature(small):
    g, nx, ny, dpx = small
    A = binned.projector(g, nx, ny, dpx)
    u, sig = binned.geometry_arrays(g, nx, ny, dpx)
    rng = np.random.default_rng(0)
    w = g["bin_mm"]
    for _ in range(25):
        a, k, n = rng.integers(0, g["n_angles"]), rng.integers(0, g["n_bins"]), rng.integers(0, nx * ny)
        lo = -0.5 * g["n_bins"] * w + k * w
        dens = lambda x: math.exp(-0.5 * ((x - u[a, n]) / sig[a, n]) ** 2) / (sig[a, n] * math.sqrt(2 * math.pi))
        ref, _ = integrate.quad(dens, lo, lo + w, epsabs=1e-14, epsrel=1e-12)
        assert A[a, k, n] == pytest.approx(ref, rel=1e-9, abs=1e-14)
    # a pixel whose response lies well inside the detector: the bins hold all of it
    inside = np.abs(u) + 8 * sig < 0.5 * g["n_bins"] * w
    np.testing.assert_allclose(A.sum(axis=1)[inside], 1.0, atol=1e-12)


def test_sinogram_brute_force(small):
    g = small[0]
    rng = np.random.default_rng(1)
    half = 0.5 * g["n_bins"] * g["bin_mm"]
    angle = rng.integers(0, g["n_angles"], 300)
    u = rng.uniform(-half, half, 300)
    u[:3] = [half, -half, 0.0]
    c = binned.sinogram(g, angle, u)
    ref = np.zeros_like(c)
    for a, x in zip(angle, u):
        k = 0
        while k + 1 < g["n_bins"] and -half + (k + 1) * g["bin_mm"] <= x:
            k += 1
        ref[a, k] += 1
    np.testing.assert_array_equal(c, ref)
    assert c.sum() == 300


def test_count_identity_every_subiteration(small):
    g, nx, ny, dpx = small
    A = binned.projector(g, nx, ny, dpx)
    rng = np.random.default_rng(2)
    c = rng.poisson(3.0, (g["n_angles"], g["n_bins"])).astype(np.float64)
    f, sens, hist = binned.osem(A, c, 4, 3)
    for i, fi, y in hist:
        ci = c[i::4]
        assert np.dot(sens[i], fi) == pytest.approx(ci[y > 0].sum(), rel=1e-12)


def test_noiseless_point_source(small):
    g, nx, ny, dpx = small
    A = binned.projector(g, nx, ny, dpx)
    f_true = np.full(nx * ny, 0.01)
    hot = 3 * nx + 5
    f_true[hot] = 50.0
    c = np.einsum("akn,n->ak", A, f_true)
    lls = []
    f = None
    for iters in (1, 2, 4, 8, 16):
        f, _, _ = binned.osem(A, c, 1, iters)
        y = np.einsum("akn,n->ak", A, f)
        lls.append(np.sum(c * np.log(np.where(y > 0, y, 1.0))) - y.sum())
    assert np.all(np.diff(lls) > 0)
    assert int(np.argmax(f)) == hot
    assert f[hot] > 0.5 * f_true[hot]


def test_support_mask_threshold_and_dilation():
    nx = ny = 9
    f = np.zeros(nx * ny)
    img = f.reshape(ny, nx)
    img[3:6, 3:6] = 1.0
    img[4, 4] = 10.0
    m0 = binned.support_mask(f, nx, ny, 0.05, 0).reshape(ny, nx)
    ref = np.zeros((ny, nx), bool)
    ref[3:6, 3:6] = True
    np.testing.assert_array_equal(m0, ref)
    m1 = binned.support_mask(f, nx, ny, 0.05, 1).reshape(ny, nx)
    ref1 = np.zeros((ny, nx), bool)
    ref1[2:7, 2:7] = True
    np.testing.assert_array_equal(m1, ref1)
    # a corner pixel dilates only into the grid
    f2 = np.zeros(nx * ny)
    f2[0] = 1.0
    m2 = binned.support_mask(f2, nx, ny, 0.5, 1).reshape(ny, nx)
    assert m2.sum() == 4 and m2[:2, :2].all()
    # the threshold keeps only the hot pixel
    m3 = binned.support_mask(f, nx, ny, 0.5, 0)
    assert m3.sum() == 1 and m3[4 * nx + 4]


def test_geometry_at_the_axis_angles():
    """u_a(p) and sigma_u(d_a(p)) against their closed forms at theta = 0,
    pi/2, pi, 3 pi/2, where the lateral axis and the depth are read off the
    pixel coordinates: u = y, -x, -y, x and d = R - x, R - y, R + x, R + y."""
    g = S.geometry(4, 12, 6.0, 60.0, coll_fwhm0_mm=2.0, coll_fwhm_slope=0.1)
    nx, ny, dpx = 5, 4, 7.0
    u, sig = binned.geometry_arrays(g, nx, ny, dpx)
    f2s = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    R = g["radius_mm"]
    for n in range(nx * ny):
        x = (n % nx + 0.5 - 0.5 * nx) * dpx
        y = (n // nx + 0.5 - 0.5 * ny) * dpx
        for a, (uu, d) in enumerate(((y, R - x), (-x, R - y), (-y, R + x), (x, R + y))):
            assert u[a, n] == pytest.approx(uu, abs=1e-12)
            assert sig[a, n] == pytest.approx((2.0 + 0.1 * d) * f2s, rel=1e-13)
