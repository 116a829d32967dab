"""Pins of the oracle's event model p_jn and sensitivity s^i_n (CPU only):
brute-force path enumeration with independent line integrals, the mu = 0
closed form, the closed-form primary attenuation of a uniform medium,
quadrature of the model density against the sensitivity, and the 90-degree
symmetry of a symmetric phantom."""
import math

import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S
from tests.test_oracle_physics import clip_line_integral

F2S = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def tiny_geom(n_angles=4, n_bins=8, bin_mm=6.0, radius_mm=50.0, **kw):
    g = S.geometry(n_angles, n_bins, bin_mm, radius_mm, **kw)
    return g


def gauss(x, m, s):
    return math.exp(-0.5 * ((x - m) / s) ** 2) / (s * math.sqrt(2 * math.pi))


def brute_force_row(g, mu, dpx, support, a, u, e, mistake=None):
    """Every path from every support pixel, each with its own line integrals
    (pixel clipping, no tables), following the frozen model reading.
    ``mistake`` plants one plausible error (tests of the pin's power only):
    'response_at_n' centres the scatter path's collimator response on the
    emission pixel, 'no_inv_2pi_r' drops the 1/(2 pi r) factor,
    'flipped_angle' uses -cos(psi) in the Compton and Klein-Nishina laws,
    'det_from_n' attenuates the scattered photon from the emission pixel,
    'mu_at_n' takes the interaction probability at the emission pixel."""
    ny, nx = mu.shape
    th = g["angle0_rad"] + 2 * math.pi * a / g["n_angles"]
    om = np.array([math.cos(th), math.sin(th)])
    tv = np.array([-math.sin(th), math.cos(th)])
    far = (nx + ny + 2) * dpx
    e0 = g["e0_kev"]
    se = lambda E: g["fwhm_frac_e0"] * math.sqrt(e0 * E) * F2S
    su = lambda p: (g["coll_fwhm0_mm"] + g["coll_fwhm_slope"] * (g["radius_mm"] - p @ om)) * F2S
    kbar = oracle.kn_mean(e0)
    centre = lambda pix: np.array([(pix % nx + 0.5 - 0.5 * nx) * dpx,
                                   (pix // nx + 0.5 - 0.5 * ny) * dpx])
    scat = [m for m in range(nx * ny) if mu.reshape(-1)[m] > 0]
    row = []
    for n in support:
        pn = centre(n)
        val = (math.exp(-clip_line_integral(mu, dpx, pn, pn + far * om))
               * gauss(u, pn @ tv, su(pn)) * gauss(e, e0, se(e0)))
        for m in scat:
            if m == n:
                continue
            pm = centre(m)
            v = pm - pn
            r = math.hypot(*v)
            c = (v @ om) / r
            if mistake == "flipped_angle":
                c = -c
            e1 = oracle.compton_energy(e0, c)
            kt = oracle.kn_shape(e0, c) / kbar
            ratio = oracle.sigma_kn(e1) / oracle.sigma_kn(e0)
            pd = pn if mistake == "det_from_n" else pm
            mu_i = mu.reshape(-1)[n if mistake == "mu_at_n" else m]
            w = (dpx * dpx * mu_i * kt * math.exp(-clip_line_integral(mu, dpx, pn, pm))
                 * math.exp(-ratio * clip_line_integral(mu, dpx, pd, pd + far * om))
                 / (1.0 if mistake == "no_inv_2pi_r" else 2 * math.pi * r))
            pr = pn if mistake == "response_at_n" else pm
            val += w * gauss(u, pr @ tv, su(pr)) * gauss(e, e1, se(e1))
        row.append(val)
    return np.array(row)


@pytest.mark.parametrize("n,n_angles,seed", [(4, 3, 0), (5, 4, 1)])
def test_model_matches_brute_force_enumeration(n, n_angles, seed):
    rng = np.random.default_rng(seed)
    dpx = 7.0
    mu = rng.uniform(0.005, 0.03, (n, n)) * (rng.uniform(0, 1, (n, n)) > 0.25)
    g = tiny_geom(n_angles=n_angles, angle0_rad=0.37, radius_mm=45.0)
    g["pixel_mm"] = dpx
    support = np.ones((n, n), dtype=bool)          # includes mu = 0 pixels
    P = oracle.Problem(g, mu, support=support)
    J = 12
    a = rng.integers(0, n_angles, J).astype(np.int32)
    u = rng.uniform(-15, 15, J)
    e = rng.uniform(100, 175, J)
    p = P.model(a, u, e)
    for j in range(J):
        want = brute_force_row(g, mu, dpx, P.support, int(a[j]), u[j], e[j])
        np.testing.assert_allclose(p[j], want, rtol=1e-12, atol=1e-16 * want.max())


def test_mu_zero_reduces_to_blurred_projection():
    n, dpx = 6, 5.0
    mu = np.zeros((n, n))
    g = tiny_geom(n_angles=6, angle0_rad=0.1)
    g["pixel_mm"] = dpx
    P = oracle.Problem(g, mu, support=np.ones((n, n)))
    a = np.array([0, 1, 2, 5], dtype=np.int32)
    u = np.array([-3.0, 0.5, 7.0, 11.0])
    e = np.array([159.0, 150.0, 120.0, 170.0])
    p = P.model(a, u, e)
    xs, ys = P.pixel_centres(P.support)
    se0 = 0.1 * 159.0 * F2S
    for j in range(len(a)):
        th = g["angle0_rad"] + 2 * math.pi * a[j] / g["n_angles"]
        uc = -xs * math.sin(th) + ys * math.cos(th)
        d = g["radius_mm"] - (xs * math.cos(th) + ys * math.sin(th))
        su = (2.5 + 0.05 * d) * F2S
        want = (np.exp(-0.5 * ((u[j] - uc) / su) ** 2) / (su * math.sqrt(2 * math.pi))
                * math.exp(-0.5 * ((e[j] - 159.0) / se0) ** 2) / (se0 * math.sqrt(2 * math.pi)))
        np.testing.assert_allclose(p[j], want, rtol=1e-13)


def _gl_panels(lo, hi, n_panels, order=12):
    x, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(lo, hi, n_panels + 1)
    h = 0.5 * (edges[1:] - edges[:-1])
    c = 0.5 * (edges[1:] + edges[:-1])
    return (c[:, None] + h[:, None] * x).ravel(), (h[:, None] * w).ravel()


def test_sensitivity_is_integral_of_model_density():
    """sum_a of the model density integrated over the detector extent and the
    energy window equals the total sensitivity (pins D_u, D_E against k)."""
    rng = np.random.default_rng(5)
    n, dpx = 5, 6.0
    mu = rng.uniform(0.008, 0.03, (n, n))
    mu[0, 0] = 0.0
    g = tiny_geom(n_angles=4, n_bins=6, bin_mm=6.0, radius_mm=45.0, angle0_rad=0.2)
    g["pixel_mm"] = dpx
    P = oracle.Problem(g, mu)
    half = 0.5 * g["n_bins"] * g["bin_mm"]
    uq, uw = _gl_panels(-half, half, 24)
    eq, ew = _gl_panels(g["e_lo_kev"], g["e_hi_kev"], 25)
    U, E = np.meshgrid(uq, eq, indexing="ij")
    W = np.outer(uw, ew).ravel()
    tot = np.zeros(P.n_sup)
    for a in range(g["n_angles"]):
        p = P.model(np.full(U.size, a, dtype=np.int32), U.ravel(), E.ravel())
        tot += W @ p
    s = P.sensitivity(2)
    np.testing.assert_allclose(tot, s.sum(axis=0), rtol=2e-10)
    # and subset split: angles 0, 2 -> subset 0
    p0 = sum(W @ P.model(np.full(U.size, a, dtype=np.int32), U.ravel(), E.ravel()) for a in (0, 2))
    np.testing.assert_allclose(p0, s[0], rtol=2e-10)


def test_model_density_integrates_to_one_without_window():
    """With mu = 0 the event density of one pixel at one angle, integrated
    over all of (u, E), is one."""
    n, dpx = 2, 6.0
    mu = np.zeros((n, n))
    g = tiny_geom(n_angles=4, n_bins=40, bin_mm=6.0, e_lo_kev=60.0, e_hi_kev=260.0)
    g["pixel_mm"] = dpx
    P = oracle.Problem(g, mu, support=np.ones((n, n)))
    uq, uw = _gl_panels(-60, 60, 40)
    eq, ew = _gl_panels(60, 260, 40)
    U, E = np.meshgrid(uq, eq, indexing="ij")
    W = np.outer(uw, ew).ravel()
    p = P.model(np.full(U.size, 1, dtype=np.int32), U.ravel(), E.ravel())
    np.testing.assert_allclose(W @ p, 1.0, rtol=1e-10)


def test_symmetric_phantom_rotation_invariance():
    rng = np.random.default_rng(8)
    n, dpx = 6, 6.0
    base = rng.uniform(0.005, 0.03, (n, n)) * (rng.uniform(0, 1, (n, n)) > 0.2)
    mu = sum(np.rot90(base, k) for k in range(4)) / 4
    g = tiny_geom(n_angles=8, n_bins=10, bin_mm=6.0, radius_mm=60.0, angle0_rad=0.0)
    g["pixel_mm"] = dpx
    P = oracle.Problem(g, mu)
    s = P.sensitivity(1)[0]
    img = np.zeros(n * n)
    img[P.support] = s
    img = img.reshape(n, n)
    # a 90-degree counter-clockwise turn maps pixel (ix, iy) to (n-1-iy, ix)
    rot = np.zeros_like(img)
    for iy in range(n):
        for ix in range(n):
            rot[ix, n - 1 - iy] = img[iy, ix]
    np.testing.assert_allclose(rot, img, rtol=1e-12, atol=1e-15)
    # event model: angle a + n_angles/4 at the rotated pixel equals angle a
    J = 6
    a = rng.integers(0, 8, J).astype(np.int32)
    u = rng.uniform(-20, 20, J)
    e = rng.uniform(100, 175, J)
    p = P.model(a, u, e)
    pr = P.model((a + 2) % 8, u, e)
    idx = {pix: k for k, pix in enumerate(P.support)}
    for k, pix in enumerate(P.support):
        ix, iy = pix % n, pix // n
        k2 = idx[ix * n + (n - 1 - iy)]
        np.testing.assert_allclose(pr[:, k2], p[:, k], rtol=1e-11, atol=1e-18)


def test_pos_cut_only_drops_negligible_terms():
    ph, g, J, ns, ni = S.workload("tiny16")
    g = dict(g, pixel_mm=ph.pixel_mm)
    ev = S.simulate_events(ph, g, 200, seed=3)
    full = oracle.Problem(g, ph.mu, pos_cut=1e9).model(ev.angle, ev.u_mm, ev.e_kev)
    cut = oracle.Problem(g, ph.mu).model(ev.angle, ev.u_mm, ev.e_kev)
    np.testing.assert_allclose(cut, full, rtol=1e-14, atol=1e-15 * full.max())


def test_model_parts_add_up():
    """The primary-only and scatter-only restrictions of the path sum add up to
    the full sum, and the scatter part vanishes without matter."""
    ph, g, J, ns, ni = S.workload("tiny16")
    g = dict(g, pixel_mm=ph.pixel_mm)
    ev = S.simulate_events(ph, g, 60, seed=21)
    P = oracle.Problem(g, ph.mu)
    full = P.model(ev.angle, ev.u_mm, ev.e_kev)
    prim = P.model(ev.angle, ev.u_mm, ev.e_kev, scatter=False)
    scat = P.model(ev.angle, ev.u_mm, ev.e_kev, primary=False)
    np.testing.assert_allclose(prim + scat, full, rtol=1e-13, atol=1e-300)
    assert np.all(scat > 0) and np.all(prim >= 0)


def test_uniform_medium_primary_closed_form():
    """Closed-form attenuation: with mu uniform over the whole square grid,
    the primary path of pixel n at angle a crosses mu over the exact distance
    from its centre to the square's edge along omega_a, so its model entry is
    exp(-mu l) phi(u; p.t, sigma_u(R - p.omega)) phi(E; E0, sigma_E(E0)).
    No line-integral code is involved on this side."""
    n, dpx, mu0 = 7, 4.0, 0.015
    g = tiny_geom(n_angles=12, n_bins=16, bin_mm=4.0, radius_mm=60.0, angle0_rad=0.1)
    mu = np.full((n, n), mu0)
    P = oracle.Problem(dict(g, pixel_mm=dpx), mu)
    assert P.n_sup == n * n
    rng = np.random.default_rng(5)
    J = 40
    a = rng.integers(0, g["n_angles"], J).astype(np.int32)
    u = rng.uniform(-12.0, 12.0, J).astype(np.float32)
    e = rng.uniform(140.0, 175.0, J).astype(np.float32)
    p = P.model(a, u, e, primary=True, scatter=False)
    half = 0.5 * n * dpx
    e0 = g["e0_kev"]
    se0 = g["fwhm_frac_e0"] * e0 * F2S
    want = np.zeros((J, n * n))
    for j in range(J):
        th = g["angle0_rad"] + 2 * math.pi * a[j] / g["n_angles"]
        om = np.array([math.cos(th), math.sin(th)])
        tv = np.array([-math.sin(th), math.cos(th)])
        for q in range(n * n):
            pc = np.array([(q % n + 0.5 - 0.5 * n) * dpx, (q // n + 0.5 - 0.5 * n) * dpx])
            ell = min((math.copysign(half, om[k]) - pc[k]) / om[k] for k in range(2) if om[k] != 0.0)
            su = (g["coll_fwhm0_mm"] + g["coll_fwhm_slope"] * (g["radius_mm"] - pc @ om)) * F2S
            want[j, q] = (math.exp(-mu0 * ell) * gauss(float(u[j]), pc @ tv, su)
                          * gauss(float(e[j]), e0, se0))
    np.testing.assert_allclose(p, want, rtol=1e-11, atol=1e-15 * want.max())
