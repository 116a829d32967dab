"""Physical pin of the path weights (paper Section 2.1, Eq. 4: s_eff of a
path; Section 2.2: first-order, in-plane scatter), against photon counts.

The photon Monte-Carlo of the synthetic inputs follows each emitted photon:
emission point uniform in its pixel, Woodcock tracking through the mu-map,
Compton deflection with the Klein-Nishina law, escape, collimator and energy
blur.  It labels every detected event with its true scatter order and shares
no arithmetic with the oracle.  For E photons emitted in proportion to the
activity f, the expected number of detected events at angle a that took
path type k (0: unscattered, 1: one Compton scatter) is

    E[N^k_a] = (E / N_theta) sum_q (f_q / sum f) s^k_{a,q},

where s^k is the oracle's sensitivity restricted to that path type.  The
factor 1/N_theta is the angular acceptance of one detector angle (the
simulator assigns an escaping photon to the nearest of N_theta angles); it is
the constant the oracle leaves in T for both path types alike.  So the
absolute weight of a scatter path, D^2 mu_m Kt exp(-L) exp(-r L_det)/(2 pi r),
is checked against physics and not against a second writing of itself.

What the comparison must show, and its tolerances:

* Unscattered events match at every pixel size: the oracle's exp(-L_det) from
  the pixel centre along the angle's axis differs from the average over the
  pixel and the angular bin only at second order, (mu D)^2/24 and
  (pi/N_theta)^2/6, below 2e-3.  Bound: 4 sigma of the count plus 2e-3; the
  per-angle chi^2/dof (32 angles) below 2.
* Once-scattered events exceed the oracle by an amount of order D: the
  oracle leaves out scatter inside the emission pixel (m = n; probability
  about mu times a fraction of D) and evaluates 1/r at the centres of the
  nearest pixels, which by convexity is below the pixel average.  Both vanish
  linearly, so the excess must be positive and roughly halve when D halves
  (ratio in [0.3, 0.7]), and the Richardson extrapolation 2 r(D/2) - r(D) to
  D = 0 must be 1 within 4 sigma plus the second-order remainder (1% from
  8/4 mm, 0.5% from 4/2 mm: the three-level quadratic extrapolation of an
  8M-emission run moved it by less than 0.3%).  This is checked for the
  whole window and for three energy bands ([100, 120], [120, 143],
  [143, 175] keV), which fixes the Compton energy law and the energy blur of
  the scattered photon too; per angle, the extrapolated ratios have
  chi^2/dof below 2.

Planted mistakes, each compiled into a copy of the C oracle on the CPU, fail
the pin: mu D instead of mu D^2, a dropped 2 pi, the Klein-Nishina shape
normalised over twice the circle mean, the scattered photon attenuated at
E0 instead of E', and a flipped cos psi.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S

N_ANG = 32
N_EMIT = 4_000_000
# (grid, pixel mm, Monte-Carlo seed): one disk phantom (water r = 56 mm with an
# 8 mm bone ring, two hot disks at 6:1) at three pixel sizes, same scanner
LEVELS = [(16, 8.0, 101), (32, 4.0, 102), (64, 2.0, 103)]
FULL = (100.0, 175.0)
BANDS = [FULL, (100.0, 120.0), (120.0, 143.0), (143.0, 175.0)]
SYSTEMATIC = {(0, 1): 0.01, (1, 2): 0.005}   # second-order remainder per level pair


def _geom():
    return S.geometry(N_ANG, 16, 8.0, 80.0)


def _counts(ev, order, band):
    lo, hi = band
    m = (ev.order == order) & (ev.e_kev >= lo)
    m &= (ev.e_kev <= hi) if hi == FULL[1] else (ev.e_kev < hi)
    return np.bincount(ev.angle[m], minlength=N_ANG).astype(np.float64)


def _expected(ph, band, primary, scatter):
    """E[N^k_a] for every angle a from the loaded oracle library."""
    g = _geom()
    P = oracle.Problem(dict(g, pixel_mm=ph.pixel_mm), ph.mu)
    P.geom.e_lo_kev, P.geom.e_hi_kev = band
    s = P.sensitivity(N_ANG, primary=primary, scatter=scatter)   # [angle, q]
    act = ph.activity.reshape(-1)[P.support]
    return s @ (N_EMIT / N_ANG * act / ph.activity.sum())


@pytest.fixture(scope="module")
def mc():
    g = _geom()
    out = []
    for n, dpx, seed in LEVELS:
        ph = S.disk_phantom(n, dpx)
        ev = S.simulate_emissions(ph, g, N_EMIT, seed=seed)
        out.append(dict(ph=ph,
                        c0=_counts(ev, 0, FULL),
                        c1={b: _counts(ev, 1, b) for b in BANDS},
                        e0=_expected(ph, FULL, True, False),
                        e1={b: _expected(ph, b, False, True) for b in BANDS}))
    return out


def scatter_pin_failures(c1, e1, pairs, bands, per_angle=True):
    """The once-scattered part of the pin.  c1[level][band], e1[level][band]:
    counts and expectations per angle.  Returns the failed conditions."""
    fails = []
    for lc, lf in pairs:                      # coarse level, fine level (D, D/2)
        for b in bands:
            cc, ec, cf, ef = c1[lc][b], e1[lc][b], c1[lf][b], e1[lf][b]
            rc, rf = cc.sum() / ec.sum(), cf.sum() / ef.sum()
            xc, xf = rc - 1.0, rf - 1.0
            if not (xc > 0 and xf > 0 and 0.3 <= xf / xc <= 0.7):
                fails.append("levels %d/%d band %s: excess %.4f -> %.4f is not O(D)" % (lc, lf, b, xc, xf))
            r0 = 2.0 * rf - rc
            sig = np.sqrt(4.0 * cf.sum() / ef.sum() ** 2 + cc.sum() / ec.sum() ** 2)
            if abs(r0 - 1.0) > 4.0 * sig + SYSTEMATIC[(lc, lf)]:
                fails.append("levels %d/%d band %s: extrapolated ratio %.4f (sigma %.4f)" % (lc, lf, b, r0, sig))
            if per_angle:
                ra = 2.0 * cf / ef - cc / ec
                sa = np.sqrt(4.0 * cf / ef ** 2 + cc / ec ** 2)
                chi = float(np.mean(((ra - 1.0) / sa) ** 2))
                if chi > 2.0:
                    fails.append("levels %d/%d band %s: per-angle chi2/dof %.2f" % (lc, lf, b, chi))
    return fails


def test_unscattered_counts_match_at_every_pixel_size(mc):
    for lvl in mc:
        c, e = lvl["c0"], lvl["e0"]
        r = c.sum() / e.sum()
        assert abs(r - 1.0) <= 4.0 / np.sqrt(c.sum()) + 2e-3, (lvl["ph"].pixel_mm, r)
        chi = float(np.mean((c - e) ** 2 / e))
        assert chi < 2.0, (lvl["ph"].pixel_mm, chi)


def test_once_scattered_counts_converge_to_the_oracle(mc):
    c1 = [lvl["c1"] for lvl in mc]
    e1 = [lvl["e1"] for lvl in mc]
    fails = scatter_pin_failures(c1, e1, pairs=[(0, 1), (1, 2)], bands=BANDS)
    assert not fails, fails


# ------------------------------------------------------------------ planted mistakes

_SRC = os.path.join(os.path.dirname(oracle.__file__), "lmosem_oracle.c")
MISTAKES = {
    "mu_D_not_mu_D2": ("*w = g->pixel_mm * g->pixel_mm * mu[pix_m] * kt",
                       "*w = g->pixel_mm * mu[pix_m] * kt"),
    "dropped_2pi": ("(2.0 * ORC_PI * r);", "(r);"),
    "kn_over_twice_the_mean": ("double kt = orc_kn_shape(g->e0_kev, cos_psi) / kbar;",
                               "double kt = orc_kn_shape(g->e0_kev, cos_psi) / (2.0 * kbar);"),
    "escape_at_e0": ("double ratio = orc_sigma_kn(e1) / sig0;", "double ratio = 1.0;"),
    "flipped_cos_psi": ("double cos_psi = (vx * cos(th) + vy * sin(th)) / r;",
                        "double cos_psi = -(vx * cos(th) + vy * sin(th)) / r;"),
}


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_weight_mistakes_fail_the_count_pin(mc, name, tmp_path, monkeypatch):
    old, new = MISTAKES[name]
    src = open(_SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = oracle.load(oracle.compile_source(str(path), str(tmp_path / "libmutant.so")))
    monkeypatch.setattr(oracle, "_lib", lib)
    # the two coarser levels and the whole window suffice to expose each one
    e1 = [{FULL: _expected(lvl["ph"], FULL, False, True)} for lvl in mc[:2]]
    c1 = [{FULL: lvl["c1"][FULL]} for lvl in mc[:2]]
    assert scatter_pin_failures(c1, e1, pairs=[(0, 1)], bands=[FULL], per_angle=False), name
