"""Pins of the binned-attribute oracle (the paper's binning experiment,
Section 4): the bin-integrated model and the count-weighted EM.

* The masses of a row family that tiles the detector extent and the energy
  window sum, for every support pixel and angle, to the pixel's detection
  probability at that angle: the sensitivity, computed by a separate oracle
  function from full-range masses.
* In the limit of narrow bins the bin model divided by the bin volume is the
  list-mode event density at the bin centre (midpoint rule).
* EM and likelihood with counts equal EM and likelihood on the rows repeated
  count times.
"""
import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S
from tests._helpers import oracle_problem


def _all_bins(na, nb, nk):
    a = np.repeat(np.arange(na), nb * nk)
    pb = np.tile(np.repeat(np.arange(nb), nk), na)
    eb = np.tile(np.arange(nk), na * nb)
    return a, pb, eb


@pytest.mark.parametrize("edges", [(100.0, 143.0, 175.0), (100.0, 120.0, 143.0, 175.0)])
def test_bin_masses_sum_to_the_per_angle_sensitivity(edges):
    ph, g, J, ns, ni = S.workload("tiny16")
    P = oracle_problem(ph, g)
    na, nb = g["n_angles"], g["n_bins"]
    a, pb, eb = _all_bins(na, nb, len(edges) - 1)
    p = P.model_binned(a, pb, eb, edges)
    tot = np.zeros((na, P.n_sup))
    np.add.at(tot, a, p)
    s = P.sensitivity(na)            # one angle per subset
    np.testing.assert_allclose(tot, s, rtol=1e-12, atol=1e-14 * s.max())


def test_narrow_bins_give_the_event_density():
    ph, g, J, ns, ni = S.workload("tiny16")
    fine = dict(g, n_bins=g["n_bins"] * 1000, bin_mm=g["bin_mm"] / 1000)
    P = oracle_problem(ph, fine)
    rng = np.random.default_rng(4)
    n = 24
    a = rng.integers(0, g["n_angles"], n)
    half = 0.5 * fine["n_bins"] * fine["bin_mm"]
    pb = rng.integers(int(0.3 * fine["n_bins"]), int(0.7 * fine["n_bins"]), n)
    uc = -half + (pb + 0.5) * fine["bin_mm"]
    ec = rng.uniform(110.0, 170.0, n)
    de = 1e-2
    rows = []
    for j in range(n):
        pbin = P.model_binned([a[j]], [pb[j]], [0], [ec[j] - 0.5 * de, ec[j] + 0.5 * de])
        rows.append(pbin[0] / (fine["bin_mm"] * de))
    dens = P.model(a, uc, ec)
    got = np.array(rows)
    scale = dens.max(axis=1, keepdims=True)
    assert np.max(np.abs(got - dens) / scale) < 2e-5


def test_count_weighted_em_equals_repeated_events():
    rng = np.random.default_rng(9)
    n_rows, n_pix, n_sub = 40, 13, 4
    p = rng.uniform(0.0, 1.0, (n_rows, n_pix)) * (rng.uniform(size=(n_rows, n_pix)) < 0.7)
    p[:, 0] += 0.05
    angle = rng.integers(0, 12, n_rows)
    counts = rng.integers(1, 6, n_rows).astype(np.float64)
    s = np.stack([p[(angle % n_sub) == i].sum(0) + 0.3 for i in range(n_sub)])
    rep = np.repeat(np.arange(n_rows), counts.astype(int))
    f0 = oracle.initial_image(counts.sum(), s.sum(0))
    fw, hw = oracle.osem(p, angle, s, 3, f0, weights=counts)
    fr, hr = oracle.osem(p[rep], angle[rep], s, 3, f0)
    np.testing.assert_allclose(fw, fr, rtol=1e-12)
    lw = oracle.loglik(p, fw, s.sum(0), weights=counts)
    lr = oracle.loglik(p[rep], fr, s.sum(0))
    assert abs(lw - lr) <= 1e-10 * abs(lr)
