"""Regression of the oracle against its frozen fixture (CPU only).  The
fixture was written by tests/golden/make_golden.py, which calls only the
oracle; a change in the oracle's arithmetic must come with a regenerated
fixture and a commit message naming the passage that justifies it."""
import json
import os

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_frozen_fixture():
    with open(os.path.join(HERE, "golden", "tiny16_oracle.json")) as fh:
        G = json.load(fh)
    mu = np.array(G["mu"])
    P = oracle.Problem(G["geometry"], mu)
    assert P.support.tolist() == G["support"]
    ev = G["events"]
    a = np.array(ev["angle"], dtype=np.int32)
    u = np.array(ev["u_mm"])
    e = np.array(ev["e_kev"])
    p = P.model(a, u, e)
    for j, q, v in G["model_samples"]:
        assert abs(p[j, q] - v) <= 1e-12 * abs(v) + 1e-300
    np.testing.assert_allclose(p.sum(1), G["row_sums"], rtol=1e-12)
    s = P.sensitivity(len(G["sens"]))
    np.testing.assert_allclose(s, G["sens"], rtol=1e-12)
    f0 = oracle.initial_image(len(a), s.sum(0))
    f, hist = oracle.osem(p, a, s, len(G["loglik"]), f0)
    np.testing.assert_allclose(f, G["image"], rtol=1e-9)
    np.testing.assert_allclose([oracle.loglik(p, h, s.sum(0)) for h in hist], G["loglik"], rtol=1e-12)


def test_dat128_subset_fixture_is_the_workloads_case():
    """The frozen 128 x 128 subset (tests/golden/make_dat128_subset.py) holds
    the precision workload's phantom, scanner and ROI weights, events inside
    the detector's extent and energy window, and an oracle image and
    sensitivity of the support's size."""
    from paper_2002_12471_gb300 import synthetic as S
    G = np.load(os.path.join(HERE, "golden", "dat128_subset_oracle.npz"))
    ph, g, J, ns, ni = S.workload("dat128")
    np.testing.assert_allclose(G["mu"], ph.mu, rtol=0, atol=1e-15)
    for name in ("caudate", "putamen"):
        np.testing.assert_allclose(G["roi_" + name], ph.rois[name], rtol=0, atol=1e-6)
    gd = dict(zip(G["geometry_keys"].tolist(), G["geometry_values"].tolist()))
    assert gd == {k: float(v) for k, v in g.items()}
    assert (int(G["n_subsets"]), int(G["n_iters"]), float(G["pixel_mm"])) == (ns, ni, ph.pixel_mm)
    half = 0.5 * g["n_bins"] * g["bin_mm"]
    assert np.all(np.abs(G["u_mm"]) <= half)
    assert np.all((G["e_kev"] >= g["e_lo_kev"]) & (G["e_kev"] <= g["e_hi_kev"]))
    assert np.all((G["angle"] >= 0) & (G["angle"] < g["n_angles"]))
    assert np.array_equal(G["support"], np.nonzero(ph.mu.reshape(-1) > 0)[0])
    n_sup = len(G["support"])
    assert G["image"].shape == (n_sup,) and G["sens"].shape == (ns, n_sup)
    assert np.all(G["image"] >= 0) and np.all(np.isfinite(G["loglik"]))
