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
