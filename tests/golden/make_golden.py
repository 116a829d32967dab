"""Writes tests/golden/tiny16_oracle.json from the oracle alone.

The fixture freezes a small, fully specified case (the 16 x 16 disk phantom
with two hot disks, 32 angles, 300 events stored verbatim) and the oracle's
outputs on it: the subset sensitivities, sampled model entries, the image
after 5 OS-LM-MLEM iterations over 4 subsets (Eqs. 7-8) and the
log-likelihood (Eq. 3 without log J!).  A later change of the oracle's
arithmetic shows up as a failure of tests/test_golden.py.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2002_12471_gb300 import synthetic as S  # noqa: E402


def main():
    ph, g, _, ns, ni = S.workload("tiny16")
    g = dict(g, pixel_mm=ph.pixel_mm)
    ev = S.simulate_events(ph, g, 300, seed=1)
    P = oracle.Problem(g, ph.mu)
    p = P.model(ev.angle, ev.u_mm, ev.e_kev)
    s = P.sensitivity(ns)
    f0 = oracle.initial_image(len(ev), s.sum(0))
    f, hist = oracle.osem(p, ev.angle, s, ni, f0)
    ll = [oracle.loglik(p, h, s.sum(0)) for h in hist]
    rng = np.random.default_rng(0)
    jj = rng.integers(0, p.shape[0], 40)
    qq = rng.integers(0, p.shape[1], 40)
    out = {
        "case": "16x16 disk phantom, 8 mm pixels, 32 angles, 16 x 8 mm detector, R = 80 mm, "
                "window 100-175 keV, 10% FWHM at 159 keV, 4 subsets x 5 iterations, T = 1",
        "geometry": g,
        "mu": ph.mu.tolist(),
        "events": {"angle": ev.angle.tolist(), "u_mm": [float(x) for x in ev.u_mm],
                   "e_kev": [float(x) for x in ev.e_kev]},
        "support": P.support.tolist(),
        "sens": s.tolist(),
        "model_samples": [[int(j), int(q), float(p[j, q])] for j, q in zip(jj, qq)],
        "row_sums": p.sum(1).tolist(),
        "image": f.tolist(),
        "loglik": ll,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny16_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=None, separators=(",", ":"))
    print("wrote", path)


if __name__ == "__main__":
    main()
