"""Writes tests/golden/dat128_subset_oracle.npz from the oracle alone.

The precision form's workload is the 128 x 128 DaT-like brain at 2 mm with
1,000,000 events (120 angles x 128 bins of 2 mm, R = 150 mm, 8 subsets x 10
iterations).  An FP64 oracle reconstruction of all of it is out of reach on a
CPU, so this script freezes a seeded subset of 20,000 of those events, stored
verbatim with the mu-map and the striatal ROI weights, and the oracle's
outputs on it: the subset sensitivities (denominator of Eq. 7), the image
after 10 OS-LM-MLEM iterations over 8 subsets (Eqs. 7-8) and the
log-likelihood after every iteration (Eq. 3 without log J!).  The GPU tests
and the benchmark reconstruct the same events in every model format and
report their error against this image.

Run:  python tests/golden/make_dat128_subset.py      (about 15 minutes on 8 cores)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2002_12471_gb300 import synthetic as S  # noqa: E402

J_SUBSET = 20_000
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dat128_subset_oracle.npz")


def main():
    t0 = time.time()
    ph, g, J, ns, ni = S.workload("dat128")
    ev = S.simulate_events(ph, g, J, seed=3)          # the full 1M-event set
    rng = np.random.default_rng(128)
    pick = np.sort(rng.choice(J, J_SUBSET, replace=False))
    a, u, e = ev.angle[pick], ev.u_mm[pick], ev.e_kev[pick]
    P = oracle.Problem(dict(g, pixel_mm=ph.pixel_mm), ph.mu)
    s = P.sensitivity(ns)
    p = P.model(a, u, e)
    f0 = oracle.initial_image(J_SUBSET, s.sum(0))
    f, hist = oracle.osem(p, a, s, ni, f0)
    ll = np.array([oracle.loglik(p, h, s.sum(0)) for h in hist])
    np.savez_compressed(
        OUT,
        case=np.array("128x128 DaT-like brain at 2 mm, 120 angles x 128 bins x 2 mm, R = 150 mm, "
                      "window 100-175 keV, 10%% FWHM at 159 keV; %d events picked (seed 128) from "
                      "the 1,000,000 events of seed 3; 8 subsets x 10 iterations, T = 1" % J_SUBSET),
        geometry_keys=np.array(sorted(g)), geometry_values=np.array([float(g[k]) for k in sorted(g)]),
        pixel_mm=np.float64(ph.pixel_mm), mu=ph.mu.astype(np.float64),
        roi_caudate=ph.rois["caudate"].astype(np.float32), roi_putamen=ph.rois["putamen"].astype(np.float32),
        angle=a.astype(np.int16), u_mm=u.astype(np.float32), e_kev=e.astype(np.float32),
        n_subsets=np.int32(ns), n_iters=np.int32(ni), support=P.support.astype(np.int32),
        sens=s.astype(np.float32), image=f, loglik=ll)
    print("wrote %s in %.0f s" % (OUT, time.time() - t0))


if __name__ == "__main__":
    main()
