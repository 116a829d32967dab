"""The precision form's reconstructions carry their error against the FP64
oracle (paper Eqs. 7-8 at 128 x 128).

The 128 x 128 DaT-like brain at 2 mm, 120 angles x 128 bins of 2 mm: the
oracle's reconstruction of 20,000 of the workload's 1,000,000 events (8
subsets x 10 iterations) is frozen in tests/golden/dat128_subset_oracle.npz
(written by tests/golden/make_dat128_subset.py from the oracle alone, with
the events stored verbatim).  The CUDA path reconstructs the same events
with every model format.  N_nz = 6016, so the rows are 6016 wide and the
passes run the same kernel instances as the full-size workload: FP32 rows
take the cp.async pass with 6 vectors per thread, FP16 and BF16 rows the
register pass with 3.

* FP32 model: image rel-L2 <= 1e-4, log-likelihood of every iteration within
  1e-6, subset sensitivities within 1e-5;
* FP16 and BF16 model with per-event FP32 scales: image rel-L2 <= 1e-2 and
  striatal ROI means within 1%.
"""
import os
import types

import numpy as np
import pytest

import oracle
from tests._helpers import gpu_reconstruct

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dat128_subset_oracle.npz")


@pytest.fixture(scope="module")
def golden():
    import __graft_entry__
    __graft_entry__.build()
    G = dict(np.load(GOLDEN))
    g = {k: float(v) for k, v in zip(G["geometry_keys"], G["geometry_values"])}
    g["n_angles"], g["n_bins"] = int(g["n_angles"]), int(g["n_bins"])
    ev = types.SimpleNamespace(angle=G["angle"].astype(np.int32), u_mm=G["u_mm"], e_kev=G["e_kev"])
    ph = types.SimpleNamespace(mu=G["mu"], pixel_mm=float(G["pixel_mm"]))
    ref = np.zeros(G["mu"].size)
    ref[G["support"]] = G["image"]
    return dict(G=G, g=g, ev=ev, ph=ph, ref=ref)


def _roi(img, G, name):
    w = G["roi_" + name].reshape(-1).astype(np.float64)
    return float(np.dot(w, img) / w.sum())


def _run(golden, fmt):
    G = golden["G"]
    out = gpu_reconstruct(golden["ph"], golden["g"], golden["ev"], int(G["n_subsets"]),
                          int(G["n_iters"]), fmt=fmt, loglik=True)
    assert np.array_equal(out["support"], G["support"])
    img = np.zeros(G["mu"].size)
    img[G["support"]] = out["f"]
    return out, img


def test_dat128_fp32_reconstruction_matches_oracle(golden):
    G = golden["G"]
    out, img = _run(golden, "fp32")
    np.testing.assert_allclose(out["sens"], G["sens"].astype(np.float64), rtol=1e-5)
    assert oracle.rel_l2(img, golden["ref"]) <= 1e-4
    np.testing.assert_allclose(out["loglik"], G["loglik"], rtol=1e-6)


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_dat128_reduced_precision_reconstruction_against_oracle(golden, fmt):
    G = golden["G"]
    out, img = _run(golden, fmt)
    assert oracle.rel_l2(img, golden["ref"]) <= 1e-2
    for name in ("caudate", "putamen"):
        assert _roi(img, G, name) == pytest.approx(_roi(golden["ref"], G, name), rel=1e-2), name
