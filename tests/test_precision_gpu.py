"""Precision form on the 128 x 128 / 2 mm DaT workload with 1,000,000 events:
the model cached as FP16 (max_n h = 2^15) or BF16 with per-event FP32 scales,
FP32 accumulation, FP64 sensitivity and log-likelihood.

* sampled FP32 model rows against the FP64 oracle computed one by one;
* the dequantised FP16/BF16 rows against the FP32 rows: each entry within the
  format's rounding (2^-11 or 2^-8 relative) of its value, entries below the
  FP16 normal range of the row excepted;
* the reduced-precision reconstructions against the FP32 one (rel-L2 <= 1e-2,
  striatal ROI means within 1%).  A full FP64 oracle reconstruction at 1M x
  6k entries is out of reach; the FP32 path it is compared with matches the
  oracle to 1e-4 rel-L2 on the smaller workloads (test_parity_gpu.py).
"""
import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S
from tests._helpers import gpu_reconstruct, oracle_problem, row_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dat128():
    import __graft_entry__
    __graft_entry__.build()
    ph, g, J, ns, ni = S.workload("dat128")
    ev = S.simulate_events(ph, g, J, seed=3)
    rng = np.random.default_rng(3)
    rows = np.concatenate([rng.choice(np.nonzero(ev.angle == a)[0], 8, replace=False)
                           for a in (7, 64, 101)])
    out32 = gpu_reconstruct(ph, g, ev, ns, ni, rows=rows)
    return dict(ph=ph, g=g, ev=ev, ns=ns, ni=ni, rows=rows, out32=out32)


def test_dat128_fp32_rows_match_oracle(dat128):
    d = dat128
    P = oracle_problem(d["ph"], d["g"])
    ev, rows = d["ev"], d["rows"]
    p = P.model(ev.angle[rows], ev.u_mm[rows], ev.e_kev[rows])
    assert np.array_equal(d["out32"]["support"], P.support)
    assert row_close(d["out32"]["rows"], p) <= 1.0


@pytest.mark.parametrize("fmt,rel", [("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_dat128_reduced_precision_forms(dat128, fmt, rel):
    d = dat128
    out = gpu_reconstruct(d["ph"], d["g"], d["ev"], d["ns"], d["ni"], fmt=fmt, rows=d["rows"])
    p32 = d["out32"]["rows"]
    rmax = p32.max(axis=1, keepdims=True)
    floor = (6.2e-5 / 32768.0) * rmax if fmt == "fp16" else 1e-30
    assert np.all(np.abs(out["rows"] - p32) <= rel * np.abs(p32) * 1.001 + floor + 1e-6 * rel * rmax)
    f32 = d["out32"]["f"]
    assert oracle.rel_l2(out["f"], f32) <= 1e-2
    ph = d["ph"]
    img, ref = np.zeros(ph.mu.size), np.zeros(ph.mu.size)
    img[out["support"]] = out["f"]
    ref[d["out32"]["support"]] = f32
    for name, roi in ph.rois.items():
        w = roi.reshape(-1)
        assert np.dot(w, img) == pytest.approx(np.dot(w, ref), rel=1e-2), name
    assert out["model_bytes"] < 0.55 * d["out32"]["model_bytes"]
