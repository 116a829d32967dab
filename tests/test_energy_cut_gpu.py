"""The energy cut of the path sum (lmosem_options.e_sigma) on the GPU.

A scatter term of paper Eq. 2 (with Eq. 4) is dropped for an event whose
energy lies more than e_sigma energy sigmas from the Compton energy E' of
every path (n', m) of the support pixel's 128-column tile; each dropped term
is then below 2^(-e_sigma^2 log2(e) / 2) of its value at the peak (1.5e-8
at the default 6).  These tests pin the cut's three properties:
* with e_sigma < 0 the kernels count exactly the terms the host enumerates
  (the position strip only), so the count the benchmark's roofline divides
  is the one the kernels formed;
* the cut's machinery (energy hulls, staged per scatter pixel) leaves every
  row bit unchanged when it drops nothing (e_sigma = 20: every event lies
  inside every hull that has a path);
* the default cut moves no entry by more than 1e-6 of its row maximum (the
  parity bound's floor is 2e-6), and drops a measurable share of the terms.
The workload (32 x 32 brain, 60 angles, 20,000 events) runs the wide, the
narrow and the tail forms of the path sum and ragged event tiles."""
import numpy as np
import pytest

import bench
import oracle
from paper_2002_12471_gb300 import synthetic as S
from tests._helpers import gpu_reconstruct

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def dat32():
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, J, seed=5)
    return ph, g, ev, ns, ni


@pytest.fixture(scope="module")
def exact(dat32):
    ph, g, ev, ns, ni = dat32
    return gpu_reconstruct(ph, g, ev, ns, ni, rows=np.arange(len(ev)), e_sigma=-1.0)


def test_exact_sum_counts_the_enumerated_terms(dat32, exact):
    ph, g, ev, ns, ni = dat32
    terms, _ = bench.strip_terms(ph, g, ev)
    # FP32 against FP64 strip bounds: an event on a cut boundary may fall
    # either side
    assert abs(exact["terms"] - terms) <= 1e-6 * terms, (exact["terms"], terms)


def test_cut_machinery_leaves_rows_bitwise_unchanged(dat32, exact):
    ph, g, ev, ns, ni = dat32
    wide = gpu_reconstruct(ph, g, ev, ns, ni, rows=np.arange(len(ev)), e_sigma=20.0)
    assert wide["terms"] <= exact["terms"]   # (m, tile) pairs without a path count no terms
    assert np.array_equal(wide["rows"], exact["rows"])
    assert np.array_equal(wide["f"], exact["f"])


def test_default_cut_moves_entries_below_the_bound(dat32, exact):
    ph, g, ev, ns, ni = dat32
    cut = gpu_reconstruct(ph, g, ev, ns, ni, rows=np.arange(len(ev)))
    p, q = cut["rows"], exact["rows"]
    dev = np.max(np.abs(p - q) / q.max(axis=1, keepdims=True))
    assert dev <= 1e-6, dev
    assert cut["terms"] < 0.97 * exact["terms"], (cut["terms"], exact["terms"])
    assert oracle.rel_l2(cut["f"], exact["f"]) <= 1e-6
