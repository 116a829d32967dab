"""The binned form at the full 64 x 64 size (the paper's binning experiment,
Section 4), in the launch configuration the benchmark times: sampled bin rows
against the oracle's bin-integrated model, computed one by one, and the count
conservation of the last sub-iteration.  A full-size case, so it is
collected after the smaller parity files."""
import numpy as np
import pytest

from paper_2002_12471_gb300 import synthetic as S
from tests._helpers import oracle_problem, row_close
from tests.test_binned_gpu import EDGES3, _positive_bins, gpu_binned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def full_size_binned_check(wl, seed, run=None):
    """Sampled bin rows of the workload against the oracle's bin-integrated
    model, computed one by one, and the count conservation of the last
    sub-iteration after one iteration: its T s.f equals the counts of its
    bins whose model row is not all zero.  ``run`` builds and iterates
    (default: the GPU path)."""
    run = run or gpu_binned
    ph, g, J, ns, ni = S.workload(wl)
    ev = S.simulate_events(ph, g, J, seed=seed)
    counts = S.bin_events(ev, g, EDGES3)
    a, b, k, w = _positive_bins(counts)
    rng = np.random.default_rng(5)
    pick = rng.choice(g["n_angles"], 6, replace=False)
    sampled = np.sort(np.concatenate([rng.choice(np.nonzero(a == ang)[0], 8, replace=False)
                                      for ang in pick]))
    last = np.nonzero(a % ns == ns - 1)[0]
    rows = np.union1d(sampled, last)
    out = run(ph, g, counts, EDGES3, ns, 1, rows=rows)
    R = out["rows"]
    P = oracle_problem(ph, g)
    p = P.model_binned(a[sampled], b[sampled], k[sampled], EDGES3)
    assert row_close(R[np.searchsorted(rows, sampled)], p) <= 1.0
    R_last = R[np.searchsorted(rows, last)]
    want = float(np.sum(w[last][R_last.max(axis=1) > 0]))
    assert np.dot(out["sens"][ns - 1], out["f"]) == pytest.approx(want, rel=1e-4)


def test_dat64_binned_full_size_sampled_rows_and_count_conservation():
    """64 x 64 DaT phantom, 120 angles x 64 position bins x 3 energy bins
    from 200k events, 8 subsets."""
    full_size_binned_check("dat64", 7)
