"""GPU parity of the binned form (the paper's binning experiment, Section
4) against the FP64 oracle: the bin-integrated model rows, the count-weighted
reconstruction and log-likelihood, the bin sums against the sensitivity,
and the argument checks."""
import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S
from tests._helpers import oracle_problem, row_close

pytestmark = pytest.mark.gpu

EDGES2 = (100.0, 143.0, 175.0)
EDGES3 = (100.0, 120.0, 143.0, 175.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _positive_bins(counts):
    """(angle, position bin, energy bin, count) of the positive bins in dense order."""
    a, b, k = np.nonzero(counts > 0)
    return a, b, k, counts[a, b, k].astype(np.float64)


def gpu_binned(ph, g, counts, edges, n_subsets, n_iters, rows=None, T=1.0, **opts):
    import torch

    import paper_2002_12471_gb300.lmosem as L
    dev = torch.device("cuda:0")
    out = {}
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream(), **opts)
    try:
        nsup = L.lmosem_n_support(ctx)
        sens = torch.zeros((n_subsets, nsup), dtype=torch.float64, device=dev)
        L.lmosem_sensitivity(ctx, n_subsets, sens)
        L.lmosem_build_model_binned(ctx, torch.from_numpy(counts).to(dev), edges, n_subsets)
        if rows is not None:
            ids = torch.as_tensor(np.asarray(rows, dtype=np.int64), device=dev)
            buf = torch.zeros((len(rows), nsup), dtype=torch.float32, device=dev)
            L.lmosem_model_rows(ctx, ids, buf)
            out["rows"] = buf.cpu().numpy().astype(np.float64)
        f = torch.zeros(nsup, dtype=torch.float32, device=dev)
        L.lmosem_init_image(ctx, T, f)
        out["f0"] = f.cpu().numpy().astype(np.float64)
        ll = torch.zeros(max(1, n_iters), dtype=torch.float64, device=dev)
        L.lmosem_iterate(ctx, n_iters, T, f, ll)
        torch.cuda.synchronize()
        out["f"] = f.cpu().numpy().astype(np.float64)
        out["loglik"] = ll.cpu().numpy()
        out["sens"] = sens.cpu().numpy()
        out["launches"] = L.lmosem_launch_count(ctx)
    finally:
        L.lmosem_destroy(ctx)
    return out


def _oracle_binned(P, counts, edges, ns, ni, T=1.0):
    a, b, k, w = _positive_bins(counts)
    p = P.model_binned(a, b, k, edges)
    s = P.sensitivity(ns)
    f0 = oracle.initial_image(w.sum(), s.sum(0), T)
    f, hist = oracle.osem(p, a, s, ni, f0, T, weights=w)
    ll = [oracle.loglik(p, h, s.sum(0), T, weights=w) for h in hist]
    return p, s, f0, f, ll


@pytest.mark.parametrize("edges", [EDGES2, EDGES3])
def test_tiny16_binned_parity(edges):
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, J, seed=1)
    counts = S.bin_events(ev, g, edges)
    P = oracle_problem(ph, g)
    p, s, f0, f_ref, ll_ref = _oracle_binned(P, counts, edges, ns, ni)
    out = gpu_binned(ph, g, counts, edges, ns, ni, rows=np.arange(len(p)))
    assert row_close(out["rows"], p) <= 1.0
    np.testing.assert_allclose(out["f0"], f0, rtol=1e-6)
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4
    # the likelihood is a small difference of large sums: FP32 y_i carry ~1e-6
    # relative error, i.e. ~1e-6 in log y_i per counted photon
    np.testing.assert_allclose(out["loglik"], ll_ref, rtol=1e-6, atol=1e-6 * counts.sum())


def test_dat32_binned_ragged_tiles():
    # 404 support pixels (a 20-column last tile), 60 angles x 32 bins x 3 energy bins
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, J, seed=5)
    counts = S.bin_events(ev, g, EDGES3)
    P = oracle_problem(ph, g)
    p, s, f0, f_ref, ll_ref = _oracle_binned(P, counts, EDGES3, ns, 4)
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(len(p), 400, replace=False))
    out = gpu_binned(ph, g, counts, EDGES3, ns, 4, rows=rows)
    assert row_close(out["rows"], p[rows]) <= 1.0
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4
    np.testing.assert_allclose(out["loglik"], ll_ref, rtol=1e-6, atol=1e-6 * counts.sum())


def test_bin_rows_sum_to_the_gpu_sensitivity():
    """With a count in every bin, the rows of one angle add up to that angle's
    sensitivity (one angle per subset): the bins tile the detector extent and
    the window."""
    ph, g, J, ns, ni = S.workload("tiny16")
    na, nb = g["n_angles"], g["n_bins"]
    counts = np.ones((na, nb, 2), dtype=np.float32)
    out = gpu_binned(ph, g, counts, EDGES2, na, 0, rows=np.arange(na * nb * 2))
    tot = out["rows"].reshape(na, nb * 2, -1).sum(axis=1)
    np.testing.assert_allclose(tot, out["sens"], rtol=2e-5, atol=1e-7 * out["sens"].max())


def test_binned_table_paths_bitwise():
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, J, seed=6)
    counts = S.bin_events(ev, g, EDGES3)
    n = int((counts > 0).sum())
    a = gpu_binned(ph, g, counts, EDGES3, ns, 2, rows=np.arange(n))
    b = gpu_binned(ph, g, counts, EDGES3, ns, 2, rows=np.arange(n), table_budget_bytes=1 << 20)
    assert b["launches"] > a["launches"]
    assert np.array_equal(a["rows"], b["rows"]) and np.array_equal(a["f"], b["f"])


def test_binned_argument_checks():
    import torch

    import paper_2002_12471_gb300.lmosem as L
    ph, g, J, ns, ni = S.workload("tiny16")
    dev = torch.device("cuda:0")
    na, nb = g["n_angles"], g["n_bins"]
    good = torch.ones((na, nb, 2), dtype=torch.float32, device=dev)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream())
    try:
        L.lmosem_sensitivity(ctx, ns)
        cases = [
            (good, (110.0, 143.0, 175.0), ns, "fp32", L.EINVAL),    # does not start at e_lo
            (good, (100.0, 143.0, 170.0), ns, "fp32", L.EINVAL),    # does not end at e_hi
            (good, (100.0, 143.0, 143.0, 175.0), ns, "fp32", L.EINVAL),  # not increasing
            (good, EDGES2, ns, "fp16", L.ENOTIMPL),
            (good, EDGES2, 0, "fp32", L.EINVAL),
            (torch.zeros_like(good), EDGES2, ns, "fp32", L.EINVAL),     # no positive count
            (-good, EDGES2, ns, "fp32", L.EINVAL),
            (good.new_full(good.shape, float("nan")), EDGES2, ns, "fp32", L.EINVAL),
        ]
        for counts, edges, nsub, fmt, want in cases:
            with pytest.raises(L.LmosemError) as ei:
                L.lmosem_build_model_binned(ctx, counts, edges, nsub, fmt)
            assert ei.value.status == want, (edges, nsub, fmt)
        # the context still builds a binned model afterwards
        L.lmosem_build_model_binned(ctx, good, EDGES2, ns)
        f = torch.zeros(L.lmosem_n_support(ctx), dtype=torch.float32, device=dev)
        L.lmosem_init_image(ctx, 1.0, f)
        L.lmosem_iterate(ctx, 1, 1.0, f)
        assert bool(torch.isfinite(f).all())
    finally:
        L.lmosem_destroy(ctx)

