"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (derived from the arithmetic of each step):
* model entries: |p_gpu - p_orc| <= 2e-4 |p_orc| + 2e-6 max_n p_orc  (FP32
  terms with MUFU ex2, ~10^3-term FP32 sums, FP32 line integrals, and the
  6-sigma strip of the kernel, which moves entries by < 3e-7 of the row max);
* sensitivities: 1e-5 relative (FP32 terms, FP64 accumulation);
* reconstructed image, plain FP32 form: rel-L2 <= 1e-4;
* FP16 / BF16 cached forms: rel-L2 <= 1e-2 and striatal-ROI means within 1%.
"""
import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S
from tests._helpers import gpu_reconstruct, oracle_problem, row_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()


def _oracle_recon(P, ev, ns, ni, T=1.0):
    p = P.model(ev.angle, ev.u_mm, ev.e_kev)
    s = P.sensitivity(ns)
    f, hist = oracle.osem(p, ev.angle, s, ni, oracle.initial_image(len(ev), s.sum(0), T), T)
    return p, s, f, hist


def test_tiny16_full_parity():
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, J, seed=1)
    P = oracle_problem(ph, g)
    p, s, f_ref, hist = _oracle_recon(P, ev, ns, ni)
    out = gpu_reconstruct(ph, g, ev, ns, ni, rows=np.arange(J), loglik=True)
    assert np.array_equal(out["support"], P.support)
    assert row_close(out["rows"], p) <= 1.0
    np.testing.assert_allclose(out["sens"], s, rtol=1e-5)
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4
    ll_ref = [oracle.loglik(p, h, s.sum(0)) for h in hist]
    np.testing.assert_allclose(out["loglik"], ll_ref, rtol=1e-6)


def test_dat32_several_tiles_and_ragged_tails():
    # 32 x 32 brain, 60 angles, 20k events: ~330 events per angle (ragged 64-event
    # tiles), support of ~370 pixels (ragged 128-pixel tiles), 6 subsets
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, J, seed=5)
    P = oracle_problem(ph, g)
    p, s, f_ref, _ = _oracle_recon(P, ev, ns, ni)
    rng = np.random.default_rng(0)
    rows = rng.choice(J, 600, replace=False)
    out = gpu_reconstruct(ph, g, ev, ns, ni, rows=rows)
    assert row_close(out["rows"], p[rows]) <= 1.0
    np.testing.assert_allclose(out["sens"], s, rtol=1e-5)
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4


def test_reconstruct_from_host_buffers_matches_device_path():
    """lmosem_reconstruct (host events in, host image and log-likelihood out)
    runs the device-pointer calls' kernels in the same order, so its image is
    bitwise theirs; pinned and pageable inputs give the same bits, and an
    argument error leaves the context usable."""
    import torch

    import paper_2002_12471_gb300.lmosem as L

    ph, g, _, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, 4000, seed=9)
    ref = gpu_reconstruct(ph, g, ev, ns, ni)
    P = oracle_problem(ph, g)
    p, s, f_orc, _ = _oracle_recon(P, ev, ns, ni)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream())
    try:
        a = torch.from_numpy(np.ascontiguousarray(ev.angle)).pin_memory()
        u = torch.from_numpy(np.ascontiguousarray(ev.u_mm)).pin_memory()
        e = torch.from_numpy(np.ascontiguousarray(ev.e_kev)).pin_memory()
        f_h = torch.empty(L.lmosem_n_support(ctx), dtype=torch.float32).pin_memory()
        ll_h = torch.empty(1, dtype=torch.float64).pin_memory()
        f, ll = L.lmosem_reconstruct(ctx, a, u, e, ns, ni, 1.0, "fp32", f_h, ll_h)
        f = f.numpy().astype(np.float64)
        assert np.array_equal(f, ref["f"])
        assert oracle.rel_l2(f, f_orc) <= 1e-4
        assert float(ll[0]) == pytest.approx(oracle.loglik(p, f, s.sum(0)), rel=1e-6)
        with pytest.raises(L.LmosemError):
            L.lmosem_reconstruct(ctx, ev.angle[:0], ev.u_mm[:0], ev.e_kev[:0], ns, ni)
        with pytest.raises(L.LmosemError):
            L.lmosem_reconstruct(ctx, ev.angle, ev.u_mm, ev.e_kev, ns, ni, acq_time=0.0)
        f2, ll2 = L.lmosem_reconstruct(ctx, ev.angle, ev.u_mm, ev.e_kev, ns, ni)
        assert np.array_equal(f2.astype(np.float64), f)
        assert float(ll2[0]) == float(ll[0])
    finally:
        L.lmosem_destroy(ctx)


def test_dat64_full_size_sampled_rows_and_invariants():
    """The 64 x 64 DaT workload at full size (200k events, 120 angles, 8
    subsets), in the launch configuration the benchmark times: sampled model
    rows against the oracle computed one by one, the full sensitivity, and
    count conservation of the last sub-iteration."""
    ph, g, J, ns, ni = S.workload("dat64")
    ev = S.simulate_events(ph, g, J, seed=2)
    rng = np.random.default_rng(1)
    ang_pick = rng.choice(g["n_angles"], 6, replace=False)
    rows = np.concatenate([rng.choice(np.nonzero(ev.angle == a)[0], 8, replace=False) for a in ang_pick])
    out = gpu_reconstruct(ph, g, ev, ns, 1, rows=rows)
    P = oracle_problem(ph, g)
    p = P.model(ev.angle[rows], ev.u_mm[rows], ev.e_kev[rows])
    assert row_close(out["rows"], p) <= 1.0
    s = P.sensitivity(ns)
    np.testing.assert_allclose(out["sens"], s, rtol=1e-5)
    # after a full iteration the last subset's update reproduces its counts
    last = int(np.sum(ev.angle % ns == ns - 1))
    assert np.dot(out["sens"][ns - 1], out["f"]) == pytest.approx(last, rel=1e-4)


@pytest.mark.parametrize("wl,J", [("tiny16", 2000), ("dat32", 9000)])
def test_subset_totals_count_conservation(wl, J):
    """lmosem_subset_totals after an iteration: the last subset's expected
    count T s^i . f equals its number of events (Eq. 7 conserves counts),
    and every subset's total is the FP64 dot product of the returned
    sensitivity and image."""
    import torch

    import paper_2002_12471_gb300.lmosem as L
    ph, g, _, ns, ni = S.workload(wl)
    ev = S.simulate_events(ph, g, J, seed=17)
    dev = torch.device("cuda:0")
    T = 2.5
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream())
    try:
        nsup = L.lmosem_n_support(ctx)
        sens = torch.zeros((ns, nsup), dtype=torch.float64, device=dev)
        L.lmosem_sensitivity(ctx, ns, sens)
        L.lmosem_build_model(ctx, *(torch.from_numpy(x).to(dev) for x in (ev.angle, ev.u_mm, ev.e_kev)), ns)
        f = torch.zeros(nsup, dtype=torch.float32, device=dev)
        L.lmosem_init_image(ctx, T, f)
        L.lmosem_iterate(ctx, 2, T, f)
        tot = torch.zeros(ns, dtype=torch.float64, device=dev)
        L.lmosem_subset_totals(ctx, T, f, tot)
        torch.cuda.synchronize()
        tot = tot.cpu().numpy()
        ref = T * sens.cpu().numpy() @ f.double().cpu().numpy()
        np.testing.assert_allclose(tot, ref, rtol=1e-12)
        n_last = int(np.sum(ev.angle % ns == ns - 1))
        assert tot[ns - 1] == pytest.approx(n_last, rel=1e-5)
    finally:
        L.lmosem_destroy(ctx)


def test_mlem_loglik_monotone_on_gpu():
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, 3000, seed=9)
    out = gpu_reconstruct(ph, g, ev, 1, 12, loglik=True)
    ll = out["loglik"]
    assert np.all(np.diff(ll) >= -1e-9 * np.abs(ll[1:]))


def test_explicit_support_with_air_pixels():
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, 1500, seed=4)
    supp = (ph.mu > 0).copy()
    supp[0, 5:9] = True   # air pixels inside the support
    supp[8, 8] = False     # a tissue pixel outside it (still a scatter site)
    P = oracle_problem(ph, g, support=supp)
    p, s, f_ref, _ = _oracle_recon(P, ev, ns, ni)
    out = gpu_reconstruct(ph, g, ev, ns, ni, support=supp, rows=np.arange(200))
    assert np.array_equal(out["support"], P.support)
    assert row_close(out["rows"], p[:200]) <= 1.0
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4


def test_degenerate_inputs():
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, 400, seed=6)
    # one event
    one = S.Events(ev.angle[:1], ev.u_mm[:1], ev.e_kev[:1], ev.order[:1])
    P = oracle_problem(ph, g)
    p, s, f_ref, _ = _oracle_recon(P, one, 1, 3)
    out = gpu_reconstruct(ph, g, one, 1, 3, rows=[0])
    assert row_close(out["rows"], p) <= 1.0
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4
    # every event at one angle: the other subsets are empty and, by Eq. 7,
    # zero the image; both sides agree on that
    same = S.Events(np.full(len(ev), 3, dtype=np.int32), ev.u_mm, ev.e_kev, ev.order)
    p, s, f_ref, _ = _oracle_recon(P, same, 4, 1)
    out = gpu_reconstruct(ph, g, same, 4, 1)
    assert np.all(f_ref == 0) and np.all(out["f"] == 0)
    # ...while one subset holding that angle reconstructs normally
    p, s, f_ref, _ = _oracle_recon(P, same, 1, 4)
    out = gpu_reconstruct(ph, g, same, 1, 4)
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4
    # events at the extremes of the detector and the energy window
    half = np.float32(0.5 * g["n_bins"] * g["bin_mm"])
    edge = S.Events(np.array([0, 5, 31, 16], dtype=np.int32),
                    np.array([-half, half, 0.0, 63.9], dtype=np.float32),
                    np.array([100.0, 175.0, 159.0, 100.0], dtype=np.float32), np.zeros(4, np.int8))
    p = P.model(edge.angle, edge.u_mm, edge.e_kev)
    out = gpu_reconstruct(ph, g, edge, 1, 1, rows=np.arange(4))
    assert row_close(out["rows"], p) <= 1.0


def test_invalid_events_are_rejected():
    import torch

    import paper_2002_12471_gb300.lmosem as L
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, 100, seed=3)
    dev = torch.device("cuda:0")
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g)
    try:
        def build(a, u, e, nsub=4):
            L.lmosem_build_model(ctx, torch.as_tensor(a, device=dev), torch.as_tensor(u, device=dev),
                                 torch.as_tensor(e, device=dev), nsub)
        bad_a = ev.angle.copy(); bad_a[7] = 32
        bad_u = ev.u_mm.copy(); bad_u[3] = 64.5
        bad_e = ev.e_kev.copy(); bad_e[9] = 99.0
        nan_e = ev.e_kev.copy(); nan_e[1] = np.nan
        for a, u, e in ((bad_a, ev.u_mm, ev.e_kev), (ev.angle, bad_u, ev.e_kev),
                        (ev.angle, ev.u_mm, bad_e), (ev.angle, ev.u_mm, nan_e)):
            with pytest.raises(L.LmosemError) as ei:
                build(a, u, e)
            assert ei.value.status == L.EINVAL
        with pytest.raises(L.LmosemError) as ei:
            build(ev.angle, ev.u_mm, ev.e_kev, nsub=33)
        assert ei.value.status == L.EINVAL
        # iterate before a model exists
        f = torch.zeros(L.lmosem_n_support(ctx), device=dev)
        with pytest.raises(L.LmosemError) as ei:
            L.lmosem_iterate(ctx, 1, 1.0, f)
        assert ei.value.status == L.ESTATE
        # a model without a matching sensitivity
        build(ev.angle, ev.u_mm, ev.e_kev, nsub=4)
        L.lmosem_sensitivity(ctx, 2)
        with pytest.raises(L.LmosemError) as ei:
            L.lmosem_iterate(ctx, 1, 1.0, f)
        assert ei.value.status == L.ESTATE
    finally:
        L.lmosem_destroy(ctx)


def test_bitwise_deterministic():
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, 8000, seed=8)
    a = gpu_reconstruct(ph, g, ev, ns, 3, rows=np.arange(50))
    b = gpu_reconstruct(ph, g, ev, ns, 3, rows=np.arange(50))
    assert np.array_equal(a["f"], b["f"]) and np.array_equal(a["rows"], b["rows"])
    # the event order does not change the model rows
    perm = np.random.default_rng(2).permutation(len(ev))
    evp = S.Events(ev.angle[perm], ev.u_mm[perm], ev.e_kev[perm], ev.order[perm])
    inv = np.argsort(perm)
    c = gpu_reconstruct(ph, g, evp, ns, 3, rows=inv[:50])
    assert np.array_equal(a["rows"], c["rows"])
    assert oracle.rel_l2(c["f"], a["f"]) <= 1e-5


@pytest.mark.parametrize("wl,J", [("tiny16", 2000), ("dat32", 6000)])
def test_table_paths_bitwise(wl, J):
    """The scatter tables and the sensitivity come out bitwise the same
    whether every angle's tables are built in the sensitivity pass (one
    fused kernel) or per angle group by the model build under a small table
    budget (separate table and sensitivity kernels)."""
    ph, g, _, ns, ni = S.workload(wl)
    ev = S.simulate_events(ph, g, J, seed=21)
    fused = gpu_reconstruct(ph, g, ev, ns, 2, rows=np.arange(J))
    grouped = gpu_reconstruct(ph, g, ev, ns, 2, rows=np.arange(J), table_budget_bytes=1 << 20)
    assert grouped["launches"] > fused["launches"]          # the grouped path did run
    assert np.array_equal(fused["sens"], grouped["sens"])
    assert np.array_equal(fused["rows"], grouped["rows"])
    assert np.array_equal(fused["f"], grouped["f"])


def test_graph_replay_matches_direct_launches():
    """On a non-default stream lmosem_iterate replays one captured iteration
    as a CUDA graph; the image is bitwise the one of direct launches."""
    import torch
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, 7000, seed=14)
    direct = gpu_reconstruct(ph, g, ev, ns, 4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        graphed = gpu_reconstruct(ph, g, ev, ns, 4)
    torch.cuda.synchronize()
    assert np.array_equal(direct["f"], graphed["f"])
    assert graphed["launches"] == direct["launches"]


@pytest.mark.parametrize("rows_stages", [(0, 0), (1, 2), (3, 5), (8, 8)])
def test_ring_pass_variant_matches_oracle(rows_stages):
    """The bulk-copy ring pass (several stage shapes, ragged row groups)
    gives the same reconstruction and log-likelihood as the oracle."""
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, 9001, seed=13)
    P = oracle_problem(ph, g)
    p, s, f_ref, hist = _oracle_recon(P, ev, ns, 3)
    out = gpu_reconstruct(ph, g, ev, ns, 3, loglik=True, pass_variant=2,
                          ring_rows=rows_stages[0], ring_stages=rows_stages[1])
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4
    ll_ref = [oracle.loglik(p, h, s.sum(0)) for h in hist]
    np.testing.assert_allclose(out["loglik"], ll_ref, rtol=1e-6)


def test_ring_pass_shape_is_cut_to_shared_memory():
    """A caller-chosen ring shape larger than a CTA's shared memory (8 rows x
    8 stages of 22.6 KB rows at 128 x 128) is cut to fit and reconstructs
    what the register pass does."""
    ph, g, J, ns, ni = S.workload("dat128")
    ev = S.simulate_events(ph, g, 3000, seed=14)
    ref = gpu_reconstruct(ph, g, ev, ns, 2)
    out = gpu_reconstruct(ph, g, ev, ns, 2, pass_variant=2, ring_rows=8, ring_stages=8)
    assert oracle.rel_l2(out["f"], ref["f"]) <= 1e-5


def test_wait_timeout_reports_etimeout_and_context_survives():
    """A bounded device wait that runs out (a one-cycle budget set after the
    model build; the bulk copies still complete and are drained) makes
    lmosem_iterate return LMOSEM_ETIMEOUT without touching the image, and the
    GPU stays usable."""
    import torch

    import paper_2002_12471_gb300.lmosem as L
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, 500, seed=12)
    dev = torch.device("cuda:0")
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, pass_variant=2)
    try:
        L.lmosem_sensitivity(ctx, 2)
        L.lmosem_build_model(ctx, torch.from_numpy(ev.angle).to(dev), torch.from_numpy(ev.u_mm).to(dev),
                             torch.from_numpy(ev.e_kev).to(dev), 2)
        f = torch.zeros(L.lmosem_n_support(ctx), dtype=torch.float32, device=dev)
        L.lmosem_init_image(ctx, 1.0, f)
        f0 = f.clone()
        L.lmosem_set_wait_budget(ctx, 1)
        for _ in range(2):
            with pytest.raises(L.LmosemError) as ei:
                L.lmosem_iterate(ctx, 1, 1.0, f)
            assert ei.value.status == L.ETIMEOUT
            assert torch.equal(f, f0)
    finally:
        L.lmosem_destroy(ctx)
    P = oracle_problem(ph, g)
    p, s, f_ref, _ = _oracle_recon(P, ev, 2, 2)
    out = gpu_reconstruct(ph, g, ev, 2, 2)
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4


def test_persistent_pass_barrier_timeout_and_variants_agree():
    """The persistent cooperative form (every sub-iteration in one launch,
    bounded grid barriers): a one-cycle wait budget makes lmosem_iterate
    return LMOSEM_ETIMEOUT and the context stays usable; with the default
    budget its images match those of the register pass (other reduction
    order, 1e-5) and of the FP64 oracle (1e-4), and two runs are bitwise
    equal."""
    import torch

    import paper_2002_12471_gb300.lmosem as L
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, 4000, seed=13)
    dev = torch.device("cuda:0")
    a, u, e = (torch.from_numpy(x).to(dev) for x in (ev.angle, ev.u_mm, ev.e_kev))
    images = {}
    for variant in (4, 1):
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, pass_variant=variant)
        try:
            L.lmosem_sensitivity(ctx, ns)
            L.lmosem_build_model(ctx, a, u, e, ns)
            f = torch.zeros(L.lmosem_n_support(ctx), dtype=torch.float32, device=dev)
            if variant == 4:
                L.lmosem_init_image(ctx, 1.0, f)
                L.lmosem_set_wait_budget(ctx, 1)
                with pytest.raises(L.LmosemError) as ei:
                    L.lmosem_iterate(ctx, 2, 1.0, f)
                assert ei.value.status == L.ETIMEOUT
                L.lmosem_set_wait_budget(ctx, 0)
            runs = []
            for _ in range(2):
                L.lmosem_init_image(ctx, 1.0, f)
                L.lmosem_iterate(ctx, ni, 1.0, f)
                runs.append(f.cpu().numpy().astype(np.float64))
            assert np.array_equal(runs[0], runs[1])
            images[variant] = runs[0]
        finally:
            L.lmosem_destroy(ctx)
    assert oracle.rel_l2(images[4], images[1]) <= 1e-5
    P = oracle_problem(ph, g)
    p, s, f_ref, _ = _oracle_recon(P, ev, ns, ni)
    assert oracle.rel_l2(images[4], f_ref) <= 1e-4


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_scaled_model_forms(fmt):
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, J, seed=5)
    P = oracle_problem(ph, g)
    p, s, f_ref, _ = _oracle_recon(P, ev, ns, ni)
    out = gpu_reconstruct(ph, g, ev, ns, ni, fmt=fmt)
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-2
    img = np.zeros(ph.mu.size)
    ref = np.zeros(ph.mu.size)
    img[out["support"]] = out["f"]
    ref[P.support] = f_ref
    for name, roi in ph.rois.items():
        w = roi.reshape(-1)
        assert np.dot(w, img) == pytest.approx(np.dot(w, ref), rel=1e-2), name


def test_largest_scatter_set():
    """The largest scatter-pixel set a context accepts (32,768 pixels with
    mu > 0, the shared-memory bound of the path-sum kernels): model rows and
    sensitivities against the oracle, with a small explicit support; one
    more scatter pixel is rejected at creation."""
    import torch

    import paper_2002_12471_gb300.lmosem as L
    n = 182                                  # 33,124 pixels
    mu = np.full((n, n), 0.0146)
    mu.reshape(-1)[: n * n - 32768] = 0.0    # leaves exactly 32,768 scatter pixels
    yy, xx = np.mgrid[0:n, 0:n]
    support = (xx - 100.5) ** 2 + (yy - 90.5) ** 2 <= 9.7 ** 2
    g = S.geometry(8, 96, 3.0, 150.0)
    pixel_mm = 1.0
    rng = np.random.default_rng(23)
    J = 120
    angle = rng.integers(0, 8, J).astype(np.int32)
    u = rng.uniform(-30.0, 30.0, J).astype(np.float32)
    e = rng.uniform(100.0, 175.0, J).astype(np.float32)
    ev = S.Events(angle, u, e, np.zeros(J, dtype=np.int8))
    ph = S.Phantom(mu=mu, activity=np.zeros_like(mu), pixel_mm=pixel_mm, rois={})
    out = gpu_reconstruct(ph, g, ev, 4, 1, support=support, rows=np.arange(J))
    P = oracle_problem(ph, g, support=support)
    assert P.n_sup == int(support.sum()) and len(P.scatter) == 32768
    assert row_close(out["rows"], P.model(angle, u, e)) <= 1.0
    np.testing.assert_allclose(out["sens"], P.sensitivity(4), rtol=1e-5)
    mu2 = mu.copy()
    mu2.reshape(-1)[0] = 0.0146              # 32,769 scatter pixels
    with pytest.raises(L.LmosemError) as ei:
        L.lmosem_create(mu2, pixel_mm, g, support=support)
    assert ei.value.status == L.EINVAL


@pytest.mark.parametrize("extra", [1, 6, 15])
def test_short_last_column_tile(extra):
    """Supports of 128 + extra pixels: the last column tile holds 1, 2 or 4
    groups of 4 live columns and runs in the one-event-per-thread tail form;
    rows against the oracle and a reconstruction."""
    ph, g, J, ns, ni = S.workload("tiny16")
    flat = np.nonzero(ph.mu.reshape(-1) > 0)[0][: 128 + extra]
    supp = np.zeros(ph.mu.size, dtype=bool)
    supp[flat] = True
    supp = supp.reshape(ph.mu.shape)
    ev = S.simulate_events(ph, g, 1500, seed=40 + extra)
    P = oracle_problem(ph, g, support=supp)
    p, s, f_ref, _ = _oracle_recon(P, ev, ns, 3)
    out = gpu_reconstruct(ph, g, ev, ns, 3, support=supp, rows=np.arange(300))
    assert row_close(out["rows"], p[:300]) <= 1.0
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4


@pytest.mark.parametrize("fmt", ["fp32", "fp16"])
def test_cpasync_ring_pass_bitwise(fmt):
    """The cp.async ring pass (pass_variant 3) does the register pass's
    arithmetic in the same order: images and log-likelihoods bitwise equal."""
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, 9001, seed=33)
    reg = gpu_reconstruct(ph, g, ev, ns, 3, fmt=fmt, loglik=True, pass_variant=1)
    cpa = gpu_reconstruct(ph, g, ev, ns, 3, fmt=fmt, loglik=True, pass_variant=3)
    assert np.array_equal(reg["f"], cpa["f"])
    assert np.array_equal(reg["loglik"], cpa["loglik"])


@pytest.mark.parametrize("fmt", ["fp32", "fp16"])
def test_wide_rows_prefetch_and_ring_passes_bitwise(fmt):
    """128 x 128 rows (one row per pipeline step) take the register pass with
    its L2 prefetch automatically; without the prefetch, at another distance
    and through the cp.async ring the images and log-likelihoods are the same
    bits."""
    ph, g, J, ns, ni = S.workload("dat128")
    ev = S.simulate_events(ph, g, 3000, seed=35)
    auto = gpu_reconstruct(ph, g, ev, ns, 2, fmt=fmt, loglik=True)
    for kw in (dict(pass_variant=1, prefetch_groups=-1), dict(pass_variant=1, prefetch_groups=7),
               dict(pass_variant=3)):
        other = gpu_reconstruct(ph, g, ev, ns, 2, fmt=fmt, loglik=True, **kw)
        assert np.array_equal(auto["f"], other["f"]), kw
        assert np.array_equal(auto["loglik"], other["loglik"]), kw


def test_introspection_and_error_messages():
    """lmosem_n_scatter counts the mu > 0 pixels; a rejected call leaves its
    reason in lmosem_last_error, which the binding puts in the exception."""
    import torch

    import paper_2002_12471_gb300.lmosem as L
    ph, g, J, ns, ni = S.workload("tiny16")
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream())
    try:
        assert L.lmosem_n_scatter(ctx) == int(np.sum(ph.mu > 0))
        assert L.lmosem_n_support(ctx) == int(np.sum(ph.mu > 0))
        with pytest.raises(L.LmosemError) as ei:
            L.lmosem_sensitivity(ctx, g["n_angles"] + 1)
        assert ei.value.status == L.EINVAL
        msg = L.load().lmosem_last_error(ctx).decode()
        assert "n_subsets" in msg and msg in str(ei.value)
    finally:
        L.lmosem_destroy(ctx)
