"""Scatter surrogate on the GPU: its tensor-core forward and backward against
the FP64 MLP oracle, its exact training targets against the oracle's scatter
path sum, training convergence, and what the trained network gains over
reconstructing without scatter compensation, measured against the exact
model."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2002_12471_gb300 import synthetic as S
from tests._helpers import gpu_reconstruct, oracle_problem, row_close

pytestmark = pytest.mark.gpu


def bf16(x):
    """Round to bfloat16 (nearest even), returned as float64."""
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32)
    u += 0x7FFF + ((u >> 16) & 1)
    u &= 0xFFFF0000
    return a.astype(np.float64)


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    return L


def _ctx(L, ph, g):
    import torch
    return L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream())


def _perturbed_params(seed):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(seed)
    for W, b in params:
        b += rng.normal(0.0, 0.2, b.shape)
    return params


def test_gradients_match_oracle(L):
    import torch
    dev = torch.device("cuda:0")
    ph, g, *_ = S.workload("tiny16")
    params = _perturbed_params(7)
    rng = np.random.default_rng(8)
    n = 512
    X = rng.normal(0.0, 1.0, (n, 8))
    t = rng.normal(0.0, 1.0, n)
    blob = L.pack_surrogate(params)
    ctx = _ctx(L, ph, g)
    try:
        grad = torch.zeros(L.SURROGATE_PARAMS, dtype=torch.float32, device=dev)
        loss = L.lmosem_surrogate_grad(ctx, torch.from_numpy(blob).to(dev),
                                       torch.from_numpy(X.astype(np.float32)).to(dev),
                                       torch.from_numpy(t.astype(np.float32)).to(dev), grad)
        g_gpu, _, _ = L.unpack_surrogate(grad.cpu().numpy())
        out = torch.zeros(n, dtype=torch.float32, device=dev)
        L.lmosem_surrogate_infer(ctx, torch.from_numpy(blob).to(dev),
                                 torch.from_numpy(X.astype(np.float32)).to(dev), out)
        y_gpu = out.cpu().numpy().astype(np.float64)
    finally:
        L.lmosem_destroy(ctx)
    # the oracle sees the same BF16-rounded weights and inputs as the products
    pq = [[bf16(W), np.asarray(b, dtype=np.float32).astype(np.float64)] for W, b in params]
    pq[-1][0] = np.asarray(params[-1][0], dtype=np.float32).astype(np.float64)   # output layer is FP32
    Xq = bf16(X.astype(np.float32))
    tq = t.astype(np.float32).astype(np.float64)
    # (1) the plain FP64 oracle: the GPU also rounds every hidden activation and
    # every back-propagated delta to BF16 (2^-9 relative each), and ReLU masks
    # of pre-activations within that rounding of zero can flip; the size of
    # that effect depends on the draw, so it is measured on the CPU (the
    # oracle at the GPU's rounding points, (2) below, against the plain one)
    # and the GPU may differ from the plain oracle by it plus 2e-3, and by 5e-2
    # at most
    loss_ref, g_ref = mlp.mse_loss_and_grad(pq, Xq, tq)
    y_ref, _ = mlp.forward(pq, Xq)
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    assert oracle.rel_l2(y_gpu, y_ref) <= 2e-2
    # (2) FP64 with the GPU's BF16 rounding points: only the FP32 accumulation
    # order remains
    hs, zs, h = [], [], Xq
    for k, (W, b) in enumerate(pq):
        z = h @ W.T + b
        hs.append(h)
        zs.append(z)
        h = bf16(np.maximum(z, 0.0)) if k < 4 else z
    r = h[:, 0] - tq
    d = (2.0 * r / n)[:, None]
    gm = [None] * 5
    for k in range(4, -1, -1):
        if k < 4:
            d = bf16(d * (zs[k] > 0.0))
        elif k == 4:
            gm[k] = [d.T @ hs[k], d.sum(axis=0)]
            d = bf16((d @ pq[k][0]) * (zs[k - 1] > 0.0))
            continue
        gm[k] = [d.T @ hs[k], d.sum(axis=0)]
        if k > 0:
            d = d @ pq[k][0]
    for l in range(5):
        for i in range(2):
            err = oracle.rel_l2(np.ravel(g_gpu[l][i]), np.ravel(gm[l][i]))
            assert err <= 2e-3, ("bf16-mirrored", l, i, err)
            bf16_effect = oracle.rel_l2(np.ravel(gm[l][i]), np.ravel(g_ref[l][i]))
            err = oracle.rel_l2(np.ravel(g_gpu[l][i]), np.ravel(g_ref[l][i]))
            assert err <= min(bf16_effect + 2e-3, 5e-2), (l, i, err, bf16_effect)


def _mirrored_forward(params, X, round_last):
    """FP64 forward with the GPU's BF16 rounding points: inputs, hidden
    weights and the ReLU outputs of the first three hidden layers (and of the
    fourth where ``round_last``); the 256 -> 1 output layer stays FP32."""
    pq = [[bf16(W), np.asarray(b, dtype=np.float32).astype(np.float64)] for W, b in params]
    pq[-1][0] = np.asarray(params[-1][0], dtype=np.float32).astype(np.float64)
    h = bf16(X.astype(np.float32))
    for k, (W, b) in enumerate(pq):
        z = h @ W.T + b
        if k < 4:
            h = np.maximum(z, 0.0)
            if k < 3 or round_last:
                h = bf16(h)
        else:
            h = z
    return h[:, 0]


@pytest.mark.parametrize("n", [1, 129, 10007, 3 * 152 * 128 + 5])
def test_tcgen05_inference_matches_product_chain_and_oracle(L, n):
    """The fused tcgen05 inference kernel (persistent over 128-row tiles, a
    ragged last tile) against the chain of separate tcgen05 products (the
    training kernels, activations through HBM) and against the FP64 forward
    with the same BF16 rounding points."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, *_ = S.workload("tiny16")
    params = _perturbed_params(11)
    X = np.random.default_rng(12).normal(0.0, 1.0, (n, 8))
    blob = torch.from_numpy(L.pack_surrogate(params)).to(dev)
    Xd = torch.from_numpy(X.astype(np.float32)).to(dev)
    ys = {}
    for kern in (0, 1, 2):
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream(), surrogate_kernel=kern)
        try:
            out = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
            L.lmosem_surrogate_infer(ctx, blob, Xd, out)
            ys[kern] = out.cpu().numpy().astype(np.float64)
        finally:
            L.lmosem_destroy(ctx)
    assert np.all(np.isfinite(ys[2]))
    np.testing.assert_array_equal(ys[0], ys[2])          # automatic choice is tcgen05
    ref_tc = _mirrored_forward(params, X, round_last=False)
    ref_mma = _mirrored_forward(params, X, round_last=True)
    scale = max(np.sqrt(np.mean(ref_tc ** 2)), 0.1)
    err = lambda a, b: np.sqrt(np.mean((a - b) ** 2)) / scale
    # only the FP32 accumulation order (and the BF16 roundings it tips) remain
    assert err(ys[2], ref_tc) <= 1e-3
    assert err(ys[1], ref_mma) <= 1e-3
    # the two kernels differ by the BF16 rounding of the last hidden layer,
    # as the two references predict (the sum over 256 terms cancels, so that
    # rounding can be a percent of a small output)
    assert err(ys[2] - ys[1], ref_tc - ref_mma) <= 2e-3


def test_tcgen05_bounded_wait_reports_timeout(L):
    """With a one-cycle wait budget every CTA of the fused kernel gives up on
    its first tensor-core wait: the call returns LMOSEM_ETIMEOUT (after the
    pending products drained and TMEM was freed) and the GPU stays usable."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, *_ = S.workload("tiny16")
    params = _perturbed_params(13)
    n = 4 * 128 + 3
    X = np.random.default_rng(14).normal(0.0, 1.0, (n, 8))
    blob = torch.from_numpy(L.pack_surrogate(params)).to(dev)
    Xd = torch.from_numpy(X.astype(np.float32)).to(dev)
    out = torch.zeros(n, dtype=torch.float32, device=dev)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream(), surrogate_kernel=2,
                          wait_budget_cycles=1)
    try:
        with pytest.raises(L.LmosemError) as ei:
            L.lmosem_surrogate_infer(ctx, blob, Xd, out)
        assert ei.value.status == L.ETIMEOUT
    finally:
        L.lmosem_destroy(ctx)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream(), surrogate_kernel=2)
    try:
        L.lmosem_surrogate_infer(ctx, blob, Xd, out)
    finally:
        L.lmosem_destroy(ctx)
    ref = _mirrored_forward(params, X, round_last=False)
    y = out.cpu().numpy().astype(np.float64)
    assert np.sqrt(np.mean((y - ref) ** 2)) <= 1e-3 * max(np.sqrt(np.mean(ref ** 2)), 0.1)


def test_training_targets_match_oracle_scatter(L):
    import torch
    dev = torch.device("cuda:0")
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, 40, seed=31)
    P = oracle_problem(ph, g)
    ctx = _ctx(L, ph, g)
    try:
        nsup = L.lmosem_n_support(ctx)
        feat = torch.zeros((len(ev) * nsup, L.SURROGATE_INPUTS), dtype=torch.float32, device=dev)
        targ = torch.zeros(len(ev) * nsup, dtype=torch.float32, device=dev)
        rel = torch.full((len(ev) * nsup,), np.nan, dtype=torch.float32, device=dev)
        L.lmosem_surrogate_samples(ctx, torch.from_numpy(ev.angle).to(dev), torch.from_numpy(ev.u_mm).to(dev),
                                   torch.from_numpy(ev.e_kev).to(dev), feat, targ, rel)
        f = feat.cpu().numpy().astype(np.float64).reshape(len(ev), nsup, L.SURROGATE_INPUTS)
        t32 = targ.cpu().numpy().reshape(len(ev), nsup)
        p_gpu = np.exp(t32.astype(np.float64))
        r32 = rel.cpu().numpy().reshape(len(ev), nsup)
    finally:
        L.lmosem_destroy(ctx)
    # each log's offset from its row's largest log, one FP32 subtraction
    np.testing.assert_array_equal(r32, t32 - t32.max(axis=1, keepdims=True))
    scat = P.model(ev.angle, ev.u_mm, ev.e_kev, primary=False)
    assert row_close(p_gpu, scat) <= 1.0
    # inputs: pixel centre, angle, position, energy, attenuation to the edge,
    # and along the event's detector line from the pixel's depth and whole
    xs, ys = P.pixel_centres(P.support)
    th = g["angle0_rad"] + 2 * np.pi * ev.angle / g["n_angles"]
    u = ev.u_mm[:, None].astype(np.float64)
    depth = xs[None, :] * np.cos(th)[:, None] + ys[None, :] * np.sin(th)[:, None]
    a2 = np.broadcast_to(ev.angle[:, None], depth.shape)
    line_from = P.line_attenuation(a2, np.broadcast_to(u, depth.shape), depth)
    line_total = P.line_attenuation(ev.angle, ev.u_mm.astype(np.float64), np.full(len(ev), P.line_start()))
    ref = mlp.features(xs[None, :], ys[None, :], th[:, None], u, ev.e_kev[:, None].astype(np.float64),
                       P.l_edge[ev.angle][:, P.support], line_from, line_total[:, None])
    np.testing.assert_allclose(f, ref, rtol=1e-5, atol=1e-5)


def test_training_draws_pairs_by_magnitude_weight(L):
    """With magnitude_power, minibatch rows are drawn in proportion to
    exp(alpha rel_log).  Half the rows carry target a and weight 1, the other
    half target b and weight exp(-60) (never drawn in practice); the inputs are
    noise.  The normalised targets are -1 and +1 (mean and deviation over all
    rows), so a network that sees only the weighted rows drives its loss to 0,
    while uniform draws leave it at 1, the variance of the two."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, J, ns, ni = S.workload("tiny16")
    n = 1 << 16
    gen = torch.Generator().manual_seed(7)
    feat = torch.rand((n, 8), generator=gen).to(dev)
    heavy = torch.rand(n, generator=gen) < 0.5
    targ = torch.where(heavy, torch.tensor(-3.0), torch.tensor(1.0)).to(dev)
    rel = torch.where(heavy, torch.tensor(0.0), torch.tensor(-60.0)).to(dev)
    ctx = _ctx(L, ph, g)
    try:
        last = {}
        for power in (0.0, 1.0):
            blob = torch.from_numpy(L.pack_surrogate(mlp.init_params(3))).to(dev)
            curve = L.lmosem_surrogate_train(ctx, feat, targ, blob, steps=600, batch=1024, lr=1e-3, seed=9,
                                             d_rel_log=rel, magnitude_power=power)
            last[power] = float(np.mean(curve[-100:]))
        with pytest.raises(RuntimeError):
            L.lmosem_surrogate_train(ctx, feat, targ, blob, steps=1, batch=1024, d_rel_log=rel,
                                     magnitude_power=-1.0)
    finally:
        L.lmosem_destroy(ctx)
    assert last[1.0] < 0.02, last
    assert 0.8 < last[0.0] < 1.2, last


def test_target_floor_per_row_with_row_offsets(L):
    """target_floor F raises the targets below (largest - F): with the row
    offsets given, the largest of the same event's row, else the largest of
    all.  The blob's mean and deviation are those of the floored targets
    (FP64 sums, no baseline)."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, J, ns, ni = S.workload("tiny16")
    rng = np.random.default_rng(11)
    rows, width, F = 256, 64, 5.0
    t = (rng.uniform(-30.0, 0.0, (rows, 1)) + rng.uniform(-12.0, 0.0, (rows, width))).astype(np.float32)
    rel = t - t.max(axis=1, keepdims=True)
    feat = torch.from_numpy(rng.uniform(-1, 1, (rows * width, 8)).astype(np.float32)).to(dev)
    want = {"row": np.where(rel < -F, t - rel - np.float32(F), t).astype(np.float64),
            "all": np.maximum(t, t.max() - np.float32(F)).astype(np.float64)}
    ctx = _ctx(L, ph, g)
    try:
        for kind in ("row", "all"):
            blob = torch.from_numpy(L.pack_surrogate(mlp.init_params(3))).to(dev)
            L.lmosem_surrogate_train(ctx, feat, torch.from_numpy(t.reshape(-1)).to(dev), blob, steps=1, batch=64,
                                     target_floor=F,
                                     d_rel_log=torch.from_numpy(rel.reshape(-1)).to(dev) if kind == "row" else None)
            _, mu, sigma = L.unpack_surrogate(blob.cpu().numpy())
            w = want[kind]
            assert mu == pytest.approx(w.mean(), rel=1e-6), kind
            assert sigma == pytest.approx(w.std(), rel=1e-5), kind
    finally:
        L.lmosem_destroy(ctx)


@pytest.fixture(scope="module")
def trained(L):
    """Surrogate trained on exact scatter sums of 400 events of the 32 x 32
    brain workload, plus 60 held-out events."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, 460, seed=51)
    ctx = _ctx(L, ph, g)
    try:
        nsup = L.lmosem_n_support(ctx)
        feat = torch.zeros((len(ev) * nsup, L.SURROGATE_INPUTS), dtype=torch.float32, device=dev)
        targ = torch.zeros(len(ev) * nsup, dtype=torch.float32, device=dev)
        L.lmosem_surrogate_samples(ctx, torch.from_numpy(ev.angle).to(dev), torch.from_numpy(ev.u_mm).to(dev),
                                   torch.from_numpy(ev.e_kev).to(dev), feat, targ)
        ntr = 400 * nsup
        blob = torch.from_numpy(L.pack_surrogate(mlp.init_params(3))).to(dev)
        curve = L.lmosem_surrogate_train(ctx, feat[:ntr].contiguous(), targ[:ntr].contiguous(), blob,
                                         steps=3000, batch=2048, lr=1e-3, seed=5)
        out = torch.zeros(len(ev) * nsup - ntr, dtype=torch.float32, device=dev)
        L.lmosem_surrogate_infer(ctx, blob, feat[ntr:].contiguous(), out)
        _, mu, sigma = L.unpack_surrogate(blob.cpu().numpy())
        pred = mu + sigma * out.cpu().numpy().astype(np.float64)
        held = targ[ntr:].cpu().numpy().astype(np.float64)
    finally:
        L.lmosem_destroy(ctx)
    return dict(ph=ph, g=g, ns=ns, curve=curve, pred=pred, held=held, blob=blob, sigma=sigma)


def test_training_converges_and_generalises(trained):
    c = trained["curve"]
    assert np.all(np.isfinite(c))
    assert np.mean(c[-200:]) < 0.1 * np.mean(c[:20])
    err = trained["pred"] - trained["held"]
    # held-out events: log scatter within a few tens of percent (the trained
    # network's own minibatch loss, 0.0085 sigma^2, is an RMS of ~0.09 sigma)
    assert np.sqrt(np.mean(err ** 2)) < 0.3 * trained["sigma"]
    assert np.median(np.abs(err)) < 0.35


def test_surrogate_model_rows_agree_across_kernels(L, trained):
    """Model rows built with the surrogate scatter term through the fused
    tcgen05 kernel and through the chain of separate products agree to the
    BF16 rounding of the last hidden layer."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, ns = trained["ph"], trained["g"], trained["ns"]
    ev = S.simulate_events(ph, g, 3000, seed=53)
    rows = {}
    for kern in (1, 2):
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream(), surrogate_kernel=kern)
        try:
            L.lmosem_set_surrogate_check(ctx, 0.0)    # measure only: keep the surrogate's rows
            L.lmosem_surrogate_load(ctx, trained["blob"])
            nsup = L.lmosem_n_support(ctx)
            L.lmosem_build_model(ctx, torch.from_numpy(ev.angle).to(dev), torch.from_numpy(ev.u_mm).to(dev),
                                 torch.from_numpy(ev.e_kev).to(dev), ns, "surrogate")
            ids = torch.arange(0, len(ev), 7, dtype=torch.int64, device=dev)
            out = torch.zeros((ids.numel(), nsup), dtype=torch.float32, device=dev)
            L.lmosem_model_rows(ctx, ids, out)
            rows[kern] = out.cpu().numpy().astype(np.float64)
        finally:
            L.lmosem_destroy(ctx)
    assert np.all(np.isfinite(rows[2]))
    assert oracle.rel_l2(rows[2], rows[1]) <= 2e-3


def test_surrogate_model_gains_over_no_scatter_compensation(L, trained):
    """Reconstructions with the surrogate's scatter term stay close to those
    of the exact path sum; leaving scatter out altogether does not."""
    import torch
    ph, g, ns = trained["ph"], trained["g"], trained["ns"]
    ev = S.simulate_events(ph, g, 20000, seed=52)
    exact = gpu_reconstruct(ph, g, ev, ns, 4)

    def with_blob(blob):
        import paper_2002_12471_gb300.lmosem as Lm
        dev = torch.device("cuda:0")
        ctx = Lm.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream())
        try:
            Lm.lmosem_set_surrogate_check(ctx, 0.0)   # measure only: keep the surrogate's rows
            Lm.lmosem_surrogate_load(ctx, blob)
            nsup = Lm.lmosem_n_support(ctx)
            Lm.lmosem_sensitivity(ctx, ns)
            Lm.lmosem_build_model(ctx, torch.from_numpy(ev.angle).to(dev), torch.from_numpy(ev.u_mm).to(dev),
                                  torch.from_numpy(ev.e_kev).to(dev), ns, "surrogate")
            f = torch.zeros(nsup, dtype=torch.float32, device=dev)
            Lm.lmosem_init_image(ctx, 1.0, f)
            Lm.lmosem_iterate(ctx, 4, 1.0, f)
            return f.cpu().numpy().astype(np.float64)
        finally:
            Lm.lmosem_destroy(ctx)

    f_sur = with_blob(trained["blob"])
    none = trained["blob"].clone()
    none[-2] = -1.0e4        # mu: exp(mu + sigma y) = 0, i.e. no scatter paths
    none[-1] = 0.0
    f_none = with_blob(none)
    img = lambda f: np.bincount(exact["support"], weights=f, minlength=ph.mu.size)
    for name, roi in ph.rois.items():
        w = roi.reshape(-1)
        ref = np.dot(w, img(exact["f"]))
        e_sur = abs(np.dot(w, img(f_sur)) - ref) / ref
        e_none = abs(np.dot(w, img(f_none)) - ref) / ref
        assert e_sur < 0.5 * e_none, (name, e_sur, e_none)
    assert oracle.rel_l2(f_sur, exact["f"]) < 0.5 * oracle.rel_l2(f_none, exact["f"])


def _model_rows(L, ctx, n_events, nsup, step=1):
    import torch
    dev = torch.device("cuda:0")
    ids = torch.arange(0, n_events, step, dtype=torch.int64, device=dev)
    out = torch.zeros((ids.numel(), nsup), dtype=torch.float32, device=dev)
    L.lmosem_model_rows(ctx, ids, out)
    return out.cpu().numpy()


def test_surrogate_check_measures_the_row_error(L, trained):
    """The exact judge of a surrogate build (measure only): its error over
    512 sampled rows estimates the error of all rows against the exact path
    sum, and a tolerance below it replaces the model by the exact rows."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, ns = trained["ph"], trained["g"], trained["ns"]
    ev = S.simulate_events(ph, g, 6000, seed=54)
    a, u, e = (torch.from_numpy(x).to(dev) for x in (ev.angle, ev.u_mm, ev.e_kev))
    rows = {}
    for name, fmt, tol in (("exact", "fp32", None), ("sur", "surrogate", 0.0), ("fallback", "surrogate", "below")):
        ctx = _ctx(L, ph, g)
        try:
            nsup = L.lmosem_n_support(ctx)
            L.lmosem_surrogate_load(ctx, trained["blob"])
            if tol == "below":
                L.lmosem_set_surrogate_check(ctx, 0.5 * rows["check"][0])
            elif tol is not None:
                L.lmosem_set_surrogate_check(ctx, tol)
            L.lmosem_build_model(ctx, a, u, e, ns, fmt)
            if fmt == "fp32":
                with pytest.raises(L.LmosemError) as ei:
                    L.lmosem_surrogate_check(ctx)
                assert ei.value.status == L.ESTATE
            elif tol == 0.0:
                rows["check"] = L.lmosem_surrogate_check(ctx)
            else:
                rows["check_fb"] = L.lmosem_surrogate_check(ctx)
            rows[name] = _model_rows(L, ctx, len(ev), nsup)
        finally:
            L.lmosem_destroy(ctx)
    err, row_max, exact = rows["check"]
    full = oracle.rel_l2(rows["sur"].astype(np.float64), rows["exact"].astype(np.float64))
    assert not exact and err > 0.0 and row_max >= err
    assert 0.5 * full <= err <= 2.0 * full, (err, full)
    err_fb, _, exact_fb = rows["check_fb"]
    assert exact_fb and err_fb == pytest.approx(err, rel=1e-9)
    assert np.array_equal(rows["fallback"], rows["exact"])


def test_untrained_surrogate_falls_back_to_the_exact_model(L):
    """An untrained network fails the exact check at the default tolerance;
    the build then holds the exact rows, and the reconstruction matches the
    FP64 oracle (16 x 16 disk, 2,000 events, 4 subsets x 5 iterations)."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, J, seed=1)
    a, u, e = (torch.from_numpy(x).to(dev) for x in (ev.angle, ev.u_mm, ev.e_kev))
    ctx = _ctx(L, ph, g)
    try:
        nsup = L.lmosem_n_support(ctx)
        L.lmosem_surrogate_load(ctx, torch.from_numpy(L.surrogate_init(seed=4)).to(dev))
        L.lmosem_sensitivity(ctx, ns)
        L.lmosem_build_model(ctx, a, u, e, ns, "surrogate")
        err, row_max, exact = L.lmosem_surrogate_check(ctx)
        f = torch.zeros(nsup, dtype=torch.float32, device=dev)
        L.lmosem_init_image(ctx, 1.0, f)
        L.lmosem_iterate(ctx, ni, 1.0, f)
        f_gpu = f.cpu().numpy().astype(np.float64)
    finally:
        L.lmosem_destroy(ctx)
    assert exact and err > 1e-2
    P = oracle_problem(ph, g)
    p = P.model(ev.angle, ev.u_mm, ev.e_kev)
    s = P.sensitivity(ns)
    f_ref, _ = oracle.osem(p, ev.angle, s, ni, oracle.initial_image(J, s.sum(0)))
    assert oracle.rel_l2(f_gpu, f_ref) <= 1e-4


def _gated_rows(L, ph, g, ns, blob, ev, row_tol, check_tol=1.0):
    """Model rows (original event order) of a surrogate build with the
    energy gate at row_tol, and the gate's and the check's results."""
    import torch
    dev = torch.device("cuda:0")
    ctx = _ctx(L, ph, g)
    try:
        nsup = L.lmosem_n_support(ctx)
        L.lmosem_surrogate_load(ctx, blob)
        L.lmosem_set_surrogate_check(ctx, check_tol)
        L.lmosem_set_surrogate_gate(ctx, row_tol)
        a, u, e = (torch.from_numpy(x).to(dev) for x in (ev.angle, ev.u_mm, ev.e_kev))
        L.lmosem_build_model(ctx, a, u, e, ns, "surrogate")
        return _model_rows(L, ctx, len(ev), nsup), L.lmosem_surrogate_gate(ctx), L.lmosem_surrogate_check(ctx)
    finally:
        L.lmosem_destroy(ctx)


def test_energy_gate_takes_exact_rows_below_its_cut(L, trained):
    """The energy gate of the surrogate form: rows of events below the cut
    are bitwise the exact path sum's, the others bitwise the surrogate's; the
    cut sits on a bin edge of the window; a tolerance no bin meets makes every
    row exact, one every bin meets none."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, ns = trained["ph"], trained["g"], trained["ns"]
    ev = S.simulate_events(ph, g, 6000, seed=55)
    ctx = _ctx(L, ph, g)
    try:
        nsup = L.lmosem_n_support(ctx)
        a, u, e = (torch.from_numpy(x).to(dev) for x in (ev.angle, ev.u_mm, ev.e_kev))
        L.lmosem_build_model(ctx, a, u, e, ns, "fp32")
        exact = _model_rows(L, ctx, len(ev), nsup)
    finally:
        L.lmosem_destroy(ctx)
    sur, (cut0, frac0), _ = _gated_rows(L, ph, g, ns, trained["blob"], ev, 0.0)
    assert cut0 == g["e_lo_kev"] and frac0 == 0.0
    assert not np.array_equal(sur, exact)
    for tol in (3e-2, 1e-2, 3e-3):
        rows, (cut, frac), (err, row_max, all_exact) = _gated_rows(L, ph, g, ns, trained["blob"], ev, tol)
        k = (cut - g["e_lo_kev"]) / 5.0
        assert abs(k - round(k)) < 1e-9 and g["e_lo_kev"] <= cut <= g["e_hi_kev"], cut
        low = ev.e_kev < cut
        assert frac == pytest.approx(low.mean(), abs=1e-12)
        assert np.array_equal(rows[low], exact[low])
        assert np.array_equal(rows[~low], sur[~low])
        assert all_exact == (frac == 1.0)
    # every sampled bin fails: the cut is the top edge of the highest one
    rows, (cut, frac), (err, _, all_exact) = _gated_rows(L, ph, g, ns, trained["blob"], ev, 1e-12)
    low = ev.e_kev < cut
    assert cut >= g["e_hi_kev"] - 5.0 and frac > 0.99 and err == 0.0
    assert frac == pytest.approx(low.mean(), abs=1e-12) and all_exact == (frac == 1.0)
    assert np.array_equal(rows[low], exact[low])
    rows, (cut, frac), _ = _gated_rows(L, ph, g, ns, trained["blob"], ev, 1e12)
    assert cut == g["e_lo_kev"] and frac == 0.0
    assert np.array_equal(rows, sur)


@pytest.fixture(scope="module")
def trained_dat32(L):
    """Surrogate trained as the benchmark trains it (pairs drawn by
    magnitude, alpha = 1; per-row floor 14; quadratic residual baseline) on
    exact scatter sums of 3,000 events of the 32 x 32 brain workload
    (20,000 steps, about 10 s)."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, 3000, seed=61)
    ctx = _ctx(L, ph, g)
    try:
        nsup = L.lmosem_n_support(ctx)
        feat = torch.zeros((len(ev) * nsup, L.SURROGATE_INPUTS), dtype=torch.float32, device=dev)
        targ = torch.zeros(len(ev) * nsup, dtype=torch.float32, device=dev)
        rel = torch.zeros(len(ev) * nsup, dtype=torch.float32, device=dev)
        L.lmosem_surrogate_samples(ctx, torch.from_numpy(ev.angle).to(dev), torch.from_numpy(ev.u_mm).to(dev),
                                   torch.from_numpy(ev.e_kev).to(dev), feat, targ, rel)
        blob = torch.from_numpy(L.surrogate_init(seed=3)).to(dev)
        L.lmosem_surrogate_train(ctx, feat, targ, blob, steps=20000, batch=4096, lr=1e-3, seed=5,
                                 target_floor=14.0, residual_fit=True, d_rel_log=rel, magnitude_power=1.0)
    finally:
        L.lmosem_destroy(ctx)
    return dict(ph=ph, g=g, ns=ns, blob=blob)


def test_surrogate_form_reconstructs_within_the_bound(L, trained_dat32):
    """The surrogate form as the library builds it (energy gate at a mean
    row error of 1e-2, exact check at 1e-2) reconstructs 20,000 events of the
    32 x 32 brain (6 subsets x 10 iterations) within 1e-2 relative L2 of the
    exact model's image, with striatal ROI means within 1%, while the
    surrogate still serves part of the rows."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, ns = trained_dat32["ph"], trained_dat32["g"], trained_dat32["ns"]
    ni = 10
    ev = S.simulate_events(ph, g, 20000, seed=62)
    exact = gpu_reconstruct(ph, g, ev, ns, ni)
    ctx = _ctx(L, ph, g)
    try:
        nsup = L.lmosem_n_support(ctx)
        L.lmosem_surrogate_load(ctx, trained_dat32["blob"])
        L.lmosem_set_surrogate_gate(ctx, 1e-2)
        L.lmosem_sensitivity(ctx, ns)
        a, u, e = (torch.from_numpy(x).to(dev) for x in (ev.angle, ev.u_mm, ev.e_kev))
        L.lmosem_build_model(ctx, a, u, e, ns, "surrogate")
        cut, frac = L.lmosem_surrogate_gate(ctx)
        f = torch.zeros(nsup, dtype=torch.float32, device=dev)
        L.lmosem_init_image(ctx, 1.0, f)
        L.lmosem_iterate(ctx, ni, 1.0, f)
        f_sur = f.cpu().numpy().astype(np.float64)
    finally:
        L.lmosem_destroy(ctx)
    assert frac < 1.0, (cut, frac)
    assert oracle.rel_l2(f_sur, exact["f"]) <= 1e-2, (cut, frac)
    img = lambda f: np.bincount(exact["support"], weights=f, minlength=ph.mu.size)
    for name, roi in ph.rois.items():
        w = roi.reshape(-1)
        ref = np.dot(w, img(exact["f"]))
        assert abs(np.dot(w, img(f_sur)) - ref) <= 1e-2 * ref, name


def test_inputs_match_oracle_at_the_benchmark_geometry(L):
    """All eight surrogate inputs at the 128 x 128 benchmark geometry (2 mm
    pixels, 120 angles, 128 bins) for 12 events against the oracle's
    encoding, with the two line attenuations from its own exact node
    integrals."""
    import torch
    dev = torch.device("cuda:0")
    ph, g, *_ = S.workload("dat128")
    ev = S.simulate_events(ph, g, 12, seed=71)
    P = oracle_problem(ph, g)
    ctx = _ctx(L, ph, g)
    try:
        nsup = L.lmosem_n_support(ctx)
        feat = torch.zeros((len(ev) * nsup, L.SURROGATE_INPUTS), dtype=torch.float32, device=dev)
        targ = torch.zeros(len(ev) * nsup, dtype=torch.float32, device=dev)
        L.lmosem_surrogate_samples(ctx, torch.from_numpy(ev.angle).to(dev), torch.from_numpy(ev.u_mm).to(dev),
                                   torch.from_numpy(ev.e_kev).to(dev), feat, targ)
        f = feat.cpu().numpy().astype(np.float64).reshape(len(ev), nsup, L.SURROGATE_INPUTS)
    finally:
        L.lmosem_destroy(ctx)
    xs, ys = P.pixel_centres(P.support)
    th = g["angle0_rad"] + 2 * np.pi * ev.angle / g["n_angles"]
    u = ev.u_mm[:, None].astype(np.float64)
    depth = xs[None, :] * np.cos(th)[:, None] + ys[None, :] * np.sin(th)[:, None]
    line_from = P.line_attenuation(np.broadcast_to(ev.angle[:, None], depth.shape),
                                   np.broadcast_to(u, depth.shape), depth)
    line_total = P.line_attenuation(ev.angle, ev.u_mm.astype(np.float64), np.full(len(ev), P.line_start()))
    ref = mlp.features(xs[None, :], ys[None, :], th[:, None], u, ev.e_kev[:, None].astype(np.float64),
                       P.l_edge[ev.angle][:, P.support], line_from, line_total[:, None])
    np.testing.assert_allclose(f, ref, rtol=1e-5, atol=1e-5)
