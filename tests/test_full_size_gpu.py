"""Parity at the benchmark's full sizes, in the launch configurations it
times, on outputs the FP64 oracle can compute one by one:

* the batching workload (64 realisations of the 64 x 64 DaT phantom, Poisson
  event counts with means in [50k, 400k], one persistent launch): sampled
  model rows of several realisations against the oracle, and the EM count
  identity T sum_n s^i_n f_n = |S_i| of every realisation after an iteration;
* the surrogate's inference at the model build's launch size (2^24 rows per
  launch): sampled outputs against the FP64 forward at the kernel's BF16
  rounding points, and every output finite."""
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

from oracle import mlp
from paper_2002_12471_gb300 import synthetic as S
from tests._helpers import oracle_problem, row_close

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    return L


def test_batch64_full_size(L):
    import torch
    sys.path.insert(0, ROOT)
    import bench
    counts = S.realisation_counts(64, seed=4)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        parts = pool.map(bench._realisation_events, list(enumerate(counts)))
    ph, g, _, ns, _ = S.workload("dat64")
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    a_h = np.concatenate([p[0] for p in parts])
    u_h = np.concatenate([p[1] for p in parts])
    e_h = np.concatenate([p[2] for p in parts])
    dev = torch.device("cuda:0")
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream())
    try:
        nsup = L.lmosem_n_support(ctx)
        sens = torch.zeros((ns, nsup), dtype=torch.float64, device=dev)
        L.lmosem_sensitivity(ctx, ns, sens)
        L.lmosem_build_model_batch(ctx, torch.from_numpy(a_h).to(dev), torch.from_numpy(u_h).to(dev),
                                   torch.from_numpy(e_h).to(dev), off, ns)
        rng = np.random.default_rng(7)
        reals = [0, 17, 40, 63]
        ids = np.concatenate([off[r] + rng.choice(counts[r], 25, replace=False) for r in reals])
        rows = torch.zeros((len(ids), nsup), dtype=torch.float32, device=dev)
        L.lmosem_model_rows(ctx, torch.from_numpy(ids.astype(np.int64)).to(dev), rows)
        f = torch.zeros((64, nsup), dtype=torch.float32, device=dev)
        L.lmosem_init_image_batch(ctx, 1.0, f)
        L.lmosem_iterate_batch(ctx, 1, 1.0, f)
        torch.cuda.synchronize()
        rows = rows.cpu().numpy().astype(np.float64)
        fr = f.cpu().numpy().astype(np.float64)
        s_last = sens[ns - 1].cpu().numpy()
    finally:
        L.lmosem_destroy(ctx)
    P = oracle_problem(ph, g)
    p = P.model(a_h[ids], u_h[ids], e_h[ids])
    assert row_close(rows, p) <= 1.0
    # after a full iteration the last sub-iteration was subset N_s - 1
    for r in range(64):
        n_last = int(np.sum(a_h[off[r]:off[r + 1]] % ns == ns - 1))
        assert np.dot(s_last, fr[r]) == pytest.approx(n_last, rel=2e-5), r


def test_surrogate_inference_at_launch_size(L):
    import torch
    dev = torch.device("cuda:0")
    ph, g, *_ = S.workload("tiny16")
    rng = np.random.default_rng(9)
    params = mlp.init_params(11)
    for W, b in params:
        b += rng.normal(0.0, 0.2, b.shape)
    n = 1 << 24
    X = torch.randn((n, 8), dtype=torch.float32, device=dev, generator=torch.Generator(dev).manual_seed(5))
    out = torch.empty(n, dtype=torch.float32, device=dev)
    blob = torch.from_numpy(L.pack_surrogate(params)).to(dev)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream(), surrogate_kernel=2)
    try:
        L.lmosem_surrogate_infer(ctx, blob, X, out)
    finally:
        L.lmosem_destroy(ctx)
    assert bool(torch.isfinite(out).all())
    idx = np.sort(rng.choice(n, 4096, replace=False))
    xs = X[torch.from_numpy(idx).to(dev)].cpu().numpy().astype(np.float64)
    ys = out[torch.from_numpy(idx).to(dev)].cpu().numpy().astype(np.float64)
    from tests.test_surrogate_gpu import _mirrored_forward
    ref = _mirrored_forward(params, xs, round_last=False)
    assert np.sqrt(np.mean((ys - ref) ** 2)) <= 1e-3 * max(np.sqrt(np.mean(ref ** 2)), 0.1)
