"""Batching form: many independent noise realisations (uneven and empty event
sets) reconstructed by one persistent launch.  Every realisation must match
the single-data-set path (itself checked against the FP64 oracle) and the
oracle directly; the chunked, claim-ordered execution must still be
bitwise deterministic; the autotuner's choice must not change the results."""
import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S
from tests._helpers import gpu_reconstruct, oracle_problem

pytestmark = pytest.mark.gpu


def _events(ph, g, counts, seed0):
    evs = [S.simulate_events(ph, g, n, seed=seed0 + r) if n else None for r, n in enumerate(counts)]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    cat = lambda k, dt: np.concatenate([getattr(e, k) for e in evs if e is not None]).astype(dt)
    return evs, off, cat("angle", np.int32), cat("u_mm", np.float32), cat("e_kev", np.float32)


def _batch_run(ph, g, a, u, e, off, ns, ni, tiles=None, autotune=False, budget_after_build=0, **opts):
    import torch

    import paper_2002_12471_gb300.lmosem as L
    dev = torch.device("cuda:0")
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream(), **opts)
    try:
        nsup = L.lmosem_n_support(ctx)
        L.lmosem_sensitivity(ctx, ns)
        L.lmosem_build_model_batch(ctx, torch.from_numpy(a).to(dev), torch.from_numpy(u).to(dev),
                                   torch.from_numpy(e).to(dev), off, ns)
        f = torch.zeros((len(off) - 1, nsup), dtype=torch.float32, device=dev)
        L.lmosem_init_image_batch(ctx, 1.0, f)
        choice = None
        if autotune:
            choice = L.lmosem_autotune_batch(ctx, 1.0, f)
        if tiles:
            L.lmosem_set_batch_tiles(ctx, *tiles)
        if budget_after_build:
            L.lmosem_set_wait_budget(ctx, budget_after_build)
        L.lmosem_iterate_batch(ctx, ni, 1.0, f)
        torch.cuda.synchronize()
        return f.cpu().numpy().astype(np.float64), choice
    finally:
        L.lmosem_destroy(ctx)


@pytest.fixture(scope="module")
def batch32():
    import __graft_entry__
    __graft_entry__.build()
    ph, g, J, ns, ni = S.workload("dat32")
    counts = [3000, 0, 9500, 120, 6100, 1]
    evs, off, a, u, e = _events(ph, g, counts, 40)
    return dict(ph=ph, g=g, ns=ns, ni=3, counts=counts, evs=evs, off=off, a=a, u=u, e=e)


@pytest.mark.parametrize("tiles", [(512, 2), (64, 1), (1000, 4)])
def test_batch_matches_single_and_oracle(batch32, tiles):
    d = batch32
    f, _ = _batch_run(d["ph"], d["g"], d["a"], d["u"], d["e"], d["off"], d["ns"], d["ni"], tiles=tiles)
    for r, ev in enumerate(d["evs"]):
        if ev is None:
            assert np.all(f[r] == 0)
            continue
        single = gpu_reconstruct(d["ph"], d["g"], ev, d["ns"], d["ni"])
        if not np.any(single["f"]):
            # a realisation with an empty subset is zeroed by Eq. 7 on both paths
            assert not np.any(f[r]), r
            continue
        assert oracle.rel_l2(f[r], single["f"]) <= 1e-5, (r, oracle.rel_l2(f[r], single["f"]))
    # one realisation against the oracle directly
    ev = d["evs"][2]
    P = oracle_problem(d["ph"], d["g"])
    p = P.model(ev.angle, ev.u_mm, ev.e_kev)
    s = P.sensitivity(d["ns"])
    f_ref, _ = oracle.osem(p, ev.angle, s, d["ni"], oracle.initial_image(len(ev), s.sum(0)))
    assert oracle.rel_l2(f[2], f_ref) <= 1e-4


def test_batch_is_deterministic_and_autotune_keeps_results(batch32):
    import torch
    d = batch32
    args = (d["ph"], d["g"], d["a"], d["u"], d["e"], d["off"], d["ns"], d["ni"])
    f1, _ = _batch_run(*args, tiles=(256, 3))
    f2, _ = _batch_run(*args, tiles=(256, 3))
    assert np.array_equal(f1, f2)
    s = torch.cuda.Stream()       # graph-replayed launch on a non-default stream
    with torch.cuda.stream(s):
        f3, choice = _batch_run(*args, autotune=True)
    torch.cuda.synchronize()
    assert choice[0] in (128, 256, 512, 1024, 2048) and 1 <= choice[1] <= 4
    assert oracle.rel_l2(f3, f1) <= 1e-5


def test_batch_wait_budget_runs_out_cleanly(batch32):
    """A one-cycle idle budget makes the persistent kernel give up (status
    word, LMOSEM_ETIMEOUT) instead of waiting; the GPU stays usable."""
    import paper_2002_12471_gb300.lmosem as L
    d = batch32
    with pytest.raises(L.LmosemError) as ei:
        _batch_run(d["ph"], d["g"], d["a"], d["u"], d["e"], d["off"], d["ns"], 4, tiles=(64, 4),
                   budget_after_build=1)
    assert ei.value.status == L.ETIMEOUT
    f, _ = _batch_run(d["ph"], d["g"], d["a"], d["u"], d["e"], d["off"], d["ns"], 1)
    assert np.all(np.isfinite(f))


def test_batch_rejects_bad_offsets(batch32):
    import torch

    import paper_2002_12471_gb300.lmosem as L
    d = batch32
    dev = torch.device("cuda:0")
    ctx = L.lmosem_create(d["ph"].mu, d["ph"].pixel_mm, d["g"])
    try:
        a, u, e = (torch.from_numpy(x).to(dev) for x in (d["a"], d["u"], d["e"]))
        for bad in ([1, 5, 9], [0, 7, 3], [0]):
            with pytest.raises(L.LmosemError) as ei:
                L.lmosem_build_model_batch(ctx, a, u, e, bad, 2)
            assert ei.value.status == L.EINVAL
        with pytest.raises(L.LmosemError) as ei:
            L.lmosem_build_model_batch(ctx, a, u, e, [0, len(d["a"])], 2, fmt="fp16")
        assert ei.value.status == L.ENOTIMPL
    finally:
        L.lmosem_destroy(ctx)
