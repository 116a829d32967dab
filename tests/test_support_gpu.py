"""The binned-OSEM support initialiser on the GPU against its FP64 oracle
(oracle/binned.py), and what it buys the list-mode reconstruction: a smaller
support that still covers the activity.

Tolerances: the crude image is a sum of FP32 erf differences (2 ulp each)
over a few thousand pixels per bin and twelve EM sub-iterations, so rel-L2 <=
1e-4; the mask is the oracle's except where the oracle image lies within
1e-3 (relative) of the threshold, or within the dilation of such a pixel."""
import numpy as np
import pytest

import oracle
from oracle import binned
from paper_2002_12471_gb300 import synthetic as S
from tests._helpers import gpu_reconstruct

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    return L


def _gpu_support(L, ph, g, ev, **kw):
    import torch
    dev = torch.device("cuda:0")
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=torch.cuda.current_stream())
    try:
        img = torch.zeros(ph.mu.size, dtype=torch.float32, device=dev)
        mask = L.lmosem_binned_support(ctx, torch.from_numpy(ev.angle).to(dev), torch.from_numpy(ev.u_mm).to(dev),
                                       torch.from_numpy(ev.e_kev).to(dev), d_image=img, **kw)
        return mask, img.cpu().numpy().astype(np.float64)
    finally:
        L.lmosem_destroy(ctx)


@pytest.mark.parametrize("name,n_ev,ns,ni,thr,dil", [("tiny16", 2000, 4, 3, 0.15, 1),
                                                     ("dat32", 20000, 6, 2, 0.1, 0),
                                                     ("dat32", 20000, 1, 4, 0.02, 2)])
def test_binned_support_matches_oracle(L, name, n_ev, ns, ni, thr, dil):
    ph, g, *_ = S.workload(name)
    ev = S.simulate_events(ph, g, n_ev, seed=41)
    ny, nx = ph.mu.shape
    A = binned.projector(g, nx, ny, ph.pixel_mm)
    c = binned.sinogram(g, ev.angle, ev.u_mm)
    f_ref, _, _ = binned.osem(A, c, ns, ni)
    mask, img = _gpu_support(L, ph, g, ev, n_subsets=ns, n_iters=ni, threshold=thr, dilate=dil)
    assert oracle.rel_l2(img, f_ref) <= 1e-4
    m_ref = binned.support_mask(f_ref, nx, ny, thr, dil)
    near = np.abs(f_ref / f_ref.max() - thr) <= 1e-3 * thr
    allowed = binned.support_mask(near.astype(float), nx, ny, 0.5, dil) if near.any() else near
    bad = (mask.astype(bool) != m_ref) & ~allowed
    assert not bad.any(), np.nonzero(bad)


def test_binned_support_shrinks_the_support_and_keeps_the_activity(L):
    ph, g, J, ns, ni = S.workload("dat64")
    ev = S.simulate_events(ph, g, J, seed=42)
    mask, _ = _gpu_support(L, ph, g, ev)
    act = ph.activity.reshape(-1)
    mu = ph.mu.reshape(-1)
    assert np.all(mask[act > 0.5 * act.max() / 8.0])          # every pixel with brain-level activity
    assert mask.sum() < 0.95 * np.count_nonzero(mu > 0)         # smaller than {mu > 0}
    assert not np.any(mask[mu == 0])                            # and no air
    # reconstructions on both supports agree on the striatal ROI means
    full = gpu_reconstruct(ph, g, ev, ns, ni)
    small = gpu_reconstruct(ph, g, ev, ns, ni, support=mask.reshape(ph.mu.shape))
    img = lambda out: np.bincount(out["support"], weights=out["f"], minlength=act.size)
    for k, w in ph.rois.items():
        w = w.reshape(-1)
        a, b = np.dot(w, img(full)), np.dot(w, img(small))
        assert abs(b / a - 1.0) < 0.05, (k, a, b)
    assert small["model_bytes"] < full["model_bytes"]


def test_binned_support_rejects_bad_arguments(L):
    import torch
    ph, g, *_ = S.workload("tiny16")
    ev = S.simulate_events(ph, g, 100, seed=43)
    for kw in (dict(n_subsets=0), dict(n_subsets=33), dict(n_iters=0), dict(threshold=0.0),
               dict(threshold=1.5), dict(dilate=-1), dict(dilate=9)):
        with pytest.raises(L.LmosemError) as ei:
            _gpu_support(L, ph, g, ev, **kw)
        assert ei.value.status == L.EINVAL, kw
    bad = S.Events(ev.angle.copy(), ev.u_mm.copy(), ev.e_kev.copy(), ev.order)
    bad.angle[5] = 32
    with pytest.raises(L.LmosemError) as ei:
        _gpu_support(L, ph, g, bad)
    assert ei.value.status == L.EINVAL
