"""The allocation-free sub-iteration entry point, for callers that cannot call
cudaMalloc (their own allocator owns the device memory, or their loop must
not make calls that can synchronise the device).  It must give the same image
as the context path's lmosem_iterate on the same model rows, two calls in a
row.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def test_noalloc_subiteration_matches_iterate_twice():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, J, seed=11)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream)
    try:
        nsup = L.lmosem_n_support(ctx)
        sens = torch.zeros((1, nsup), dtype=torch.float64, device=dev)
        L.lmosem_sensitivity(ctx, 1, sens)
        a = torch.from_numpy(ev.angle).to(dev)
        u = torch.from_numpy(ev.u_mm).to(dev)
        e = torch.from_numpy(ev.e_kev).to(dev)
        L.lmosem_build_model(ctx, a, u, e, 1, "fp32")
        # the context's model rows, copied into a caller-owned padded buffer
        rows = torch.zeros((J, nsup), dtype=torch.float32, device=dev)
        L.lmosem_model_rows(ctx, torch.arange(J, dtype=torch.int64, device=dev), rows)
        ld = (nsup + 4 + 3) // 4 * 4           # padded row stride
        padded = torch.zeros((J, ld), dtype=torch.float32, device=dev)
        padded[:, :nsup] = rows
        f_ref = torch.zeros(nsup, dtype=torch.float32, device=dev)
        L.lmosem_init_image(ctx, 1.0, f_ref)
        f_na = f_ref.clone()
        for call in range(2):
            L.lmosem_iterate(ctx, 1, 1.0, f_ref)     # one subset: one sub-iteration
            L.lmosem_osem_subiter_noalloc(padded, nsup, f_na, sens[0], 1.0, stream=stream)
            torch.cuda.synchronize()
            got, want = f_na.cpu().numpy(), f_ref.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert oracle.rel_l2(got, want) <= 1e-5, (call, oracle.rel_l2(got, want))
        # sizes beyond the static scratch array are rejected before any launch
        big = torch.zeros((4, 16388), dtype=torch.float32, device=dev)
        fb = torch.ones(16388, dtype=torch.float32, device=dev)
        sb = torch.ones(16388, dtype=torch.float64, device=dev)
        with pytest.raises(L.LmosemError) as ei:
            L.lmosem_osem_subiter_noalloc(big, 16388, fb, sb, 1.0, stream=stream)
        assert ei.value.status == L.EINVAL
    finally:
        L.lmosem_destroy(ctx)
