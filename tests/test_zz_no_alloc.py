"""The allocation-free sub-iteration entry point, for callers that cannot call
cudaMalloc (their own allocator owns the device memory, or their loop must
not make calls that can synchronise the device).  It must give the same image
as the context path's lmosem_iterate on the same model rows, two calls in a
row, and leave the device's free memory unchanged after its first call.  This
file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

MAX_WIDTH = 8192   # 256 threads x 8 vectors x 4 floats of the register pass


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    return L


def test_noalloc_subiteration_matches_iterate_twice():
    import torch
    L = _lib()

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
    finally:
        L.lmosem_destroy(ctx)


def test_noalloc_widest_rows_and_free_memory():
    """Rows of the widest accepted width (8192) against the FP64 oracle's
    sub-iteration on the same rows; free device memory unchanged across
    calls after the first; one column more is rejected before any launch."""
    import torch
    L = _lib()

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    n_rows = 300
    p = rng.uniform(0.0, 1.0, (n_rows, MAX_WIDTH)) * (rng.uniform(0, 1, (n_rows, MAX_WIDTH)) < 0.3)
    f0 = rng.uniform(0.5, 1.5, MAX_WIDTH)
    s = rng.uniform(0.5, 2.0, MAX_WIDTH)
    s[::97] = 0.0                               # pixels without sensitivity go to zero
    p32 = p.astype(np.float32)
    rows = torch.from_numpy(p32).to(dev)
    f = torch.from_numpy(f0.astype(np.float32)).to(dev)
    sd = torch.from_numpy(s).to(dev)
    small = torch.from_numpy(p32[:, :64].copy()).to(dev)
    fs = f[:64].clone()
    torch.cuda.synchronize()
    L.lmosem_osem_subiter_noalloc(small, 64, fs, sd[:64], 1.0, stream=stream)   # first call: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    want = f0.astype(np.float32).astype(np.float64)
    for call in range(2):
        L.lmosem_osem_subiter_noalloc(rows, MAX_WIDTH, f, sd, 2.0, stream=stream)
        torch.cuda.synchronize()
        want = oracle.osem_subiteration(p32.astype(np.float64), want, s, T=2.0)
        got = f.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        assert oracle.rel_l2(got, want) <= 1e-5, (call, oracle.rel_l2(got, want))
    assert torch.cuda.mem_get_info(dev)[0] == free0
    # one column beyond the widest row is rejected (support and row stride)
    wide = torch.zeros((4, MAX_WIDTH + 4), dtype=torch.float32, device=dev)
    fw = torch.ones(MAX_WIDTH + 1, dtype=torch.float32, device=dev)
    sw = torch.ones(MAX_WIDTH + 1, dtype=torch.float64, device=dev)
    for nsup in (MAX_WIDTH + 1, MAX_WIDTH):   # support too wide; stride too wide
        with pytest.raises(L.LmosemError) as ei:
            L.lmosem_osem_subiter_noalloc(wide, nsup, fw, sw, 1.0, stream=stream)
        assert ei.value.status == L.EINVAL
