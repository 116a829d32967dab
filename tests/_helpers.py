"""Shared test helpers: run the CUDA path through the C ABI and the oracle
on the same seeded inputs."""
import numpy as np

import oracle
from paper_2002_12471_gb300 import synthetic as S


def oracle_problem(ph, g, support=None):
    return oracle.Problem(dict(g, pixel_mm=ph.pixel_mm), ph.mu, support=support)


def gpu_reconstruct(ph, g, ev, n_subsets, n_iters, fmt="fp32", T=1.0, support=None,
                    rows=None, loglik=False, k_sigma=0.0, **opts):
    """Sensitivity, model build and n_iters OSEM iterations on cuda:0.
    Returns a dict with the image, sensitivities, optional model rows (by
    original event index) and optional per-iteration log-likelihoods."""
    import torch

    import paper_2002_12471_gb300.lmosem as L

    dev = torch.device("cuda:0")
    out = {}
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, support=support, k_sigma=k_sigma,
                          stream=torch.cuda.current_stream(), **opts)
    try:
        nsup = L.lmosem_n_support(ctx)
        out["support"] = L.lmosem_support(ctx)
        a = torch.from_numpy(np.ascontiguousarray(ev.angle)).to(dev)
        u = torch.from_numpy(np.ascontiguousarray(ev.u_mm)).to(dev)
        e = torch.from_numpy(np.ascontiguousarray(ev.e_kev)).to(dev)
        sens = torch.zeros((n_subsets, nsup), dtype=torch.float64, device=dev)
        L.lmosem_sensitivity(ctx, n_subsets, sens)
        L.lmosem_build_model(ctx, a, u, e, n_subsets, fmt)
        try:
            out["terms"] = L.lmosem_model_terms(ctx)
        except L.LmosemError:   # a build without path-sum rows
            out["terms"] = None
        if rows is not None:
            ids = torch.as_tensor(np.asarray(rows, dtype=np.int64), device=dev)
            buf = torch.zeros((len(rows), nsup), dtype=torch.float32, device=dev)
            L.lmosem_model_rows(ctx, ids, buf)
            out["rows"] = buf.cpu().numpy().astype(np.float64)
        f = torch.zeros(nsup, dtype=torch.float32, device=dev)
        L.lmosem_init_image(ctx, T, f)
        out["f0"] = f.cpu().numpy().astype(np.float64)
        ll = torch.zeros(max(1, n_iters), dtype=torch.float64, device=dev) if loglik else None
        L.lmosem_iterate(ctx, n_iters, T, f, ll)
        torch.cuda.synchronize()
        out["f"] = f.cpu().numpy().astype(np.float64)
        out["sens"] = sens.cpu().numpy()
        if loglik:
            out["loglik"] = ll.cpu().numpy()
        out["launches"] = L.lmosem_launch_count(ctx)
        out["model_bytes"] = L.lmosem_model_bytes(ctx)
    finally:
        L.lmosem_destroy(ctx)
    return out


def row_close(p_gpu, p_ref, rel=2e-4, floor=2e-6):
    """Entry-wise bound: |gpu - ref| <= rel |ref| + floor * max_n ref_jn.
    Returns the worst ratio of the deviation to that bound (<= 1 passes)."""
    bound = rel * np.abs(p_ref) + floor * p_ref.max(axis=1, keepdims=True)
    return float(np.max(np.abs(p_gpu - p_ref) / bound))
