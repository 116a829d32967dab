"""Variants the paper compares, on the GPU path against the FP64 oracle:
energy windows (Sec. 3: photopeak only [143, 175] keV and [120, 175] keV
beside the full spectrum [100, 175] keV, applied to the same acquisition)
and ordered subsets against plain LM-MLEM (Sec. 4: similar images, about
N_s times faster per iteration count)."""
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


@pytest.mark.parametrize("e_lo", [143.0, 120.0])
def test_energy_window_matches_oracle(e_lo):
    ph, g_full, J, ns, ni = S.workload("tiny16")
    ev_all = S.simulate_events(ph, g_full, 3 * J, seed=21)
    keep = ev_all.e_kev >= e_lo                       # the same photons, narrower window
    ev = S.Events(ev_all.angle[keep], ev_all.u_mm[keep], ev_all.e_kev[keep], ev_all.order[keep])
    g = dict(g_full, e_lo_kev=e_lo)
    P = oracle_problem(ph, g)
    p = P.model(ev.angle, ev.u_mm, ev.e_kev)
    s = P.sensitivity(ns)
    f_ref, _ = oracle.osem(p, ev.angle, s, ni, oracle.initial_image(len(ev), s.sum(0)))
    rows = np.random.default_rng(3).choice(len(ev), min(400, len(ev)), replace=False)
    out = gpu_reconstruct(ph, g, ev, ns, ni, rows=rows)
    assert row_close(out["rows"], p[rows]) <= 1.0
    np.testing.assert_allclose(out["sens"], s, rtol=1e-5)
    assert oracle.rel_l2(out["f"], f_ref) <= 1e-4
    # a narrower window sees fewer scattered photons: lower sensitivity everywhere
    s_full = oracle_problem(ph, g_full).sensitivity(ns)
    assert np.all(s.sum(0) < s_full.sum(0))


def test_events_outside_the_window_are_rejected():
    import paper_2002_12471_gb300.lmosem as L
    ph, g_full, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g_full, 500, seed=22)
    assert np.any(ev.e_kev < 143.0)
    with pytest.raises(L.LmosemError) as ei:
        gpu_reconstruct(ph, dict(g_full, e_lo_kev=143.0), ev, ns, 1)
    assert ei.value.status == L.EINVAL


def test_ordered_subsets_against_mlem():
    ph, g, J, ns, ni = S.workload("dat32")
    ev = S.simulate_events(ph, g, J, seed=23)
    ml = gpu_reconstruct(ph, g, ev, 1, 40, loglik=True)
    os_ = gpu_reconstruct(ph, g, ev, ns, 5, loglik=True)
    ll_ml, ll_os = ml["loglik"], os_["loglik"]
    assert np.all(np.diff(ll_ml) >= -1e-9 * np.abs(ll_ml[1:]))   # EM ascent (N_s = 1)
    # MLEM iterations needed to reach what 5 OS iterations reach
    need = int(np.searchsorted(ll_ml, ll_os[-1])) + 1
    assert need >= 2 * 5, (need, ll_os[-1], ll_ml[:12])
    # and the images are similar once both have converged comparably
    assert oracle.rel_l2(os_["f"], ml["f"]) < 0.35
