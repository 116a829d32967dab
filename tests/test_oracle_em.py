"""Pins of the oracle's OS-LM-MLEM update (Eqs. 6-9) and log-likelihood
(Eq. 3) by invariants that the EM algebra fixes (CPU only)."""
import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S


@pytest.fixture(scope="module")
def tiny():
    ph, g, J, ns, ni = S.workload("tiny16")
    g = dict(g, pixel_mm=ph.pixel_mm)
    ev = S.simulate_events(ph, g, J, seed=1)
    P = oracle.Problem(g, ph.mu)
    p = P.model(ev.angle, ev.u_mm, ev.e_kev)
    return dict(P=P, p=p, ev=ev, s4=P.sensitivity(4), s1=P.sensitivity(1), J=J)


def test_count_conservation_every_subiteration(tiny):
    """T sum_n s^i_n f_new_n = number of subset events with y_j > 0 (the
    denominator of Eq. 7 makes every sub-iterate reproduce the counts)."""
    p, s, ev = tiny["p"], tiny["s4"], tiny["ev"]
    T = 2.5
    f = oracle.initial_image(tiny["J"], s.sum(0), T)
    sub = oracle.subset_of(ev.angle, 4)
    for it in range(3):
        for i in range(4):
            rows = p[sub == i]
            f_new = oracle.osem_subiteration(rows, f, s[i], T)
            n_pos = int(np.sum(rows @ f > 0))
            assert T * np.dot(s[i], f_new) == pytest.approx(n_pos, rel=1e-12)
            f = f_new


def test_initial_image_reproduces_counts(tiny):
    s = tiny["s4"].sum(0)
    f0 = oracle.initial_image(tiny["J"], s, T=3.0)
    assert 3.0 * np.dot(s, f0) == pytest.approx(tiny["J"], rel=1e-14)
    assert np.all(f0 == f0[0])


def test_single_pixel_support_closed_form():
    """With one emission pixel every sub-iterate is |S_i| / (T s^i)."""
    ph, g, J, ns, ni = S.workload("tiny16")
    g = dict(g, pixel_mm=ph.pixel_mm)
    ev = S.simulate_events(ph, g, 400, seed=2)
    supp = np.zeros_like(ph.mu)
    supp[8, 7] = 1
    P = oracle.Problem(g, ph.mu, support=supp)
    p = P.model(ev.angle, ev.u_mm, ev.e_kev)
    s = P.sensitivity(4)
    T = 0.7
    f = np.array([5.0])
    sub = oracle.subset_of(ev.angle, 4)
    for i in range(4):
        f = oracle.osem_subiteration(p[sub == i], f, s[i], T)
        assert f[0] == pytest.approx(np.sum(sub == i) / (T * s[i, 0]), rel=1e-13)


def test_mlem_loglik_is_monotone(tiny):
    p, s = tiny["p"], tiny["s1"]
    f = oracle.initial_image(tiny["J"], s[0])
    prev = -np.inf
    for _ in range(60):
        f = oracle.osem_subiteration(p, f, s[0])
        ll = oracle.loglik(p, f, s[0])
        assert ll >= prev - 1e-9 * abs(ll)
        prev = ll


def test_mlem_fixed_point_is_kkt():
    """After many MLEM iterations the Kuhn-Tucker conditions of the Poisson
    list-mode likelihood hold: sum_j p_jn / y_j = T s_n where f_n > 0 and
    <= T s_n where f_n vanishes."""
    ph, g, J, ns, ni = S.workload("tiny16")
    g = dict(g, pixel_mm=ph.pixel_mm)
    ev = S.simulate_events(ph, g, 20000, seed=7)
    P = oracle.Problem(g, ph.mu)
    p = P.model(ev.angle, ev.u_mm, ev.e_kev)
    s = P.sensitivity(1)[0]
    T = 1.0
    f = oracle.initial_image(len(ev), s, T)
    for _ in range(3000):
        f = oracle.osem_subiteration(p, f, s, T)
    grad = p.T @ (1.0 / (p @ f))
    big = f > 1e-3 * f.max()
    np.testing.assert_allclose(grad[big], T * s[big], rtol=2e-4)
    assert np.all(grad[~big] <= T * s[~big] * (1 + 2e-4))


def test_os_and_mlem_agree_in_the_limit(tiny):
    """Ordered subsets reach an image close to MLEM's (paper Section 4:
    'the reconstruction results were similar')."""
    p, ev = tiny["p"], tiny["ev"]
    f_os, _ = oracle.osem(p, ev.angle, tiny["s4"], 10, oracle.initial_image(tiny["J"], tiny["s4"].sum(0)))
    f_ml, _ = oracle.osem(p, ev.angle, tiny["s1"], 40, oracle.initial_image(tiny["J"], tiny["s1"][0]))
    assert oracle.rel_l2(f_os, f_ml) < 0.35
    assert tiny["s4"].sum(0) == pytest.approx(tiny["s1"][0], rel=1e-13)
