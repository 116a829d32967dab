"""The pins have teeth: plausible mistakes planted on the CPU each fail a
check that the unmodified oracle passes.

* EM (Eqs. 3, 7 and 8): mistakes in copies of the update and the
  log-likelihood break count conservation at every sub-iteration, the
  single-pixel closed form, or the likelihood maximum at the MLEM fixed
  point.
* Event model (Eqs. 2 and 4): each mistake planted in the brute-force path
  enumeration makes it disagree with the oracle far beyond the 1e-12 bound of
  the enumeration pin, so the same mistake in the oracle would fail it.
* Surrogate MLP: mistakes planted in the backward pass fail the central-
  difference check of the gradients.
* Support initialiser: mistakes planted in copies of its bin-integrated
  projector fail the quadrature check."""
import numpy as np
import pytest

import oracle
from paper_2002_12471_gb300 import synthetic as S


@pytest.fixture(scope="module")
def tiny():
    ph, g, J, _, _ = S.workload("tiny16")
    g = dict(g, pixel_mm=ph.pixel_mm)
    ev = S.simulate_events(ph, g, J, seed=1)
    P = oracle.Problem(g, ph.mu)
    p = P.model(ev.angle, ev.u_mm, ev.e_kev)
    s4 = P.sensitivity(4)
    supp = np.zeros_like(ph.mu)
    supp[8, 7] = 1
    P1 = oracle.Problem(g, ph.mu, support=supp)
    ev1 = S.simulate_events(ph, g, 400, seed=2)
    return dict(p=p, ev=ev, s4=s4, s1=P.sensitivity(1)[0], J=J,
                p1=P1.model(ev1.angle, ev1.u_mm, ev1.e_kev), ev1=ev1, s1pix=P1.sensitivity(4))


# ------------------------------------------------------------------ checks

def conserves_counts(update, d, T=2.5):
    p, s, ev = d["p"], d["s4"], d["ev"]
    f = oracle.initial_image(d["J"], s.sum(0), T)
    sub = oracle.subset_of(ev.angle, 4)
    for _ in range(2):
        for i in range(4):
            rows = p[sub == i]
            n_pos = int(np.sum(rows @ f > 0))
            f = update(rows, f, s[i], T, s.sum(0))
            if abs(T * np.dot(s[i], f) - n_pos) > 1e-10 * n_pos:
                return False
    return True


def single_pixel_closed_form(update, d, T=0.7):
    p, s, ev = d["p1"], d["s1pix"], d["ev1"]
    sub = oracle.subset_of(ev.angle, 4)
    f = np.array([5.0])
    for i in range(4):
        f = update(p[sub == i], f, s[i], T, s.sum(0))
        if abs(f[0] - np.sum(sub == i) / (T * s[i, 0])) > 1e-11 * f[0]:
            return False
    return True


def fixed_point_is_a_likelihood_maximum(loglik, d, n_iters=400, seed=3):
    """After MLEM iterations the image is close to the maximiser, so small
    non-negative perturbations along the support lower the likelihood."""
    p, s = d["p"], d["s1"]
    f = oracle.initial_image(d["J"], s)
    for _ in range(n_iters):
        f = oracle.osem_subiteration(p, f, s)
    base = loglik(p, f, s)
    rng = np.random.default_rng(seed)
    for _ in range(8):
        df = rng.normal(size=f.shape) * 0.05 * f
        if loglik(p, f + df, s) > base + 1e-9 * abs(base):
            return False
    return True


def oracle_update(p_sub, f, s_i, T, s_total):
    return oracle.osem_subiteration(p_sub, f, s_i, T)


# ------------------------------------------------------------------ mutants

def m_total_sensitivity(p_sub, f, s_i, T, s_total):
    """Normalises by the total sensitivity instead of the subset's."""
    return oracle.osem_subiteration(p_sub, f, s_total, T)


def m_dropped_T(p_sub, f, s_i, T, s_total):
    """Forgets the acquisition time in the normalisation."""
    return oracle.osem_subiteration(p_sub, f, s_i, 1.0)


def m_squared_denominator(p_sub, f, s_i, T, s_total):
    """Back-projects 1 / y_j^2 instead of 1 / y_j."""
    y = p_sub @ f
    b = p_sub.T @ (1.0 / y ** 2)
    return f * b / (T * s_i)


def m_damped(p_sub, f, s_i, T, s_total):
    """A square-root (damped) multiplicative step: same fixed point, but not
    the EM update."""
    y = p_sub @ f
    b = p_sub.T @ (1.0 / y)
    return f * np.sqrt(b / (T * s_i))


def m_forward_with_ones(p_sub, f, s_i, T, s_total):
    """Forward-projects a uniform image instead of the current one."""
    y = p_sub @ np.ones_like(f)
    b = p_sub.T @ (1.0 / y)
    return f * b / (T * s_i)


def ll_flipped_sensitivity(p, f, s_total, T=1.0):
    return float(np.sum(np.log(T * (p @ f))) + T * np.dot(s_total, f))


def ll_no_log(p, f, s_total, T=1.0):
    return float(np.sum(T * (p @ f)) - T * np.dot(s_total, f))


# ------------------------------------------------------------------ tests

def test_the_oracle_passes_every_check(tiny):
    assert conserves_counts(oracle_update, tiny)
    assert single_pixel_closed_form(oracle_update, tiny)
    assert fixed_point_is_a_likelihood_maximum(oracle.loglik, tiny)


@pytest.mark.parametrize("mutant", [m_total_sensitivity, m_dropped_T, m_squared_denominator,
                                    m_damped, m_forward_with_ones],
                         ids=lambda m: m.__name__)
def test_planted_update_mistakes_fail_a_pin(tiny, mutant):
    results = {"count conservation": conserves_counts(mutant, tiny),
               "single-pixel closed form": single_pixel_closed_form(mutant, tiny)}
    assert not all(results.values()), results


@pytest.mark.parametrize("mutant", [ll_flipped_sensitivity, ll_no_log], ids=lambda m: m.__name__)
def test_planted_likelihood_mistakes_fail_the_maximum_check(tiny, mutant):
    assert not fixed_point_is_a_likelihood_maximum(mutant, tiny)


@pytest.mark.parametrize("mistake", ["response_at_n", "no_inv_2pi_r", "flipped_angle", "det_from_n",
                                     "mu_at_n"])
def test_planted_model_mistakes_break_the_enumeration_pin(mistake):
    from tests.test_oracle_model import brute_force_row, tiny_geom
    rng = np.random.default_rng(1)
    n, dpx = 5, 7.0
    mu = rng.uniform(0.005, 0.03, (n, n)) * (rng.uniform(0, 1, (n, n)) > 0.25)
    g = tiny_geom(n_angles=4, angle0_rad=0.37, radius_mm=45.0)
    g["pixel_mm"] = dpx
    P = oracle.Problem(g, mu, support=np.ones((n, n), dtype=bool))
    a = rng.integers(0, 4, 6).astype(np.int32)
    u = rng.uniform(-15, 15, 6)
    e = rng.uniform(100, 175, 6)
    p = P.model(a, u, e)
    worst = 0.0
    for j in range(6):
        good = brute_force_row(g, mu, dpx, P.support, int(a[j]), u[j], e[j])
        bad = brute_force_row(g, mu, dpx, P.support, int(a[j]), u[j], e[j], mistake=mistake)
        np.testing.assert_allclose(p[j], good, rtol=1e-12, atol=1e-16 * good.max())
        worst = max(worst, float(np.max(np.abs(p[j] - bad) / (1e-12 * np.abs(good) + 1e-16 * good.max()))))
    assert worst > 1e3, worst


# ------------------------------------------------------------------ MLP oracle

def _fd_agrees(seed=1):
    """The central-difference check of the MLP oracle's gradients, as a
    predicate (the loss comes from the forward pass alone)."""
    from oracle import mlp
    rng = np.random.default_rng(seed)
    params = mlp.init_params(3, (6, 16, 12, 8, 1))
    for W, b in params:
        b += rng.normal(0, 0.3, b.shape)
    X = rng.normal(0, 1, (40, 6))
    t = rng.normal(0, 1, 40)
    _, grads = mlp.mse_loss_and_grad(params, X, t)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            for ix in list(zip(*[rng.integers(0, s, 4) for s in arr.shape])):
                old = arr[ix]
                arr[ix] = old + h
                lp = float(np.mean((mlp.forward(params, X)[0] - t) ** 2))
                arr[ix] = old - h
                lm = float(np.mean((mlp.forward(params, X)[0] - t) ** 2))
                arr[ix] = old
                if abs(g[ix] - (lp - lm) / (2 * h)) > 1e-6 * abs(g[ix]) + 1e-9:
                    return False
    return True


def _backward_no_relu_mask(params, cache, dy):
    g = np.asarray(dy, dtype=np.float64)[:, None]
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        h, z = cache[k]
        W, _ = params[k]
        grads[k] = [g.T @ h, g.sum(axis=0)]
        g = g @ W
    return grads


def _backward_mean_bias(params, cache, dy):
    g = np.asarray(dy, dtype=np.float64)[:, None]
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        h, z = cache[k]
        if k < len(params) - 1:
            g = g * (z > 0.0)
        W, _ = params[k]
        grads[k] = [g.T @ h, g.mean(axis=0)]
        g = g @ W
    return grads


def _backward_relu_value_as_slope(params, cache, dy):
    """Multiplies by the ReLU's value instead of its slope."""
    g = np.asarray(dy, dtype=np.float64)[:, None]
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        h, z = cache[k]
        if k < len(params) - 1:
            g = g * np.maximum(z, 0.0)
        W, _ = params[k]
        grads[k] = [g.T @ h, g.sum(axis=0)]
        g = g @ W
    return grads


def test_mlp_oracle_passes_the_difference_check():
    assert _fd_agrees()


@pytest.mark.parametrize("mutant", [_backward_no_relu_mask, _backward_mean_bias,
                                    _backward_relu_value_as_slope],
                         ids=lambda m: m.__name__)
def test_planted_backward_mistakes_fail_the_difference_check(monkeypatch, mutant):
    from oracle import mlp
    monkeypatch.setattr(mlp, "backward", mutant)
    assert not _fd_agrees()


# ------------------------------------------------------------------ support initialiser

def _projector_agrees_with_quadrature(projector):
    """The quadrature check of the support initialiser's projector, as a
    predicate: bin masses of the Gaussian collimator response."""
    import math

    from scipy import integrate

    from oracle import binned
    g = S.geometry(8, 12, 6.0, 60.0)
    nx = ny = 8
    dpx = 7.0
    A = projector(g, nx, ny, dpx)
    u, sig = binned.geometry_arrays(g, nx, ny, dpx)
    rng = np.random.default_rng(0)
    w = g["bin_mm"]
    for _ in range(25):
        a, k, n = rng.integers(0, g["n_angles"]), rng.integers(0, g["n_bins"]), rng.integers(0, nx * ny)
        lo = -0.5 * g["n_bins"] * w + k * w
        dens = lambda x: math.exp(-0.5 * ((x - u[a, n]) / sig[a, n]) ** 2) / (sig[a, n] * math.sqrt(2 * math.pi))
        ref, _ = integrate.quad(dens, lo, lo + w, epsabs=1e-14, epsrel=1e-12)
        if abs(A[a, k, n] - ref) > 1e-9 * ref + 1e-14:
            return False
    return True


def _projector_without_sqrt2(g, nx, ny, pixel_mm):
    """erf of (edge - u) / sigma, missing the 1/sqrt(2)."""
    from oracle import binned
    u, sigma = binned.geometry_arrays(g, nx, ny, pixel_mm)
    w = g["bin_mm"]
    edges = -0.5 * g["n_bins"] * w + w * np.arange(g["n_bins"] + 1)
    E = binned._erf((edges[None, :, None] - u[:, None, :]) / sigma[:, None, :])
    return 0.5 * (E[:, 1:, :] - E[:, :-1, :])


def _projector_edges_from_zero(g, nx, ny, pixel_mm):
    """Bin edges counted from the detector centre instead of its edge."""
    import math

    from oracle import binned
    u, sigma = binned.geometry_arrays(g, nx, ny, pixel_mm)
    w = g["bin_mm"]
    edges = w * np.arange(g["n_bins"] + 1)
    E = binned._erf((edges[None, :, None] - u[:, None, :]) / (math.sqrt(2.0) * sigma[:, None, :]))
    return 0.5 * (E[:, 1:, :] - E[:, :-1, :])


def test_support_projector_passes_and_planted_mistakes_fail_quadrature():
    from oracle import binned
    assert _projector_agrees_with_quadrature(binned.projector)
    assert not _projector_agrees_with_quadrature(_projector_without_sqrt2)
    assert not _projector_agrees_with_quadrature(_projector_edges_from_zero)
