"""Pins of the oracle's gradient formulas (envelope theorem on the dual)
against central finite differences of the oracle's high-precision solves."""
import numpy as np
import pytest

from oracle import grad, uot


def small_case(seed=3, N=5):
    rng = np.random.default_rng(seed)
    pix = uot.grid_index(N, 2) / N
    mu = rng.uniform(0.5, 1.5, N * N) / N ** 2
    nu = rng.uniform(0.5, 1.5, N * N) / N ** 2 * 1.2
    return pix, pix.copy(), mu, nu


@pytest.mark.parametrize("lam", [0.5, 3.0])
def test_gradients_match_central_differences(lam):
    X, Y, mu, nu = small_case()
    eps = 0.02
    S0, a, b = grad.value(mu, nu, X, Y, eps, lam)
    g_mu, g_nu, g_x = grad.dual_gradients(a, b, X, Y, mu, nu, eps, lam)
    h = 1e-4
    rng = np.random.default_rng(0)
    for k in rng.choice(len(mu), 3, replace=False):
        e = np.zeros_like(mu)
        e[k] = h * mu[k]
        fd = (grad.value(mu + e, nu, X, Y, eps, lam)[0] - grad.value(mu - e, nu, X, Y, eps, lam)[0]) / (2 * e[k])
        assert abs(fd - g_mu[k]) <= 1e-6 * (1 + abs(g_mu[k]))
        e = np.zeros_like(nu)
        e[k] = h * nu[k]
        fd = (grad.value(mu, nu + e, X, Y, eps, lam)[0] - grad.value(mu, nu - e, X, Y, eps, lam)[0]) / (2 * e[k])
        assert abs(fd - g_nu[k]) <= 1e-6 * (1 + abs(g_nu[k]))
        for dim in range(2):
            Xp, Xm = X.copy(), X.copy()
            Xp[k, dim] += h
            Xm[k, dim] -= h
            fd = (grad.value(mu, nu, Xp, Y, eps, lam)[0] - grad.value(mu, nu, Xm, Y, eps, lam)[0]) / (2 * h)
            assert abs(fd - g_x[k, dim]) <= 1e-6 * (1 + abs(g_x[k, dim])) + 1e-9


def test_gradient_closed_form_at_optimum():
    """At the optimum P_X = e^{-alpha/lam} mu and P_Y = e^{-beta/lam} nu
    (stationarity of Eq. dual-problem), so dS/dmu reduces to
    eps(|nu| - e^{-alpha/lam}) - lam(e^{-alpha/lam} - 1), and likewise for nu.
    The Y side holds to rounding (the last half-step was a Y-half, Eq.
    sinkhorn-iters-ot); the X side to the square root of the stopping gap."""
    X, Y, mu, nu = small_case(5)
    eps, lam = 0.03, 1.0
    S0, a, b = grad.value(mu, nu, X, Y, eps, lam)
    g_mu, g_nu, _ = grad.dual_gradients(a, b, X, Y, mu, nu, eps, lam)
    ea = np.exp(-a / lam)
    eb = np.exp(-b / lam)
    assert np.allclose(g_nu, eps * (mu.sum() - eb) - lam * (eb - 1.0), rtol=0, atol=1e-13)
    assert np.allclose(g_mu, eps * (nu.sum() - ea) - lam * (ea - 1.0), rtol=0, atol=1e-7)
