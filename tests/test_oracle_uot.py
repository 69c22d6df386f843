"""Pins of the oracle's global UOT layer against facts fixed by the paper and by
convex analysis (brute-force dual maximisation, the PD-gap identity, the
balanced limit, optimality conditions)."""
import numpy as np
import pytest

from oracle import brute, uot
from oracle.cell import prox_root

INF = float("inf")


def tiny_problem(seed, N=3, d=2):
    rng = np.random.default_rng(seed)
    pix = uot.grid_index(N, d)
    C = uot.sq_cost(pix, pix, 1.0 / N)
    n = len(pix)
    return rng.uniform(0.3, 1.7, n) / n, rng.uniform(0.3, 1.7, n) / n, C


@pytest.mark.parametrize("seed,eps,lam", [(0, 0.05, 0.7), (1, 0.2, 3.0), (2, 0.02, 0.1)])
def test_sinkhorn_fixed_point_is_brute_force_dual_optimum(seed, eps, lam):
    """Sinkhorn's fixed point (Eq. sinkhorn-iters-ot) maximises the dual
    (Eq. dual-problem); zero duality gap at the optimum (Theorem 2.2)."""
    mu, nu, C = tiny_problem(seed)
    a, b = brute.dual_newton(mu, nu, C, eps, lam)
    al, be, it, gap = uot.full_sinkhorn(mu, nu, C, eps, lam, err=0.0, maxit=3000)
    # Sinkhorn stalls in FP64 along the slowly contracting direction
    # (alpha + t, beta - t) at a few 1e-8; the plans agree far more tightly.
    scale = max(1.0, np.abs(a).max())
    assert np.abs(a - al).max() < 1e-7 * scale
    assert np.abs(b - be).max() < 1e-7 * scale
    pi_s = uot.plan(al, be, C, mu, nu, eps)
    assert np.abs(pi_s - uot.plan(a, b, C, mu, nu, eps)).sum() < 1e-8 * pi_s.sum()
    pi = uot.plan(a, b, C, mu, nu, eps)
    P = uot.primal_score(pi, C, mu, nu, eps, lam)
    D = uot.dual_score(a, b, C, mu, nu, eps, lam)
    assert abs(P - D) < 1e-12 * max(1.0, abs(P))


@pytest.mark.parametrize("eps,lam", [(0.05, 0.5), (0.01, 2.0), (0.3, 10.0)])
def test_pd_gap_identity_after_y_half(eps, lam):
    """E(pi^l) - D(alpha^l, beta^l) = lam KL(P_X pi^l | e^{-alpha^l/lam} mu)
    after every Y-half (Eq. PD-gap / PD-gap-KL)."""
    mu, nu, C = tiny_problem(5, N=4)
    beta = np.zeros(len(nu))
    for _ in range(6):
        alpha = uot.x_half(beta, C, nu, eps, lam)
        beta = uot.y_half(alpha, C, mu, eps, lam)
        pi = uot.plan(alpha, beta, C, mu, nu, eps)
        lhs = uot.primal_score(pi, C, mu, nu, eps, lam) - uot.dual_score(alpha, beta, C, mu, nu, eps, lam)
        rhs = lam * uot.pd_gap_over_lam(alpha, uot.x_marginal(alpha, beta, C, mu, nu, eps), mu, lam)
        assert abs(lhs - rhs) <= 1e-10 * max(abs(rhs), 1e-14) + 1e-15


def test_pd_gap_identity_with_background_measure():
    """The same identity for the cell problem with nu_- > 0, where the Y-half
    is the root of Eq. proxdiv-problem (Section 5.1)."""
    rng = np.random.default_rng(7)
    mu, nu, C = tiny_problem(8, N=3)
    mu = mu[:4]
    C = C[:4]
    num = rng.uniform(0.0, 1.5, len(nu)) * nu
    eps, lam = 0.04, 0.8
    alpha = np.zeros(4)
    for _ in range(5):
        z = uot.lse((alpha[:, None] - C) / eps + np.log(mu)[:, None], 0)
        beta = prox_root(z, num / nu, eps, lam)
        pi = uot.plan(alpha, beta, C, mu, nu, eps)
        lhs = (uot.primal_score(pi, C, mu, nu, eps, lam, num)
               - uot.dual_score(alpha, beta, C, mu, nu, eps, lam, num))
        rhs = lam * uot.kl(pi.sum(1), np.exp(-alpha / lam) * mu)
        assert abs(lhs - rhs) <= 1e-9 * abs(rhs) + 1e-14
        alpha = uot.x_half(beta, C, nu, eps, lam)


def balanced_sinkhorn_textbook(mu, nu, C, eps, iters):
    """Matrix-scaling Sinkhorn for balanced entropic OT: u = mu/(K v),
    v = nu/(K^T u), K = exp(-C/eps)."""
    K = np.exp(-C / eps)
    v = nu.copy()  # beta = 0 in the potential form pi = e^{(a+b-c)/eps} mu nu
    for _ in range(iters):
        u = mu / (K @ v)
        v = nu / (K.T @ u)
    return u[:, None] * K * v[None, :]


def test_balanced_limit_lambda_infinity():
    """lam = inf gives the balanced Sinkhorn iterates (Definition 2.3, last
    sentence); plans for finite lam converge to it as lam grows."""
    mu, nu, C = tiny_problem(3, N=4)
    nu = nu * (mu.sum() / nu.sum())
    eps = 0.1
    al, be, it, _ = uot.full_sinkhorn(mu, nu, C, eps, INF, err=-1.0, maxit=300)
    assert it == 300
    pi_inf = uot.plan(al, be, C, mu, nu, eps)
    pi_txt = balanced_sinkhorn_textbook(mu, nu, C, eps, 300)
    assert np.abs(pi_inf - pi_txt).max() < 1e-13
    errs = []
    for lam in (1e0, 1e1, 1e2, 1e3):
        a, b, _, _ = uot.full_sinkhorn(mu, nu, C, eps, lam, err=1e-15, maxit=20000)
        errs.append(np.abs(uot.plan(a, b, C, mu, nu, eps) - pi_txt).sum())
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-2 * errs[0]


@pytest.mark.parametrize("lam", [0.3, 1.0, 5.0])
def test_optimality_conditions_at_convergence(lam):
    """Eq. optimality-conditions-KL: e^{-alpha/lam} mu = P_X pi and
    e^{-beta/lam} nu = P_Y pi at the optimum."""
    mu, nu, C = tiny_problem(11, N=4)
    a, b, it, gap = uot.full_sinkhorn(mu, nu, C, 0.05, lam, err=-1.0, maxit=4000)
    pi = uot.plan(a, b, C, mu, nu, 0.05)
    assert np.abs(np.exp(-a / lam) * mu - pi.sum(1)).sum() < 1e-8
    assert np.abs(np.exp(-b / lam) * nu - pi.sum(0)).sum() < 1e-12


def test_kl_and_lse_basic_values():
    """KL(a|b) = 0 iff a = b, KL(0|b) = |b|, and the LSE of equal entries."""
    b = np.array([0.2, 0.5, 1.0])
    assert uot.kl(b, b) == 0.0
    assert abs(uot.kl(np.zeros(3), b) - b.sum()) < 1e-15
    assert abs(uot.kl(2 * b, b) - (2 * np.log(2) - 1) * b.sum()) < 1e-15
    M = np.full((2, 5), -1000.0)
    assert np.allclose(uot.lse(M, 1), -1000.0 + np.log(5), rtol=0, atol=1e-12)
