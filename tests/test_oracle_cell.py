"""Pins of the oracle's cell solver: the Y-half root, the rho = 0 reduction to
the closed-form Sinkhorn, brute-force dual maximisation with a background
measure, and the paper's worked example (Remark 4.5)."""
import os

import numpy as np
import pytest

from oracle import brute, uot
from oracle.cell import cell_sinkhorn, prox_residual, prox_root

HERE = os.path.dirname(os.path.abspath(__file__))
INF = float("inf")


def bisect_root(z, rho, eps, lam):
    """Independent scalar root of Eq. proxdiv-problem by bisection."""
    out = np.empty_like(z)
    for k in range(len(z)):
        lo, hi = -1e4, 1e4
        for _ in range(400):
            mid = 0.5 * (lo + hi)
            if prox_residual(mid, z[k], rho[k], eps, lam) > 0:
                hi = mid
            else:
                lo = mid
        out[k] = 0.5 * (lo + hi)
    return out


@pytest.mark.parametrize("eps,lam", [(1e-3, 1.0), (0.05, 0.1), (1e-5, 10.0)])
def test_prox_root_matches_bisection(eps, lam):
    rng = np.random.default_rng(1)
    z = rng.uniform(-30, 30, 64) / max(eps, 1e-3)
    rho = np.where(rng.random(64) < 0.2, 0.0, rng.uniform(0, 3, 64))
    rho[:4] = [1e-12, 1e3, 0.999, 1.0]
    b = prox_root(z, rho, eps, lam)
    ref = bisect_root(z, rho, eps, lam)
    assert np.abs(b - ref).max() <= 1e-11 * np.maximum(1, np.abs(ref)).max()


def test_prox_root_rho_zero_closed_form():
    """rho = 0 gives the closed form of Eq. sinkhorn-iters-ot exactly."""
    z = np.linspace(-50, 50, 21)
    for eps, lam in [(0.01, 1.0), (0.2, 0.3)]:
        b = prox_root(z, np.zeros_like(z), eps, lam)
        assert np.array_equal(b, -uot.kappa(eps, lam) * z)
    b = prox_root(z, np.zeros_like(z), 0.1, INF)
    assert np.allclose(b, -0.1 * z, rtol=0, atol=1e-14)


def test_cell_with_rho_zero_reproduces_global_sinkhorn():
    """nu_- = 0 and a single cell J = I gives the global problem (Section 5.1,
    'Stopping criterion'): the cell iterates equal full_sinkhorn's."""
    rng = np.random.default_rng(2)
    pix = uot.grid_index(5, 2)
    C = uot.sq_cost(pix, pix, 0.2)
    mu = rng.uniform(0.5, 1.5, 25) / 25
    nu = rng.uniform(0.5, 1.5, 25) / 25
    eps, lam = 0.03, 0.7
    a_ref, b_ref, it_ref, gap_ref = uot.full_sinkhorn(mu, nu, C, eps, lam, err=1e-7)
    alpha0 = uot.x_half(np.zeros(25), C, nu, eps, lam)
    res = cell_sinkhorn(mu, nu, np.zeros(25), C, eps, lam, alpha0, err=1e-7)
    assert res.iters == it_ref
    assert np.abs(res.alpha - a_ref).max() < 1e-13
    assert np.abs(res.beta - b_ref).max() < 1e-13
    assert abs(res.gap - gap_ref) < 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cell_solve_is_brute_force_cell_dual_optimum(seed):
    """The cell Sinkhorn's limit maximises the cell dual with the
    -<beta, nu_{-J}> term (Eq. cell-dual-problem)."""
    rng = np.random.default_rng(seed)
    pix = uot.grid_index(4, 2)
    C = uot.sq_cost(pix[:6], pix, 0.25)
    mu = rng.uniform(0.5, 1.5, 6) / 16
    nu = rng.uniform(0.5, 1.5, 16) / 16
    rho = rng.uniform(0, 2, 16)
    eps, lam = 0.05, [0.5, 2.0, 8.0][seed]
    a, b = brute.dual_newton(mu, nu, C, eps, lam, nu_minus=rho * nu)
    res = cell_sinkhorn(mu, nu, rho, C, eps, lam, np.zeros(6), err=-1.0, maxit=3000)
    # FP64 Sinkhorn stalls at a few 1e-8 along (alpha + t, beta - t)
    assert np.abs(res.alpha - a).max() < 1e-7
    assert np.abs(res.beta - b).max() < 1e-7
    pi_s = uot.plan(res.alpha, res.beta, C, mu, nu, eps)
    assert np.abs(pi_s - uot.plan(a, b, C, mu, nu, eps)).sum() < 1e-8 * pi_s.sum()


def load_worked_example():
    rows = []
    with open(os.path.join(HERE, "golden", "worked_example_remark_4_5.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def stationary_ab(M, eps):
    """Independent 2-variable solve of the discretised Remark 4.5 problem with
    eps > 0: minimise eps/2 M[phi(a/M) + phi(b/M)] + M phi((a+b)/(2M))
    + phi(a)/2 + phi(b+1)/2 over a, b > 0 (Newton in log a, log b)."""
    u = np.array([np.log(np.sqrt(2 * M)), np.log(M)])
    for _ in range(200):
        a, b = np.exp(u)
        s = a + b
        g = np.array([eps * np.log(a / M) + np.log(s / (2 * M)) + np.log(a),
                      eps * np.log(b / M) + np.log(s / (2 * M)) + np.log1p(b)])
        J = np.array([[eps + a / s + 1.0, b / s],
                      [a / s, eps + b / s + b / (1 + b)]])
        du = np.linalg.solve(J, -g)
        du = np.clip(du, -2, 2)
        u = u + du
        if np.abs(du).max() < 1e-15:
            break
    return np.exp(u)


@pytest.mark.parametrize("row", range(3))
def test_worked_example_remark_4_5(row):
    """Zero cost, one X point of mass M, lam = 1, nu uniform.  With a 0/1
    pattern of rho the cell optimum has densities (sqrt(2M), 0) as eps -> 0;
    with rho = 1/2 it is sqrt(1/16 + M) - 1/4 (values of Remark 4.5)."""
    M, a_ref, b_ref, f_ref = load_worked_example()[row]
    n = 8
    nu = np.full(n, 1.0 / n)
    C = np.zeros((1, n))
    pattern = np.array([0, 1] * (n // 2), float)
    for eps in (0.1, 0.01):
        res = cell_sinkhorn([M], nu, pattern, C, eps, 1.0, [0.0], err=-1.0, maxit=2000)
        dens = M * np.exp((res.alpha[0] + res.beta) / eps)
        a_e, b_e = stationary_ab(M, eps)
        assert np.allclose(dens[pattern == 0], a_e, rtol=1e-7)
        assert np.allclose(dens[pattern == 1], b_e, rtol=1e-6)
    # eps -> 0 limit against the paper's printed values
    # (deviation at eps = 3e-3 is O(eps): about 1.1e-3 for these M)
    eps = 3e-3
    res = cell_sinkhorn([M], nu, pattern, C, eps, 1.0, [0.0], err=1e-13, maxit=10000)
    assert res.converged
    dens = M * np.exp((res.alpha[0] + res.beta) / eps)
    assert np.allclose(dens[pattern == 0], a_ref, atol=2e-3)
    assert np.all(dens[pattern == 1] < 1e-12 + b_ref)
    res = cell_sinkhorn([M], nu, np.full(n, 0.5), C, eps, 1.0, [0.0], err=1e-13, maxit=10000)
    assert res.converged
    dens = M * np.exp((res.alpha[0] + res.beta) / eps)
    assert np.allclose(dens, f_ref, atol=2e-3)
