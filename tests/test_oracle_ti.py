"""Pins of the translation step of the cell / global Sinkhorn (oracle/cell.py,
``ti=True``), an addition to the paper's iteration: it must maximise the
dual of Eq. dual-problem along (alpha + t, beta - t), never lower it, and
leave the fixed point of plain alternation unchanged."""
import numpy as np
import pytest

from oracle import uot
from oracle.cell import cell_sinkhorn, prox_root, ti_shift


def random_cell(seed, nx=16, ny=30, eps=2e-3, lam=1.0):
    rng = np.random.default_rng(seed)
    ix = rng.integers(0, 8, size=(nx, 2))
    iy = rng.integers(0, 10, size=(ny, 2))
    C = uot.sq_cost(ix, iy, 1.0 / 16)
    mu = rng.uniform(0.5, 1.5, nx) / 256
    nu = rng.uniform(0.5, 1.5, ny) / 256
    rho = np.where(rng.uniform(size=ny) < 0.3, 0.0, rng.uniform(0.0, 0.8, ny))
    return mu, nu, rho, C, eps, lam, rng


def y_half_cell(alpha, mu, nu, rho, C, eps, lam):
    z = uot.lse((alpha[:, None] - C) / eps + np.log(mu)[:, None], 0)
    return prox_root(z, rho, eps, lam)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_shift_maximises_cell_dual(seed):
    mu, nu, rho, C, eps, lam, rng = random_cell(seed)
    alpha = rng.normal(0, 0.02, mu.size)
    beta = y_half_cell(alpha, mu, nu, rho, C, eps, lam)
    t = ti_shift(alpha, beta, mu, nu, rho, lam)

    def F(tt):
        return uot.dual_score(alpha + tt, beta - tt, C, mu, nu, eps, lam, nu_minus=rho * nu)

    f0 = F(t)
    for d in (1e-3, 1e-4, -1e-4, -1e-3):
        assert F(t + d) <= f0 + 1e-15
    # first-order condition by central difference
    h = 1e-6
    assert abs(F(t + h) - F(t - h)) / (2 * h) <= 1e-8
    # the step does not lower the dual from the plain iterate
    assert f0 >= F(0.0) - 1e-15


@pytest.mark.parametrize("seed", [3, 4])
def test_cell_fixed_point_unchanged(seed):
    mu, nu, rho, C, eps, lam, rng = random_cell(seed, eps=5e-3)
    a0 = rng.normal(0, 0.05, mu.size)
    r0 = cell_sinkhorn(mu, nu, rho, C, eps, lam, a0, err=1e-14, maxit=200000)
    r1 = cell_sinkhorn(mu, nu, rho, C, eps, lam, a0, err=1e-14, maxit=200000, ti=True)
    assert r0.converged and r1.converged
    # the stopping test bounds KL(P_X | e^{-alpha/lam} mu) by err |mu|, which
    # pins the potentials to about lam sqrt(2 err) (the slow mass mode, a
    # common shift, is the loosest direction)
    tol = 2 * lam * np.sqrt(2 * 1e-14)
    assert np.abs(r1.alpha - r0.alpha).max() <= tol and np.abs(r1.beta - r0.beta).max() <= tol
    assert r1.iters < r0.iters


def test_cell_dual_monotone_along_iteration():
    mu, nu, rho, C, eps, lam, rng = random_cell(5, eps=1e-3)
    alpha = rng.normal(0, 0.05, mu.size)
    kap = uot.kappa(eps, lam)
    prev = -np.inf
    for _ in range(40):
        beta = y_half_cell(alpha, mu, nu, rho, C, eps, lam)
        d1 = uot.dual_score(alpha, beta, C, mu, nu, eps, lam, nu_minus=rho * nu)
        assert d1 >= prev - 1e-15
        alpha = -kap * uot.lse((beta[None, :] - C) / eps + np.log(nu)[None, :], 1)
        d2 = uot.dual_score(alpha, beta, C, mu, nu, eps, lam, nu_minus=rho * nu)
        t = ti_shift(alpha, beta, mu, nu, rho, lam)
        d3 = uot.dual_score(alpha + t, beta - t, C, mu, nu, eps, lam, nu_minus=rho * nu)
        assert d2 >= d1 - 1e-15 and d3 >= d2 - 1e-15
        alpha = alpha + t
        prev = d3


def test_global_sinkhorn_translation_same_optimum_fewer_iterations():
    """eps << lam: the plain iteration is slow along the mass mode; the
    translation step reaches the same optimum in far fewer iterations."""
    N = 10
    rng = np.random.default_rng(11)
    pix = uot.grid_index(N)
    C = uot.sq_cost(pix, pix, 1.0 / N)
    mu = rng.uniform(0.5, 1.5, N * N) / N ** 2
    nu = rng.uniform(0.5, 1.5, N * N) / N ** 2 * 1.4
    eps, lam = 4e-3, 1.0
    a0, b0, it0, g0 = uot.full_sinkhorn(mu, nu, C, eps, lam, err=1e-13, maxit=500000)
    a1, b1, it1, g1 = uot.full_sinkhorn(mu, nu, C, eps, lam, err=1e-13, maxit=500000, ti=True)
    assert g0 <= 1e-13 * mu.sum() and g1 <= 1e-13 * mu.sum()
    tol = 2 * lam * np.sqrt(2 * 1e-13)   # potentials pinned by the stopping test (see above)
    assert np.abs(a1 - a0).max() <= tol and np.abs(b1 - b0).max() <= tol
    assert it1 * 3 < it0


def test_balanced_limit_ignores_translation():
    mu, nu, rho, C, eps, lam, rng = random_cell(6)
    rho = np.zeros_like(nu)
    nu = nu * (mu.sum() / nu.sum())
    a0 = np.zeros(mu.size)
    r0 = cell_sinkhorn(mu, nu, rho, C, eps, np.inf, a0, err=1e-10, maxit=5000)
    r1 = cell_sinkhorn(mu, nu, rho, C, eps, np.inf, a0, err=1e-10, maxit=5000, ti=True)
    assert r0.iters == r1.iters and np.array_equal(r0.alpha, r1.alpha)
