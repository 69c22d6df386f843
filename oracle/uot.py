"""Global entropic unbalanced OT with KL marginal penalties (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Notation follows the paper: marginals mu on X and nu on Y, cost c(x,y) =
|x-y|^2, entropic strength eps, KL marginal penalty strength lam
(D_1 = D_2 = lam*KL, Section 5.1), background measure nu_minus (Definition
2.2).  lam = inf denotes the balanced limit.
"""
from __future__ import annotations

import numpy as np

INF = float("inf")


# ---------------------------------------------------------------- divergences
def phi_kl(s):
    """Entropy function of KL: phi(s) = s log s - s + 1, phi(0) = 1
    (Example after Definition 2.1)."""
    s = np.asarray(s, dtype=np.float64)
    out = np.ones_like(s)
    pos = s > 0
    sp = s[pos]
    out[pos] = sp * np.log(sp) - sp + 1.0
    return out


def kl(a, b):
    """KL(a|b) = sum_z b(z) phi(a(z)/b(z)) for b > 0 (Eq. KL)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sum(b * phi_kl(a / b)))


def lse(M, axis):
    """log(sum(exp(M))) along ``axis`` with the maximum subtracted."""
    m = np.max(M, axis=axis, keepdims=True)
    m_safe = np.where(np.isfinite(m), m, 0.0)
    out = np.log(np.sum(np.exp(M - m_safe), axis=axis)) + np.squeeze(m_safe, axis)
    return out


# ------------------------------------------------------------------- geometry
def grid_index(N, d=2):
    """Integer pixel coordinates of the uniform grid {0..N-1}^d, row-major."""
    idx = np.indices((N,) * d).reshape(d, -1).T
    return idx.astype(np.int64)


def sq_cost(ix, iy, h):
    """c(x,y) = |x-y|^2 for pixel index arrays ix (n,d), iy (m,d) and grid
    spacing h (Section 5.1, 'Choice of cost and divergence')."""
    diff = ix[:, None, :] - iy[None, :, :]
    return (h * h) * np.sum(diff * diff, axis=-1).astype(np.float64)


# ------------------------------------------------------------ primal and dual
def primal_score(pi, C, mu, nu, eps, lam, nu_minus=None):
    """E(pi | nu_-) = <c,pi> + eps KL(pi | mu x nu) + lam KL(P_X pi | mu)
    + lam KL(P_Y pi + nu_- | nu)  (Eq. unbalanced-problem, D_i = lam KL)."""
    mu = np.asarray(mu, np.float64)
    nu = np.asarray(nu, np.float64)
    pi = np.asarray(pi, np.float64)
    prod = mu[:, None] * nu[None, :]
    e = float(np.sum(C * pi)) + eps * kl(pi, prod)
    px = pi.sum(1)
    py = pi.sum(0) + (0.0 if nu_minus is None else nu_minus)
    if np.isinf(lam):
        raise ValueError("primal score with lam = inf is an indicator; not used")
    return e + lam * kl(px, mu) + lam * kl(py, nu)


def conj_term(pot, m, lam):
    """int phi*(-pot) dm for D = lam KL: (lam phi)^*(z) = lam (exp(z/lam) - 1)
    evaluated at z = -pot; for lam = inf it is the linear term -<pot, m>."""
    if np.isinf(lam):
        return -float(np.sum(pot * m))
    return float(np.sum(lam * (np.exp(-pot / lam) - 1.0) * m))


def dual_score(alpha, beta, C, mu, nu, eps, lam, nu_minus=None):
    """D(alpha, beta | nu_-) of Eq. dual-problem with D_i = lam KL."""
    mu = np.asarray(mu, np.float64)
    nu = np.asarray(nu, np.float64)
    expo = (alpha[:, None] + beta[None, :] - C) / eps
    ent = eps * float(np.sum((1.0 - np.exp(expo)) * mu[:, None] * nu[None, :]))
    d = ent - conj_term(alpha, mu, lam) - conj_term(beta, nu, lam)
    if nu_minus is not None:
        d -= float(np.sum(beta * nu_minus))
    return d


def plan(alpha, beta, C, mu, nu, eps):
    """pi = exp((alpha (+) beta - c)/eps) mu x nu (Eq. sinkhorn-primal)."""
    return np.exp((alpha[:, None] + beta[None, :] - C) / eps) * mu[:, None] * nu[None, :]


# ------------------------------------------------------------- global Sinkhorn
def kappa(eps, lam):
    """Scaling of the closed-form KL half-step: eps / (1 + eps/lam)."""
    return eps if np.isinf(lam) else eps / (1.0 + eps / lam)


def x_half(beta, C, nu, eps, lam):
    """alpha = -kappa * log int exp((beta - c)/eps) dnu (Eq. sinkhorn-iters-ot)."""
    return -kappa(eps, lam) * lse((beta[None, :] - C) / eps + np.log(nu)[None, :], 1)


def y_half(alpha, C, mu, eps, lam):
    """beta = -kappa * log int exp((alpha - c)/eps) dmu (Eq. sinkhorn-iters-ot)."""
    return -kappa(eps, lam) * lse((alpha[:, None] - C) / eps + np.log(mu)[:, None], 0)


def x_marginal(alpha, beta, C, mu, nu, eps):
    """P_X pi for the diagonal scaling pi(alpha, beta)."""
    w = lse((beta[None, :] - C) / eps + np.log(nu)[None, :], 1)
    return mu * np.exp(alpha / eps + w)


def pd_gap_over_lam(alpha, px, mu, lam):
    """PD / lam = KL(P_X pi | exp(-alpha/lam) mu) (Eq. PD-gap-KL); for
    lam = inf this is KL(P_X pi | mu)."""
    ref = mu if np.isinf(lam) else np.exp(-alpha / lam) * mu
    return kl(px, ref)


def full_sinkhorn(mu, nu, C, eps, lam, err=2e-5, maxit=10000, beta0=None,
                  min_iters=1, ti=False):
    """Generalised Sinkhorn for the global problem (nu_- = 0), Eq.
    sinkhorn-iters-ot, starting from beta0 (default 0, Definition 2.3).

    One iteration = X-half then Y-half.  After each Y-half the stopping
    quantity PD/lam = KL(P_X pi | e^{-alpha/lam} mu) is evaluated (Eq. PD-gap-KL,
    with nu_- = 0 and a single cell); the loop stops once it is
    <= err * |mu| (Section 5.3, 'Stopping criterion') or after maxit iterations.
    ``ti``: after each X-half, alpha += (lam/2) log(<e^{-alpha/lam}, mu> /
    <e^{-beta/lam}, nu>), the maximiser of the dual along (alpha + t, beta - t)
    (the cell problem's translation step with nu_{-J} = 0; not in the paper).
    Returns (alpha, beta, iterations, last PD/lam)."""
    mu = np.asarray(mu, np.float64)
    nu = np.asarray(nu, np.float64)
    beta = np.zeros(nu.shape[0]) if beta0 is None else np.array(beta0, np.float64)
    tol = err * mu.sum()
    gap = INF
    it = 0
    while it < maxit:
        alpha = x_half(beta, C, nu, eps, lam)
        if ti and not np.isinf(lam):
            alpha = alpha + 0.5 * lam * np.log(np.sum(mu * np.exp(-alpha / lam))
                                               / np.sum(nu * np.exp(-beta / lam)))
        beta = y_half(alpha, C, mu, eps, lam)
        it += 1
        px = x_marginal(alpha, beta, C, mu, nu, eps)
        gap = pd_gap_over_lam(alpha, px, mu, lam)
        if it >= min_iters and gap <= tol:
            break
    return alpha, beta, it, gap
