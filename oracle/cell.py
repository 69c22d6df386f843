"""Unbalanced cell subproblem solver (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The cell subproblem (Definition 3.1, Eq. cell-primal-problem) is solved by the
generalised Sinkhorn iteration of Section 5.1:
  X-half  (Eq. sinkhorn-X-iteration): closed form
          alpha = -(eps*lam/(eps+lam)) * log int exp((beta - c)/eps) dnu
  Y-half  (Eq. sinkhorn-Y-iteration, log form Eq. proxdiv-problem): per y the
          scalar root of  log(rho(y) + exp(beta/eps + z(y))) + beta/lam = 0,
          z(y) = log int_{X_J} exp((alpha - c(.,y))/eps) dmu_J,
          rho = d nu_{-J} / d nu.
  stop    (Eq. PD-gap-KL): PD/lam = KL(P_X pi | exp(-alpha/lam) mu_J)
          <= err * |mu_J|, evaluated after each Y-half.

Optional translation step (``ti=True``; not in the paper).  With lam KL
penalties and eps << lam, plain alternation contracts the total-mass mode of
the cell problem only by about 1 - eps/lam per iteration.  The cell dual
  F(alpha, beta) = -lam <e^{-alpha/lam} - 1, mu_J> - lam <e^{-beta/lam} - 1, nu>
                   - <nu_{-J}, beta> - eps <e^{(alpha + beta - c)/eps} - 1, mu_J x nu>
(the Y term is the conjugate of lam KL(. + nu_{-J} | nu) on the branch where
the cell's own Y-marginal is positive, which holds after every Y-half) keeps
its entropic term under alpha + t, beta - t.  Along that line
  G(t) = -lam A e^{-t/lam} - lam B e^{t/lam} + t a + const,
  A = <e^{-alpha/lam}, mu_J>, B = <e^{-beta/lam}, nu>, a = |nu_{-J}| on B_J,
is maximised at e^{t/lam} = (a + sqrt(a^2 + 4 A B)) / (2 B) (the quadratic
B u^2 - a u - A = 0).  After each X-half, alpha += t* (the translation-
invariant Sinkhorn idea of Sejourne, Vialard and Peyre, 2022, written here for
the cell problem).  The fixed points are those of plain alternation (at the
optimum G'(0) = 0, so t* = 0), and F does not decrease.
"""
from __future__ import annotations

import numpy as np

from .uot import kappa, kl, lse

INF = float("inf")


def prox_residual(beta, z, rho, eps, lam):
    """Left side of Eq. proxdiv-problem."""
    with np.errstate(divide="ignore"):
        logrho = np.log(np.asarray(rho, np.float64))
    return np.logaddexp(logrho, beta / eps + z) + (0.0 if np.isinf(lam) else beta / lam)


def prox_root(z, rho, eps, lam, maxit=500):
    """Solve Eq. proxdiv-problem for beta, elementwise.

    f(beta) = log(rho + e^{beta/eps + z}) + beta/lam is convex and strictly
    increasing (f' = sigma/eps + 1/lam with sigma in (0,1]), so the root is
    unique.  Newton starts at the rho = 0 closed form beta0 = -kappa*z, where
    f(beta0) >= 0 because log(rho + e^u) >= u; from the right of the root of a
    convex increasing function Newton decreases monotonically to the root.
    (The paper states only that Newton is used; start, tolerance and cap are
    this implementation's reading.)"""
    z = np.asarray(z, np.float64)
    rho = np.broadcast_to(np.asarray(rho, np.float64), z.shape)
    if np.isinf(lam):
        # balanced limit: rho + e^{beta/eps+z} = 1 (requires rho < 1)
        return eps * (np.log1p(-rho) - z)
    logrho = np.log(np.where(rho > 0, rho, 1.0))
    logrho = np.where(rho > 0, logrho, -INF)
    beta = -kappa(eps, lam) * z
    active = rho > 0
    for _ in range(maxit):
        if not np.any(active):
            break
        u = beta / eps + z
        la = np.logaddexp(logrho, u)
        f = la + beta / lam
        sig = np.exp(u - la)
        fp = sig / eps + 1.0 / lam
        step = f / fp
        new = beta - step
        done = np.abs(step) <= 1e-15 * np.maximum(1.0, np.abs(beta))
        beta = np.where(active, new, beta)
        active = active & ~done
    return beta


class CellResult:
    __slots__ = ("alpha", "beta", "px", "iters", "converged", "gap")

    def __init__(self, alpha, beta, px, iters, converged, gap):
        self.alpha, self.beta, self.px = alpha, beta, px
        self.iters, self.converged, self.gap = iters, converged, gap


def ti_shift(alpha, beta, mu_J, nu_B, rho, lam):
    """t* of the translation step (module docstring): maximiser of the cell
    dual along (alpha + t, beta - t)."""
    A = float(np.sum(mu_J * np.exp(-alpha / lam)))
    B = float(np.sum(nu_B * np.exp(-beta / lam)))
    a = float(np.sum(np.asarray(rho) * nu_B))
    u = (a + np.sqrt(a * a + 4.0 * A * B)) / (2.0 * B)
    return lam * np.log(u)


def cell_sinkhorn(mu_J, nu_B, rho, C, eps, lam, alpha0, err=2e-5, maxit=2000, ti=False):
    """Cell Sinkhorn on X_J x B_J (Section 5.1, 'Solving cell subproblems').

    mu_J (n_x), nu_B (n_y) positive; rho = nu_{-J}/nu on B_J (n_y, >= 0);
    C (n_x, n_y) the cost; alpha0 the warm start on X_J.  Each iteration is a
    Y-half from the current alpha, the X-marginal of the resulting plan, the
    stopping test (Eq. PD-gap-KL with per-cell tolerance err*|mu_J|) and, if
    not stopped, the X-half (followed by the translation step if ``ti``).
    The solve therefore ends after a Y-half."""
    mu_J = np.asarray(mu_J, np.float64)
    nu_B = np.asarray(nu_B, np.float64)
    logmu = np.log(mu_J)
    lognu = np.log(nu_B)
    kap = kappa(eps, lam)
    alpha = np.array(alpha0, np.float64)
    tol = err * mu_J.sum()
    it = 0
    while True:
        it += 1
        z = lse((alpha[:, None] - C) / eps + logmu[:, None], 0)
        beta = prox_root(z, rho, eps, lam)
        w = lse((beta[None, :] - C) / eps + lognu[None, :], 1)
        px = mu_J * np.exp(alpha / eps + w)
        ref = mu_J if np.isinf(lam) else np.exp(-alpha / lam) * mu_J
        gap = kl(px, ref)
        if gap <= tol:
            return CellResult(alpha, beta, px, it, True, gap)
        if it >= maxit:
            return CellResult(alpha, beta, px, it, False, gap)
        alpha = -kap * w
        if ti and not np.isinf(lam):
            alpha = alpha + ti_shift(alpha, beta, mu_J, nu_B, rho, lam)
