"""Brute-force convex maximisation of the UOT dual on tiny problems.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

D(alpha, beta | nu_-) (Eq. dual-problem / Eq. cell-dual-problem with
D_i = lam KL) is smooth and strictly concave for finite lam on finite spaces
with full-support marginals (Lemma 4.2).  It is maximised here by a damped
Newton method with exact gradient and Hessian, independently of any Sinkhorn
iteration:
  dD/dalpha(x) = -P_X pi(x) + mu(x) e^{-alpha(x)/lam}
  dD/dbeta(y)  = -P_Y pi(y) + nu(y) e^{-beta(y)/lam} - nu_-(y)
with pi = exp((alpha (+) beta - c)/eps) mu x nu.
"""
from __future__ import annotations

import numpy as np

from .uot import dual_score


def dual_newton(mu, nu, C, eps, lam, nu_minus=None, tol=1e-13, maxit=500):
    mu = np.asarray(mu, np.float64)
    nu = np.asarray(nu, np.float64)
    n, m = len(mu), len(nu)
    num = np.zeros(m) if nu_minus is None else np.asarray(nu_minus, np.float64)
    a = np.zeros(n)
    b = np.zeros(m)

    def value(a, b):
        return dual_score(a, b, C, mu, nu, eps, lam, num)

    val = value(a, b)
    for _ in range(maxit):
        pi = np.exp((a[:, None] + b[None, :] - C) / eps) * mu[:, None] * nu[None, :]
        px, py = pi.sum(1), pi.sum(0)
        ea = mu * np.exp(-a / lam)
        eb = nu * np.exp(-b / lam)
        g = np.concatenate([-px + ea, -py + eb - num])
        if np.max(np.abs(g)) < tol:
            break
        H = np.zeros((n + m, n + m))
        H[:n, :n] = -np.diag(px / eps + ea / lam)
        H[n:, n:] = -np.diag(py / eps + eb / lam)
        H[:n, n:] = -pi / eps
        H[n:, :n] = -pi.T / eps
        step = np.linalg.solve(-H, g)
        t = 1.0
        while t > 1e-12:
            na, nb = a + t * step[:n], b + t * step[n:]
            nv = value(na, nb)
            if nv >= val + 1e-4 * t * float(g @ step) or nv >= val:
                break
            t *= 0.5
        a, b, val = na, nb, nv
    return a, b
