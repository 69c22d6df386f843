"""Gradients of the unbalanced OT value (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The value S(mu, nu, X) = min_pi E(pi) = max_{alpha,beta} D(alpha, beta)
(Eq. unbalanced-problem / dual-problem, nu_- = 0, D_i = lam KL).  The paper
does not differentiate S; the formulas below follow from the envelope theorem
applied to the dual at fixed potentials (alpha, beta):

  dD/dmu(x) = eps |nu| - eps sum_y nu(y) e^{(alpha(x)+beta(y)-c(x,y))/eps}
              - lam (e^{-alpha(x)/lam} - 1)
  dD/dnu(y) = eps |mu| - eps sum_x mu(x) e^{(alpha(x)+beta(y)-c(x,y))/eps}
              - lam (e^{-beta(y)/lam} - 1)
  dD/dx     = sum_y pi(x,y) dc/dx = 2 P_X pi(x) (x - T(x)),
              T(x) = sum_y pi(x,y) y / P_X pi(x)   (barycentric projection)

with pi = exp((alpha + beta - c)/eps) mu x nu.  At the optimal potentials they
are the derivatives of S.  Pinned by central finite differences of S computed
with ``uot.full_sinkhorn`` to high precision.
"""
from __future__ import annotations

import numpy as np

from . import uot


def dual_gradients(alpha, beta, X, Y, mu, nu, eps, lam):
    """(grad_mu, grad_nu, grad_x) of D(alpha, beta) at fixed potentials.
    X (n, d), Y (m, d) are point coordinates; c = |x - y|^2."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    C = np.sum((X[:, None, :] - Y[None, :, :]) ** 2, axis=-1)
    pi = uot.plan(alpha, beta, C, mu, nu, eps)
    px = pi.sum(1)
    py = pi.sum(0)
    g_mu = eps * nu.sum() - eps * px / mu - lam * (np.exp(-alpha / lam) - 1.0)
    g_nu = eps * mu.sum() - eps * py / nu - lam * (np.exp(-beta / lam) - 1.0)
    T = (pi @ Y) / px[:, None]
    g_x = 2.0 * px[:, None] * (X - T)
    return g_mu, g_nu, g_x


def value(mu, nu, X, Y, eps, lam, err=1e-14, maxit=200000):
    """S(mu, nu, X) by global Sinkhorn; returns (S, alpha, beta)."""
    C = np.sum((np.asarray(X)[:, None, :] - np.asarray(Y)[None, :, :]) ** 2, axis=-1)
    a, b, it, gap = uot.full_sinkhorn(mu, nu, C, eps, lam, err=err, maxit=maxit)
    return uot.dual_score(a, b, C, mu, nu, eps, lam), a, b
