"""Differentiable unbalanced OT score on the N x N grid (torch.autograd).

``uot_score(mu, nu, eps, lam, x=None)`` solves the entropic UOT problem of
Eq. unbalanced-problem (squared-Euclidean cost on the grid {0..N-1}^2 / N,
lam KL penalties) with the domain-decomposition solver and returns its score
as a 0-d tensor; ``backward`` gives d(score)/d mu, d(score)/d nu and, when the
source positions ``x`` take part, d(score)/d x.  The gradients come from the
adjoint kernels of the library (``domdec_gradients``: envelope theorem at the
final potentials, barycentric projection over the implicit plan); PyTorch only
carries device memory, the stream and the chain rule's scalar factor.

The solve: global separable Sinkhorn from ``eps_start`` down to 2 eps (float
while eps is coarse, double below, Section 5.3's warm start), then DomDec
sweeps in A/B pairs until the certificate's relative primal-dual gap is at most
``gap`` or ``max_sweeps`` is reached.
"""
from __future__ import annotations

import torch

from . import domdec as dd

__all__ = ["solve", "uot_score", "UOTScore", "grid_positions"]


def grid_positions(N, device=None, dtype=torch.float64):
    """Source positions of the grid, (N*N, 2), row-major: x = (i, j) / N."""
    t = torch.arange(N, device=device, dtype=dtype) / N
    return torch.stack(torch.meshgrid(t, t, indexing="ij"), -1).reshape(N * N, 2)


def solve(mu, nu, eps, lam, s=8, gap=1e-6, max_sweeps=200, precision="fp32", cell_err=1e-7, cell_maxit=1000,
          eps_start=1.0, warm_err=5e-6, warm_maxit=4000, alpha0=None, beta0=None, eps0=None, stream=None):
    """DomDec solve to a relative PD gap.  mu, nu: contiguous float64 CUDA
    tensors with N*N entries.  alpha0/beta0 (with their eps0) replace the
    global Sinkhorn warm start.  Returns (DomDec handle, info dict); the
    caller closes the handle."""
    n = mu.numel()
    N = int(round(n ** 0.5))
    if alpha0 is None:
        alpha0 = torch.empty(n, dtype=torch.float64, device=mu.device)
        beta0 = torch.empty_like(alpha0)
        dd.domdec_full_sinkhorn(mu, nu, N, 2 * eps, lam, eps_start=eps_start, variant=dd.SINKHORN_SEPARABLE,
                                precision=dd.MIXED, maxit=warm_maxit, err=warm_err, check_every=10,
                                alpha=alpha0, beta=beta0, stream=stream)
        eps0 = 2 * eps
    g = dd.DomDec(mu, nu, eps, lam, s, alpha0=alpha0, beta0=beta0, eps_init=eps if eps0 is None else eps0,
                  precision=precision, tau=0.0, err=cell_err, maxit=cell_maxit, cell_ctas=2, stream=stream)
    sweeps, rel = 0, float("inf")
    try:
        while sweeps < max_sweeps:
            g.iterate(2)
            sweeps += 2
            rel = g.pd_gap()[2]
            if rel <= gap:
                break
    except Exception:
        g.close()
        raise
    return g, {"sweeps": sweeps, "rel_gap": rel}


class UOTScore(torch.autograd.Function):
    """score = E_hat of the DomDec solution (Eq. tracked score); gradients by
    the library's adjoint (FP64 or FP32 summation, ``grad_precision``)."""

    @staticmethod
    def forward(ctx, mu, nu, x, eps, lam, opts):
        opts = dict(opts or {})
        grad_precision = opts.pop("grad_precision", dd.FP64)
        n = mu.numel()
        N = int(round(n ** 0.5))
        if N * N != n or nu.numel() != n:
            raise ValueError("mu and nu must hold N*N weights of the same grid")
        if not mu.is_cuda:
            raise ValueError("uot_score runs on CUDA tensors only")
        if x is not None:
            if tuple(x.shape) != (n, 2):
                raise ValueError("x must be the (N*N, 2) source positions")
            if not torch.allclose(x.detach().to(torch.float64), grid_positions(N, x.device), atol=1e-12, rtol=0):
                raise ValueError("x must be the grid positions (i, j)/N: the solver works on the grid")
        mu64 = mu.detach().to(torch.float64).contiguous().view(-1)
        nu64 = nu.detach().to(torch.float64).contiguous().view(-1)
        g, info = solve(mu64, nu64, eps, lam, **opts)
        try:
            score = g.score()[0]
            gm = torch.empty(n, dtype=torch.float64, device=mu.device)
            gn = torch.empty_like(gm)
            gx = torch.empty(2 * n, dtype=torch.float64, device=mu.device)
            g.gradients(grad_precision, gm, gn, gx)
        finally:
            g.close()
        ctx.info = info
        ctx.save_for_backward(gm.view_as(mu).to(mu.dtype), gn.view_as(nu).to(nu.dtype),
                              gx.view(n, 2).to(x.dtype if x is not None else mu.dtype))
        ctx.has_x = x is not None
        return torch.tensor(score, dtype=mu.dtype, device=mu.device)

    @staticmethod
    def backward(ctx, grad_out):
        gm, gn, gx = ctx.saved_tensors
        return (grad_out * gm, grad_out * gn, grad_out * gx if ctx.has_x else None, None, None, None)


def uot_score(mu, nu, eps, lam, x=None, **opts):
    """Differentiable UOT score (see the module docstring); opts go to
    ``solve`` (s, gap, max_sweeps, precision, ...) plus ``grad_precision``."""
    return UOTScore.apply(mu, nu, x, eps, lam, opts)
