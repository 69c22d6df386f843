"""GPU adjoint (gradients of the UOT value) against the FP64 oracle and
against central finite differences of the GPU solver's own scores.

* Parity: at fixed potentials (alpha, beta) the adjoint must reproduce
  oracle.grad.dual_gradients element by element (FP64: 1e-11 of the largest
  entry; FP32 exponentials and sums: 1e-4 -- each summed term carries a
  relative error of a few 1e-6 from the float exponential of an exponent
  formed in double, the conditional means a few 1e-6 of the window width).
* Full size (512 x 512, eps = (2/512)^2, lam = 1, masses 1.0 / 1.1): sampled
  points against the oracle formula evaluated one by one in FP64 at the GPU's
  potentials, and directional central differences (h = 1e-4) of the GPU score
  along smooth perturbations of mu and nu, with the bound implied by the
  solves' primal-dual gaps.
"""
import numpy as np
import pytest

from oracle import grad as ograd
from oracle import uot
from paper_2410_08859_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_08859_gb300 import domdec
    return domdec


def potentials(mu, nu, N, eps, lam, iters, noise, seed):
    """Realistically shaped potentials: a few oracle Sinkhorn iterations, plus
    optional noise (the adjoint is exact at any fixed potentials)."""
    pix = uot.grid_index(N)
    C = uot.sq_cost(pix, pix, 1.0 / N)
    a, b, _, _ = uot.full_sinkhorn(mu, nu, C, eps, lam, err=-1.0, maxit=iters)
    rng = np.random.default_rng(seed)
    if noise:
        a = a + noise * eps * rng.standard_normal(a.shape)
        b = b + noise * eps * rng.standard_normal(b.shape)
    return a, b, pix / N


def rel_inf(x, ref):
    return np.abs(x - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("N,eps_num,noise", [(32, 1.0, 0.0), (37, 2.0, 0.5), (64, 2.0, 0.0)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_matches_oracle(dd, N, eps_num, noise, prec):
    mu, nu = inputs.mixture_small(N=N, seed=1100 + N)
    mu, nu = mu.ravel(), nu.ravel()
    eps, lam = (eps_num / N) ** 2, 1.0
    a, b, X = potentials(mu, nu, N, eps, lam, 40 if N <= 37 else 15, noise, N)
    gm_o, gn_o, gx_o = ograd.dual_gradients(a, b, X, X, mu, nu, eps, lam)
    gm, gn, gx = np.empty(N * N), np.empty(N * N), np.empty(2 * N * N)
    p = dd.FP64 if prec == "fp64" else dd.FP32
    out = dd.domdec_uot_gradients(mu, nu, a, b, N, eps, lam, p, gm, gn, gx)
    tol = 1e-11 if prec == "fp64" else 1e-4
    assert rel_inf(gm, gm_o) <= tol
    assert rel_inf(gn, gn_o) <= tol
    assert rel_inf(gx.reshape(-1, 2), gx_o) <= tol
    # the value D(alpha, beta) and the masses
    pi = uot.plan(a, b, uot.sq_cost(uot.grid_index(N), uot.grid_index(N), 1.0 / N), mu, nu, eps)
    D = uot.dual_score(a, b, uot.sq_cost(uot.grid_index(N), uot.grid_index(N), 1.0 / N), mu, nu, eps, lam)
    assert abs(out[0] - D) <= (1e-11 if prec == "fp64" else 1e-6) * abs(D) + 1e-14
    assert abs(out[1] - mu.sum()) <= 1e-13 and abs(out[2] - nu.sum()) <= 1e-13
    assert abs(out[3] - pi.sum()) <= tol * pi.sum() and abs(out[4] - pi.sum()) <= tol * pi.sum()


def test_adjoint_balanced_limit(dd):
    """lam = +inf: the penalty terms become alpha and beta (Eq. dual-problem
    with D_i the indicator of equality)."""
    N = 24
    mu, nu = inputs.mixture_small(N=N, seed=1300)
    mu, nu = mu.ravel(), nu.ravel()
    eps = (1.0 / N) ** 2
    a, b, X = potentials(mu, nu, N, eps, 1.0, 20, 0.0, 0)
    gm_o, gn_o, gx_o = ograd.dual_gradients(a, b, X, X, mu, nu, eps, 1.0)
    gm_o = gm_o + (np.exp(-a) - 1.0) + a       # replace lam (e^{-alpha/lam} - 1), lam = 1, by -alpha
    gn_o = gn_o + (np.exp(-b) - 1.0) + b
    gm, gn, gx = np.empty(N * N), np.empty(N * N), np.empty(2 * N * N)
    dd.domdec_uot_gradients(mu, nu, a, b, N, eps, float("inf"), dd.FP64, gm, gn, gx)
    assert rel_inf(gm, gm_o) <= 1e-11 and rel_inf(gn, gn_o) <= 1e-11
    assert rel_inf(gx.reshape(-1, 2), gx_o) <= 1e-11


def test_adjoint_rejects_bad_input(dd):
    N = 8
    mu = np.full(N * N, 1.0 / 64)
    nu = mu.copy()
    nu[5] = 0.0
    z = np.zeros(N * N)
    with pytest.raises(dd.DomDecError) as e:
        dd.domdec_uot_gradients(mu, nu, z, z, N, 0.01, 1.0, dd.FP64, np.empty(N * N))
    assert e.value.code == dd.DOMDEC_EINVAL
    with pytest.raises(dd.DomDecError):
        dd.domdec_uot_gradients(mu, mu, z, z, N, 0.01, 1.0, 7, np.empty(N * N))


def smooth_field(N, kx, ky, phase):
    t = np.arange(N) / N
    I, J = np.meshgrid(t, t, indexing="ij")
    return (np.cos(2 * np.pi * kx * I + phase) * np.sin(2 * np.pi * ky * J + 0.3)).ravel()


def solve_gpu(torch, mu_d, nu_d, eps, lam, s, precision, gap, alpha0=None, beta0=None, max_sweeps=200):
    from paper_2410_08859_gb300 import autograd as ag
    g, info = ag.solve(mu_d, nu_d, eps, lam, s=s, gap=gap, precision=precision, max_sweeps=max_sweeps,
                       alpha0=alpha0, beta0=beta0, eps0=eps if alpha0 is not None else None)
    return g, info


def fd_directional(dd, torch, mu, nu, eps, lam, s, precision, gap, base, which, phi, h):
    """(S(w (1 + h phi)) - S(w (1 - h phi))) / (2 h) and its error bound from the gaps."""
    a0, b0 = base
    vals, bound = [], 0.0
    for sgn in (1.0, -1.0):
        m = mu * (1 + sgn * h * phi) if which == "mu" else mu
        n_ = nu * (1 + sgn * h * phi) if which == "nu" else nu
        md = torch.tensor(m, dtype=torch.float64, device="cuda")
        nd = torch.tensor(n_, dtype=torch.float64, device="cuda")
        g, info = solve_gpu(torch, md, nd, eps, lam, s, precision, gap, a0, b0)
        cert = g.pd_gap()
        g.close()
        vals.append(cert[0])
        bound += abs(cert[0] - cert[1])
    return (vals[0] - vals[1]) / (2 * h), bound / (2 * h)


def test_gradients_directional_fd_fp64(dd):
    """64 x 64, FP64 cells: directional central differences of the GPU score
    match <grad, w phi> within the certificate's bound."""
    import torch
    N, s = 64, 4
    mu, nu = inputs.mixture_blobs(N=N, seed=5100, mass_ratio=1.1)
    mu, nu = mu.ravel(), nu.ravel()
    eps, lam = (2.0 / N) ** 2, 1.0
    md = torch.tensor(mu, dtype=torch.float64, device="cuda")
    nd = torch.tensor(nu, dtype=torch.float64, device="cuda")
    g, info = solve_gpu(torch, md, nd, eps, lam, s, "fp64", 1e-10)
    a = g.duals()
    gm, gn, gx, out = g.gradients(dd.FP64, beta=(b := np.empty(N * N)))
    g.close()
    for which, grad, w in (("mu", gm, mu), ("nu", gn, nu)):
        phi = smooth_field(N, 1, 2, 0.4 if which == "mu" else 1.1)
        pred = float(np.dot(grad, w * phi))
        fd, bnd = fd_directional(dd, torch, mu, nu, eps, lam, s, "fp64", 1e-10, (a, b), which, phi, 1e-4)
        assert abs(fd - pred) <= bnd + 1e-4 * abs(pred), (which, fd, pred, bnd)


def oracle_rows(alpha, beta, mu, nu, N, eps, lam, xs):
    """Oracle gradients at the sampled source points xs (one row of the plan each)."""
    pix = uot.grid_index(N) / N
    gm = np.empty(len(xs))
    gx = np.empty((len(xs), 2))
    for r, x in enumerate(xs):
        m, _, g = ograd.dual_gradients(alpha[x:x + 1], beta, pix[x:x + 1], pix, mu[x:x + 1], nu, eps, lam)
        gm[r] = m[0]
        gx[r] = g[0]
    return gm, gx


def oracle_cols(alpha, beta, mu, nu, N, eps, lam, ys):
    """Oracle d/dnu at the sampled target points ys (roles of the sides swapped)."""
    pix = uot.grid_index(N) / N
    gn = np.empty(len(ys))
    for r, y in enumerate(ys):
        m, _, _ = ograd.dual_gradients(beta[y:y + 1], alpha, pix[y:y + 1], pix, nu[y:y + 1], mu, eps, lam)
        gn[r] = m[0]
    return gn


def test_gradients_full_size_512(dd):
    """512 x 512, eps = (2/512)^2, lam = 1, masses 1.0 / 1.1, FP32 cells: the
    adjoint at the solver's potentials against the oracle on 48 sampled points,
    the FP32 adjoint against the FP64 one, and directional central differences."""
    import torch
    N, s = 512, 8
    mu, nu = inputs.mixture_blobs(N=N, seed=5000, mass_ratio=1.1)
    mu, nu = mu.ravel(), nu.ravel()
    eps, lam = (2.0 / N) ** 2, 1.0
    md = torch.tensor(mu, dtype=torch.float64, device="cuda")
    nd = torch.tensor(nu, dtype=torch.float64, device="cuda")
    g, info = solve_gpu(torch, md, nd, eps, lam, s, "fp32", 1e-6)
    a = g.duals()
    b = np.empty(N * N)
    gm, gn, gx, out = g.gradients(dd.FP64, beta=b)
    gm32, gn32, gx32, out32 = g.gradients(dd.FP32)
    g.close()
    rng = np.random.default_rng(7)
    xs = rng.choice(N * N, 48, replace=False)
    om, ox = oracle_rows(a, b, mu, nu, N, eps, lam, xs)
    on = oracle_cols(a, b, mu, nu, N, eps, lam, xs)
    scale_m, scale_n, scale_x = np.abs(gm).max(), np.abs(gn).max(), np.abs(gx).max()
    assert np.abs(gm[xs] - om).max() <= 1e-10 * scale_m
    assert np.abs(gn[xs] - on).max() <= 1e-10 * scale_n
    assert np.abs(gx.reshape(-1, 2)[xs] - ox).max() <= 1e-10 * scale_x
    # FP32 exponentials/sums against FP64 (the stated FP32-vs-FP64 error)
    assert np.abs(gm32 - gm).max() <= 1e-4 * scale_m
    assert np.abs(gn32 - gn).max() <= 1e-4 * scale_n
    assert np.abs(gx32 - gx).max() <= 1e-4 * scale_x
    for which, grad, w in (("mu", gm, mu), ("nu", gn, nu)):
        phi = smooth_field(N, 2, 1, 0.2 if which == "mu" else 0.9)
        pred = float(np.dot(grad, w * phi))
        fd, bnd = fd_directional(dd, torch, mu, nu, eps, lam, s, "fp32", 1e-7, (a, b), which, phi, 1e-4)
        assert abs(fd - pred) <= bnd + 1e-3 * abs(pred), (which, fd, pred, bnd)


def test_autograd_function(dd):
    """uot_score: backward returns the adjoint's gradients in the inputs'
    dtype; positions off the grid are rejected."""
    import torch
    from paper_2410_08859_gb300 import autograd as ag
    N = 32
    mu, nu = inputs.mixture_small(N=N, seed=1400)
    mu_t = torch.tensor(mu.ravel(), dtype=torch.float32, device="cuda", requires_grad=True)
    nu_t = torch.tensor(nu.ravel(), dtype=torch.float32, device="cuda", requires_grad=True)
    x = ag.grid_positions(N, "cuda", torch.float32).requires_grad_(True)
    eps, lam = (1.0 / N) ** 2, 1.0
    S = ag.uot_score(mu_t, nu_t, eps, lam, x=x, s=4, gap=1e-7, precision="fp64")
    (3.0 * S).backward()
    assert mu_t.grad.dtype == torch.float32 and x.grad.shape == (N * N, 2)
    md = mu_t.detach().double().contiguous()
    nd = nu_t.detach().double().contiguous()
    g, _ = ag.solve(md, nd, eps, lam, s=4, gap=1e-7, precision="fp64")
    gm, gn, gx, out = g.gradients(dd.FP64)
    sc = g.score()[0]
    g.close()
    assert abs(S.item() - sc) <= 1e-6 * abs(sc)
    assert np.allclose(mu_t.grad.cpu().numpy(), 3.0 * gm, rtol=1e-5, atol=1e-7)
    assert np.allclose(nu_t.grad.cpu().numpy(), 3.0 * gn, rtol=1e-5, atol=1e-7)
    assert np.allclose(x.grad.cpu().numpy(), 3.0 * gx.reshape(-1, 2), rtol=1e-5, atol=1e-7)
    with pytest.raises(ValueError):
        ag.uot_score(mu_t, nu_t, eps, lam, x=x.detach() + 0.5 / N, s=4)
