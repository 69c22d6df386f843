"""Pins of the balancing step (Section 5.3, 'Balancing', Eq. balancing) in the
oracle: the basic-cell masses reach the targets m_i, nu_J is preserved at
every y, the targets reduce to mu(X_i) |nu_J| / mu(X_J) in the balanced limit
(the balanced scheme the paper cites), the bookkeeping (C_i, H_i, P_X) is that
of the explicitly balanced plan, and DomDec with balancing still converges to
the global optimum."""
import numpy as np
import pytest

from oracle import domdec as odd
from oracle import uot
from paper_2410_08859_gb300 import inputs


def one_cell(seed, lam, N=16, s=2, sweeps_before=1, which=None):
    mu, nu = inputs.mixture_small(N=N, seed=seed)
    geo = odd.Geometry(N, s)
    st = odd.init_product(geo, mu.ravel(), nu.ravel(), (1.0 / N) ** 2, lam)
    if sweeps_before:
        odd.run(st, sweeps_before, strategy="safe")
    which = which or "AB"[sweeps_before % 2]
    cells = [c for c in st.geo.parts[which] if len(c["members"]) == 4]
    cell = cells[len(cells) // 2]
    prob = odd.cell_problem(st, cell)
    return st, cell, prob


@pytest.mark.parametrize("seed,lam", [(1300, 1.0), (1301, 5.0), (1302, 0.5)])
def test_targets_reached_and_nu_J_preserved(seed, lam):
    st, cell, prob = one_cell(seed, lam)
    plain = odd.solve_cell(st, cell, prob, err=1e-10, maxit=5000)
    bal = odd.solve_cell(st, cell, prob, err=1e-10, maxit=5000, balance=True)
    mem = cell["members"]
    nuJ0 = sum(plain["nut"][i] for i in mem)
    nuJ1 = sum(bal["nut"][i] for i in mem)
    assert np.allclose(nuJ1, nuJ0, rtol=1e-12, atol=1e-300)
    # targets from one more X-half of the final beta
    g = st.geo
    X, Y = cell["X"], prob["Y"]
    C = uot.sq_cost(g.pix[X], g.pix[Y], g.h)
    a2 = uot.x_half(plain["beta"], C, st.nu[Y], st.eps, lam)
    mubar = st.mu[X] * np.exp(-a2 / lam)
    bop = g.basic_of_pixel[X]
    mJ = float(nuJ0.sum())
    for i in mem:
        m_i = mubar[bop == i].sum() * mJ / mubar.sum()
        assert abs(bal["nut"][i].sum() - m_i) <= 1e-12 * mJ
    assert all((bal["nut"][i] >= 0).all() for i in mem)
    assert (bal["pi"] >= 0).all()
    # the bookkeeping is that of the balanced plan itself
    pi = bal["pi"]
    assert np.allclose(bal["px"], pi.sum(1), rtol=1e-13, atol=0)
    for i in mem:
        r = bop == i
        assert abs(bal["Ct"][i] - float(np.sum(C[r] * pi[r]))) <= 1e-13 * abs(bal["Ct"][i])
        ref = pi[r] / (st.mu[X][r][:, None] * st.nu[Y][None, :])
        Hi = float(np.sum(np.where(pi[r] > 0, pi[r] * np.log(np.where(ref > 0, ref, 1.0)), 0.0)
                          - pi[r])) + st.mu[X][r].sum() * st.nu.sum()
        assert abs(bal["Ht"][i] - Hi) <= 1e-11 * max(abs(Hi), 1e-12)


def test_balanced_limit_targets():
    """lam = inf: mu_bar = mu, so m_i = mu(X_i) |nu_J| / mu(X_J)."""
    N, s = 16, 2
    mu, nu = inputs.mixture_small(N=N, seed=1303, masses=(1.0, 1.0))
    geo = odd.Geometry(N, s)
    st = odd.init_product(geo, mu.ravel(), nu.ravel(), (1.0 / N) ** 2, np.inf)
    odd.run(st, 1, strategy="safe")
    cell = [c for c in st.geo.parts["B"] if len(c["members"]) == 4][3]
    prob = odd.cell_problem(st, cell)
    bal = odd.solve_cell(st, cell, prob, err=1e-10, maxit=5000, balance=True)
    bop = geo.basic_of_pixel[cell["X"]]
    mJ = sum(bal["nut"][i].sum() for i in cell["members"])
    muX = st.mu[cell["X"]]
    for i in cell["members"]:
        assert abs(bal["nut"][i].sum() - muX[bop == i].sum() * mJ / muX.sum()) <= 1e-12 * mJ


def test_balanced_run_converges_to_optimum():
    N, s = 16, 2
    mu, nu = inputs.mixture_small(N=N, seed=1304)
    mu, nu = mu.ravel(), nu.ravel()
    geo = odd.Geometry(N, s)
    eps, lam = (1.0 / N) ** 2, 5.0
    st = odd.init_product(geo, mu, nu, eps, lam)
    odd.run(st, 24, strategy="staggered", err=1e-10, maxit=5000, balance=True)
    C = odd.full_cost(geo)
    a, b, _, _ = uot.full_sinkhorn(mu, nu, C, eps, lam, err=1e-13, maxit=200000)
    Eopt = uot.primal_score(uot.plan(a, b, C, mu, nu, eps), C, mu, nu, eps, lam)
    E = odd.tracked_score(st)
    assert Eopt - 1e-12 * abs(Eopt) <= E <= Eopt + 1e-5 * abs(Eopt)
