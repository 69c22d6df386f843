"""Pins of the oracle's domain decomposition against the paper's structural
facts: partition geometry, the single-cell reduction to global Sinkhorn,
exactness / upper-bound property of the tracked score, monotone decrease for
safe / swift / staggered, convergence to the unique global optimum, weak
duality of the certificate, and the qualitative strategy behaviour of the
1-D toy problem (Section 4.4)."""
import numpy as np
import pytest

from oracle import domdec, uot
from paper_2410_08859_gb300 import inputs


def small_problem(N=16, seed=1001):
    mu, nu = inputs.mixture_small(N=N, seed=seed)
    return mu.ravel(), nu.ravel()


def test_partition_geometry_2d():
    geo = domdec.Geometry(16, 2)
    A, B = geo.parts["A"], geo.parts["B"]
    assert len(A) == 16 and len(B) == 25
    assert sorted(len(c["members"]) for c in B) == [1] * 4 + [2] * 12 + [4] * 9
    for part in (A, B):
        allx = np.concatenate([c["X"] for c in part])
        assert np.array_equal(np.sort(allx), np.arange(geo.n))
        for c in part:
            mem = set(geo.basic_of_pixel[c["X"]])
            assert mem == set(c["members"])
    subA = [sum(c["sub"] == b for c in A) for b in range(4)]
    subB = [sum(c["sub"] == b for c in B) for b in range(4)]
    assert subA == [4, 4, 4, 4] and subB == [9, 6, 6, 4]
    # no two composite cells of one sub-batch are adjacent (staggered)
    for part in (A, B):
        for b in range(4):
            Ps = [np.array(c["P"]) for c in part if c["sub"] == b]
            for i in range(len(Ps)):
                for j in range(i + 1, len(Ps)):
                    assert np.abs(Ps[i] - Ps[j]).max() >= 2


def test_partition_geometry_1d_toy():
    """Section 4.4: A pairs neighbouring points, B has singletons at the ends."""
    geo = domdec.Geometry(32, 1, d=1)
    A, B = geo.parts["A"], geo.parts["B"]
    assert [list(c["X"]) for c in A[:2]] == [[0, 1], [2, 3]]
    assert [list(c["X"]) for c in B[:2]] == [[0], [1, 2]]
    assert list(B[-1]["X"]) == [31]


def test_single_composite_cell_equals_global_sinkhorn():
    """One composite cell covering X: nu_{-J} = 0, so the cell solve is the
    global Sinkhorn iteration started from alpha = 0 (Section 5.1)."""
    N, s = 8, 4
    geo = domdec.Geometry(N, s)
    mu, nu = small_problem(N)
    eps, lam = (1.0 / N) ** 2, 1.0
    st = domdec.init_product(geo, mu, nu, eps, lam, thr=0.0)
    lg = domdec.sweep(st, "A", "staggered", err=1e-8)
    C = domdec.full_cost(geo)
    alpha = np.zeros(geo.n)
    it = 0
    while True:
        it += 1
        beta = uot.y_half(alpha, C, mu, eps, lam)
        px = uot.x_marginal(alpha, beta, C, mu, nu, eps)
        if uot.pd_gap_over_lam(alpha, px, mu, lam) <= 1e-8 * mu.sum():
            break
        alpha = uot.x_half(beta, C, nu, eps, lam)
    assert lg[0]["iters"] == [it]
    assert np.abs(st.alpha - alpha).max() < 1e-12
    pi = uot.plan(alpha, beta, C, mu, nu, eps)
    assert np.abs(st.PX - pi.sum(1)).max() < 1e-15
    assert np.abs(st.PY - pi.sum(0)).max() < 1e-15
    E = uot.primal_score(pi, C, mu, nu, eps, lam)
    assert abs(domdec.tracked_score(st) - E) < 1e-13 * abs(E)


def test_tracked_score_exact_after_greedy_and_upper_bound_after_mixing():
    """R3: after greedy steps the tracked score is the exact score
    (Eq. domdec-score-decomp-unbalanced); after convex mixing it is an upper
    bound (convexity of the entropy)."""
    geo = domdec.Geometry(8, 2)
    mu, nu = small_problem(8, seed=1003)
    eps, lam = (1.0 / 8) ** 2, 0.5
    st = domdec.init_product(geo, mu, nu, eps, lam, thr=0.0, track_plan=True)
    assert abs(domdec.tracked_score(st) - domdec.exact_score(st)) < 1e-13
    for k in range(3):
        domdec.sweep(st, "AB"[k % 2], "greedy", err=1e-6)
        Ee = domdec.exact_score(st)
        assert abs(domdec.tracked_score(st) - Ee) < 1e-12 * abs(Ee)
    for k in range(4):
        domdec.sweep(st, "AB"[k % 2], "safe", err=1e-6)
        assert domdec.tracked_score(st) >= domdec.exact_score(st) - 1e-13


def test_init_from_duals_matches_dense_plan():
    geo = domdec.Geometry(8, 2)
    mu, nu = small_problem(8, seed=1004)
    C = domdec.full_cost(geo)
    eps0, eps, lam = 0.05, 0.02, 2.0
    a, b, _, _ = uot.full_sinkhorn(mu, nu, C, eps0, lam, err=1e-6)
    st = domdec.init_from_duals(geo, mu, nu, a, b, eps0, eps, lam, thr=0.0, track_plan=True)
    pi = uot.plan(a, b, C, mu, nu, eps0)
    assert np.abs(st.PX - pi.sum(1)).max() < 1e-16
    assert np.abs(st.PY - pi.sum(0)).max() < 1e-15
    Ee = uot.primal_score(pi, C, mu, nu, eps, lam)
    assert abs(domdec.tracked_score(st) - Ee) < 1e-12 * abs(Ee)


@pytest.mark.parametrize("strategy", ["safe", "swift", "staggered"])
def test_tracked_score_monotone(strategy):
    """Proposition 4.3: safe, swift (and swift on sub-batches) never increase
    the score (here the tracked score, R3, with tau = 0)."""
    geo = domdec.Geometry(16, 2)
    mu, nu = small_problem(16, seed=1005)
    st = domdec.init_product(geo, mu, nu, (1.0 / 16) ** 2, 1.0)
    prev = domdec.tracked_score(st)
    for k in range(4):
        for rec in domdec.sweep(st, "AB"[k % 2], strategy, tau=0.0, err=1e-6):
            assert rec["E0"] <= prev * (1 + 1e-14)
            prev = rec["E0"]
        E = domdec.tracked_score(st)
        assert E <= prev * (1 + 1e-14)
        prev = E


@pytest.mark.parametrize("strategy", ["staggered", "sequential"])
def test_converges_to_global_optimum(strategy):
    """Propositions 4.1 / 4.3: DomDec converges to the unique minimiser,
    here checked against global Sinkhorn solved to high precision."""
    N, s = 16, 2
    geo = domdec.Geometry(N, s)
    mu, nu = small_problem(N, seed=1006)
    eps, lam = (2.0 / N) ** 2, 1.0
    C = domdec.full_cost(geo)
    a, b, _, _ = uot.full_sinkhorn(mu, nu, C, eps, lam, err=-1.0, maxit=3000)
    pi = uot.plan(a, b, C, mu, nu, eps)
    Eopt = uot.primal_score(pi, C, mu, nu, eps, lam)
    st = domdec.init_product(geo, mu, nu, eps, lam, thr=1e-30)
    domdec.run(st, 20, strategy, tau=0.0, err=1e-13, maxit=6000)
    # DomDec is stationary once every cell passes its stopping test at once,
    # so the marginals agree up to ~sqrt(2 err) (KL stopping tolerance).
    assert abs(domdec.tracked_score(st) - Eopt) < 1e-9 * Eopt
    assert np.abs(st.PX - pi.sum(1)).sum() < 2e-6 * mu.sum()
    assert np.abs(st.PY - pi.sum(0)).sum() < 2e-6 * mu.sum()
    P, D, gap, beta = domdec.pd_certificate(st)
    assert 0 <= gap < 1e-7


def test_marginal_errors_closed_forms_on_the_product_plan():
    """Section 5.3 ('Solution quality') measures |P_X - e^{-alpha/lam} mu|_1 and
    |P_Y - e^{-beta/lam} nu|_1.  On the product plan pi = mu x nu the marginals
    are P_X = |nu| mu and P_Y = |mu| nu, so for constant potentials alpha = a,
    beta = b both errors have closed forms: |mu| ||nu| - e^{-a/lam}| and
    |nu| ||mu| - e^{-b/lam}|; b = -lam log|mu| makes the Y error vanish."""
    N, s = 8, 2
    geo = domdec.Geometry(N, s)
    mu, nu = inputs.mixture_small(N=N, seed=1013, masses=(0.8, 1.3))
    mu, nu = mu.ravel(), nu.ravel()
    lam = 0.5
    st = domdec.init_product(geo, mu, nu, (1.0 / N) ** 2, lam, thr=0.0)
    M, Nn = mu.sum(), nu.sum()
    for a, b in ((0.0, 0.0), (0.3, 0.7), (-0.2, -lam * np.log(M))):
        st.alpha = np.full(geo.n, a)
        ex, ey = domdec.marginal_errors(st, np.full(geo.n, b))
        assert abs(ex - M * abs(Nn - np.exp(-a / lam))) <= 1e-13
        assert abs(ey - Nn * abs(M - np.exp(-b / lam))) <= 1e-13
    assert ey <= 1e-13


def test_marginal_errors_vanish_at_the_optimum():
    """First-order optimality (Section 4, the marginal conditions of the
    primal-dual pair): at the minimiser P_X = e^{-alpha/lam} mu and
    P_Y = e^{-beta/lam} nu, so both errors fall from O(1) at the product plan
    towards 0 as DomDec converges (beta = beta* of one global Y-half)."""
    N, s = 8, 2
    geo = domdec.Geometry(N, s)
    mu, nu = small_problem(N, seed=1014)
    eps, lam = (2.0 / N) ** 2, 1.0
    st = domdec.init_product(geo, mu, nu, eps, lam, thr=1e-30)
    e0 = domdec.marginal_errors(st, domdec.y_half_global(st, st.alpha))
    assert min(e0) > 1e-2 * mu.sum()
    errs = []
    for n_sweeps, err in ((4, 1e-6), (12, 1e-13)):
        domdec.run(st, n_sweeps, "staggered", tau=0.0, err=err, maxit=6000)
        errs.append(domdec.marginal_errors(st, domdec.pd_certificate(st)[3]))
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]
    assert max(errs[1]) < 1e-6 * mu.sum()


def test_certificate_weak_duality_along_iterations():
    geo = domdec.Geometry(16, 2)
    mu, nu = small_problem(16, seed=1007)
    st = domdec.init_product(geo, mu, nu, (1.0 / 16) ** 2, 0.3)
    gaps = []
    for k in range(4):
        domdec.sweep(st, "AB"[k % 2], "staggered", err=2e-5)
        P, D, g, _ = domdec.pd_certificate(st)
        assert P >= D
        gaps.append(g)
    assert gaps[-1] < gaps[0]


def test_truncation_bounds_lost_mass():
    geo = domdec.Geometry(16, 2)
    mu, nu = small_problem(16, seed=1008)
    st = domdec.init_product(geo, mu, nu, (1.0 / 16) ** 2, 1.0, thr=1e-8)
    full = st.box_entries()
    for k in range(2):
        domdec.sweep(st, "AB"[k % 2], "staggered", err=2e-5)
    assert st.box_entries() < full
    lost = st.PX.sum() - st.PY.sum()
    assert 0 <= lost <= 1e-8 * geo.nbasic * geo.n


def toy_scores(strategy, sweeps=10):
    N = 32
    geo = domdec.Geometry(N, 1, d=1)
    mu = np.full(N, 1.0 / N)
    st = domdec.init_product(geo, mu, mu, 2.0 / N ** 2, 1.0, thr=0.0)
    sc = [domdec.tracked_score(st)]
    domdec.run(st, sweeps, strategy, err=1e-7, maxit=3000,
               record=lambda k, s, lg: sc.append(domdec.tracked_score(s)))
    return np.array(sc)


def test_toy_problem_strategy_behaviour():
    """Section 4.4, 1-D toy (N = 32, mu = nu uniform, lam = 1, eps = 2/N^2,
    pi0 = mu x nu): greedy increases the score at some iteration; safe,
    swift and staggered decrease monotonically; staggered decreases faster
    than safe.  The exact curves are figures only: parity unpinned for them."""
    g = toy_scores("greedy", 6)
    assert np.any(np.diff(g) > 0)
    sf = toy_scores("safe", 6)
    st = toy_scores("staggered", 6)
    assert np.all(np.diff(sf) <= 1e-15) and np.all(np.diff(st) <= 1e-15)
    assert st[-1] < sf[-1]
