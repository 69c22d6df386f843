"""Pins of GetWeights_line (Proposition 4.3, item 4) in the oracle: the
returned zeta minimises the tracked score over [1/|b|, 1] (brute force over a
fine grid), its derivative formula matches central differences of the score,
it never does worse than swift, and a run with it decreases the score
monotonically towards the global optimum."""
import numpy as np
import pytest

from oracle import domdec as odd
from oracle import uot
from paper_2410_08859_gb300 import inputs


def batch_state(seed, N=16, s=2, lam=1.0, sweeps_before=1):
    mu, nu = inputs.mixture_small(N=N, seed=seed)
    geo = odd.Geometry(N, s)
    st = odd.init_product(geo, mu.ravel(), nu.ravel(), (1.0 / N) ** 2, lam)
    if sweeps_before:
        odd.run(st, sweeps_before, strategy="safe")
    which = "AB"[sweeps_before % 2]
    batch = odd.batches_of(st, which, "line")[0]
    probs = [odd.cell_problem(st, c) for c in batch]
    sols = [None if p is None else odd.solve_cell(st, c, p) for c, p in zip(batch, probs)]
    lo = 1.0 / sum(p is not None for p in probs)
    return st, batch, probs, sols, lo


def score_at(st, batch, probs, sols, z):
    return odd.tracked_score(st, *odd.mixed_quantities(st, batch, probs, sols, z))


@pytest.mark.parametrize("seed,lam,before", [(1200, 1.0, 0), (1201, 1.0, 1), (1202, 5.0, 2), (1203, 0.3, 1)])
def test_line_minimises_tracked_score(seed, lam, before):
    st, batch, probs, sols, lo = batch_state(seed, lam=lam, sweeps_before=before)
    z = odd.line_search(st, batch, probs, sols, lo)
    assert lo <= z <= 1.0
    grid = np.linspace(lo, 1.0, 2001)
    Eg = np.array([score_at(st, batch, probs, sols, t) for t in grid])
    Ez = score_at(st, batch, probs, sols, z)
    assert Ez <= Eg.min() + 1e-13 * abs(Ez)
    # at least as good as both swift candidates
    assert Ez <= score_at(st, batch, probs, sols, 1.0) + 1e-15 * abs(Ez)
    assert Ez <= score_at(st, batch, probs, sols, lo) + 1e-15 * abs(Ez)


def test_line_derivative_matches_central_difference():
    """E'(zeta) used by the search against central differences of the tracked
    score (an independent evaluation through mixed_quantities)."""
    st, batch, probs, sols, lo = batch_state(1204, sweeps_before=1)
    Cg, Hg, PXg, PYg = odd.mixed_quantities(st, batch, probs, sols, 1.0)
    L = float(np.sum(Cg - st.Cc) + st.eps * np.sum(Hg - st.Hh))
    dX, dY = PXg - st.PX, PYg - st.PY
    for z in (lo, 0.5 * (lo + 1), 0.9):
        px, py = st.PX + z * dX, st.PY + z * dY
        m = dY != 0
        g = L + st.lam * np.sum(dX[dX != 0] * np.log(px[dX != 0] / st.mu[dX != 0])) \
            + st.lam * np.sum(dY[m] * np.log(py[m] / st.nu[m]))
        h = 1e-6
        fd = (score_at(st, batch, probs, sols, z + h) - score_at(st, batch, probs, sols, z - h)) / (2 * h)
        assert abs(fd - g) <= 1e-6 * (abs(g) + 1e-9)


def test_line_run_monotone_and_converges():
    N, s = 16, 2
    mu, nu = inputs.mixture_small(N=N, seed=1205)
    mu, nu = mu.ravel(), nu.ravel()
    geo = odd.Geometry(N, s)
    eps, lam = (1.0 / N) ** 2, 1.0
    st = odd.init_product(geo, mu, nu, eps, lam)
    scores = [odd.tracked_score(st)]
    odd.run(st, 30, strategy="line", err=1e-10, maxit=5000,
            record=lambda k, s_, lg: scores.append(odd.tracked_score(s_)))
    assert all(b <= a + 1e-13 * abs(a) for a, b in zip(scores, scores[1:]))
    C = odd.full_cost(geo)
    a, b, _, _ = uot.full_sinkhorn(mu, nu, C, eps, lam, err=1e-13, maxit=100000)
    Eopt = uot.primal_score(uot.plan(a, b, C, mu, nu, eps), C, mu, nu, eps, lam)
    # one uniform weight for all cells of a partition converges slowly on this
    # grid; the distance to the optimum shrinks by over 100x in 30 sweeps
    assert scores[-1] >= Eopt - 1e-12 * abs(Eopt)
    assert scores[-1] - Eopt <= 1e-2 * (scores[0] - Eopt)


def test_staggered_line_never_worse_than_staggered_swift_step():
    """On each staggered sub-batch the line search's step decreases the
    tracked score at least as much as the swift choice would (both evaluated
    on the same cell solutions)."""
    N, s = 16, 2
    mu, nu = inputs.mixture_small(N=N, seed=1206)
    geo = odd.Geometry(N, s)
    st = odd.init_product(geo, mu.ravel(), nu.ravel(), (1.0 / N) ** 2, 1.0)
    odd.run(st, 1, strategy="safe")
    for batch in odd.batches_of(st, "B", "staggered_line"):
        probs = [odd.cell_problem(st, c) for c in batch]
        sols = [None if p is None else odd.solve_cell(st, c, p) for c, p in zip(batch, probs)]
        th_line, E0, Eg, Es = odd.get_weights(st, batch, probs, sols, "staggered_line", 0.0)
        th_swift = odd.get_weights(st, batch, probs, sols, "staggered", 0.0)[0]
        E_line = score_at(st, batch, probs, sols, th_line)
        E_swift = score_at(st, batch, probs, sols, th_swift)
        assert E_line <= E_swift + 1e-13 * abs(E_swift)
        odd.apply_step(st, batch, probs, sols, th_line)
