"""GPU parity of the DomDec sweep (C ABI) against the FP64 CPU oracle.

FP64 cell arithmetic: the GPU must reproduce the oracle sweep by sub-batch --
the same theta decisions, the same cell iteration counts, the same boxes, and
scores / marginals / potentials to round-off (tolerances below).
FP32 cell arithmetic: with a fixed number of cell iterations (err < 0) the
same decisions and scores within FP32 error; run to convergence it must reach
the oracle's global optimum within the stated tolerances (relative score
<= 1e-6, plan-marginal L1 <= 1e-5 of the mass).
"""
import numpy as np
import pytest

import oracle_pool
from oracle import domdec as odd
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


def gpu_boxes(g, geo):
    box, vals = g.basic_marginals()
    out = []
    pos = 0
    for i in range(geo.nbasic):
        k0, l0, H, W = box[i]
        out.append((k0, l0, H, W, vals[pos:pos + H * W].reshape(H, W)))
        pos += H * W
    return out


def compare_state(g, st, tol_score, tol_l1, tol_alpha, check_boxes=True, tol_box=None):
    sc = g.score()
    ref = odd.score_terms(st)
    assert abs(sc[0] - ref[0]) <= tol_score * abs(ref[0]), (sc[0], ref[0])
    PX, PY = g.marginals()
    mass = st.mu.sum()
    assert np.abs(PX - st.PX).sum() <= tol_l1 * mass
    assert np.abs(PY - st.PY).sum() <= tol_l1 * mass
    a = g.duals()
    assert np.abs(a - st.alpha).max() <= tol_alpha * (1 + np.abs(st.alpha).max())
    # the tracked per-basic-cell terms (C_i + eps H_i) that the score sums
    Cg, Hg = g.basic_costs()
    assert np.abs((Cg + st.eps * Hg) - (st.Cc + st.eps * st.Hh)).sum() <= 10 * tol_score * abs(ref[0])
    if check_boxes:
        for i, (k0, l0, H, W, v) in enumerate(gpu_boxes(g, st.geo)):
            lo, hi = st.lo[i], st.hi[i]
            assert (k0, l0, H, W) == (lo[0], lo[1], hi[0] - lo[0], hi[1] - lo[1]), i
            if tol_box is not None and v.size:
                assert np.abs(v - st.vals[i]).max() <= tol_box * max(st.vals[i].max(), 1e-300)


_ORACLE_RUNS = {}


def oracle_run(N, s, mu, nu, eps, lam, sweeps, strategy, err, maxit, tau, thr, init_duals, ti, balance):
    """The oracle's trajectory (initial state, then the decision log and the state
    after every sweep), computed once per distinct problem and shared by the
    tests that replay it with different launch shapes or precisions."""
    import copy
    import hashlib

    def h(*arrs):
        m = hashlib.sha1()
        for a in arrs:
            m.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
        return m.hexdigest()

    key = (N, s, h(mu, nu), eps, lam, strategy, err, maxit, tau, thr,
           None if init_duals is None else (h(init_duals[0], init_duals[1]), init_duals[2]), ti, balance)
    if key not in _ORACLE_RUNS:
        geo = odd.Geometry(N, s)
        if init_duals is None:
            st = odd.init_product(geo, mu, nu, eps, lam, thr)
        else:
            a0, b0, e0 = init_duals
            st = odd.init_from_duals(geo, mu, nu, a0, b0, e0, eps, lam, thr)
        _ORACLE_RUNS[key] = [(None, copy.deepcopy(st))]
    traj = _ORACLE_RUNS[key]
    while len(traj) <= sweeps:   # extend a shorter trajectory of the same problem
        st = copy.deepcopy(traj[-1][1])
        log = odd.sweep(st, "AB"[(len(traj) - 1) % 2], strategy, tau=tau, err=err, maxit=maxit, ti=bool(ti),
                        balance=bool(balance))
        traj.append((log, st))
    return traj[:sweeps + 1]


def run_pair(dd, N, s, mu, nu, eps, lam, sweeps, precision, strategy="staggered", err=2e-5, maxit=2000,
             tau=0.0, thr=1e-15, tols=(1e-10, 1e-10, 1e-8), tol_box=1e-8, init_duals=None, cell_ctas=0,
             ti=0, balance=0):
    mu, nu = mu.ravel(), nu.ravel()
    if strategy == "sequential":
        raise ValueError
    kw = dict(precision=precision, strategy=strategy, err=err, maxit=maxit, tau=tau, trunc_thr=thr,
              cell_ctas=cell_ctas, cell_ti=ti, balance=balance)
    traj = oracle_run(N, s, mu, nu, eps, lam, sweeps, strategy, err, maxit, tau, thr, init_duals, ti, balance)
    if init_duals is None:
        g = dd.DomDec(mu, nu, eps, lam, s, **kw)
    else:
        a0, b0, e0 = init_duals
        g = dd.DomDec(mu, nu, eps, lam, s, alpha0=a0, beta0=b0, eps_init=e0, **kw)
    st = traj[0][1]
    compare_state(g, st, *tols, tol_box=tol_box)
    nrec = 0
    for k in range(sweeps):
        log, st = traj[k + 1]
        g.iterate(1)
        rc = g.sync()
        assert rc in (0, 1)
        dec = g.decisions()
        assert len(dec) == nrec + len(log)
        for rec, d in zip(log, dec[nrec:]):
            if strategy in ("line", "staggered_line"):   # a search's root: equal to its rounding
                assert abs(d[3] - rec["theta"]) <= 1e-9, (k, d, rec)
            else:
                assert d[3] == rec["theta"], (k, d, rec)
        nrec += len(log)
        if precision == "fp64" or err < 0:
            st_iters = sum(sum(r["iters"]) for r in log)
            assert g.stats()["cell_iters"] - getattr(g, "_it", 0) == st_iters
            g._it = g.stats()["cell_iters"]
        compare_state(g, st, *tols, tol_box=tol_box)
    return g, st


@pytest.mark.parametrize("cell_ctas", [0, 1, 2, 4, 8])
def test_fp64_sweeps_match_oracle_mix32(dd, cell_ctas):
    """Small Gaussian-mixture workload (32 x 32, s = 4, eps = (1/32)^2, lam = 1,
    FP64, pi0 = mu x nu): three sweeps, sub-batch by sub-batch; cells solved by
    one CTA each (1), by clusters of 2, 4 or 8 CTAs that split the Y box by
    rows (2, 4, 8), or chosen automatically (0)."""
    mu, nu = inputs.mixture_small(N=32, seed=1000)
    g, st = run_pair(dd, 32, 4, mu, nu, (1 / 32) ** 2, 1.0, 3, "fp64", cell_ctas=cell_ctas)
    g.close()


@pytest.mark.parametrize("cell_ctas", [0, 4])
def test_fp64_ragged_partition_and_odd_cell_size(dd, cell_ctas):
    """N = 24, s = 3: B cells clipped at the border (1x1, 1x2, 2x1 basic cells),
    odd cell sides, boxes that touch the grid edge; on one CTA or 4-CTA clusters
    (uneven row slabs)."""
    mu, nu = inputs.mixture_small(N=24, seed=1002)
    g, st = run_pair(dd, 24, 3, mu, nu, (1 / 24) ** 2, 0.5, 2, "fp64", cell_ctas=cell_ctas)
    g.close()


@pytest.mark.parametrize("strategy", ["swift", "safe", "greedy"])
def test_fp64_other_strategies(dd, strategy):
    mu, nu = inputs.mixture_small(N=16, seed=1003)
    g, st = run_pair(dd, 16, 2, mu, nu, (1 / 16) ** 2, 2.0, 2, "fp64", strategy=strategy)
    g.close()


@pytest.mark.parametrize("lam", [1.0, 5.0])
def test_fp64_line_search_matches_oracle(dd, lam):
    """GetWeights_line (strategy 'line'): the device search returns the
    oracle's zeta (to the search's rounding) and the states agree."""
    mu, nu = inputs.mixture_small(N=16, seed=1011)
    g, st = run_pair(dd, 16, 2, mu, nu, (1 / 16) ** 2, lam, 4, "fp64", strategy="line")
    dec = g.decisions()
    assert any(0.07 < d[3] < 1.0 for d in dec)   # an interior zeta (lo <= 1/16) was exercised
    g.close()


@pytest.mark.parametrize("N,s,lam", [(16, 2, 1.0), (16, 2, 5.0), (24, 3, 1.0)])
def test_fp64_balancing_matches_oracle(dd, N, s, lam):
    """Balancing step (Eq. balancing) after every cell solve: FP64 sweeps match
    the oracle's balanced sweeps (decisions, iteration counts, boxes, state),
    including border cells of the B partition with 1 or 2 basic cells."""
    mu, nu = inputs.mixture_small(N=N, seed=1012)
    g, st = run_pair(dd, N, s, mu, nu, (1 / N) ** 2, lam, 3, "fp64", balance=1)
    g.close()


_OPTIMA = {}


def global_optimum(N, seed, eps, lam):
    """The unique UOT optimum of the 32 x 32 mixture (seed), computed once by the
    oracle's global Sinkhorn with the translation step (the same fixed point as
    plain alternation, reached in far fewer iterations); (pi, score)."""
    key = (N, seed, eps, lam)
    if key not in _OPTIMA:
        mu, nu = inputs.mixture_small(N=N, seed=seed)
        mu, nu = mu.ravel(), nu.ravel()
        C = odd.full_cost(odd.Geometry(N, 4))
        # PD/lam <= 1e-11 |mu|: the score within ~1e-11 of the optimum, far inside the
        # tested 1e-6 relative score and 1e-5 marginal tolerances
        a, b, it, gap = uot.full_sinkhorn(mu, nu, C, eps, lam, err=1e-11, maxit=20000, ti=True)
        assert gap <= 1e-11 * mu.sum(), gap
        pi = uot.plan(a, b, C, mu, nu, eps)
        _OPTIMA[key] = (pi, uot.primal_score(pi, C, mu, nu, eps, lam))
    return _OPTIMA[key]


def test_fp32_balancing_converges_to_oracle_optimum(dd):
    N, s = 32, 4
    mu, nu = inputs.mixture_small(N=N, seed=1006)
    mu, nu = mu.ravel(), nu.ravel()
    eps, lam = (1 / N) ** 2, 1.0
    pi, Eopt = global_optimum(N, 1006, eps, lam)
    g = dd.DomDec(mu, nu, eps, lam, s, precision="fp32", err=1e-12, maxit=2000, tau=0.0, balance=1)
    g.iterate(30)
    g.sync()
    E = g.score()[0]
    PX, PY = g.marginals()
    assert abs(E - Eopt) <= 1e-6 * Eopt, (E, Eopt)
    assert np.abs(PX - pi.sum(1)).sum() / mu.sum() <= 1e-5
    assert np.abs(PY - pi.sum(0)).sum() / mu.sum() <= 1e-5
    g.close()


def test_fp64_staggered_line_search_matches_oracle(dd):
    """Staggered sub-batches with GetWeights_line on each (strategy 'staggered_line')."""
    mu, nu = inputs.mixture_small(N=32, seed=1013)
    g, st = run_pair(dd, 32, 4, mu, nu, (1 / 32) ** 2, 1.0, 3, "fp64", strategy="staggered_line")
    g.close()


def test_fp64_truncation_and_leniency(dd):
    mu, nu = inputs.mixture_small(N=16, seed=1004)
    g, st = run_pair(dd, 16, 2, mu, nu, (1 / 16) ** 2, 1.0, 3, "fp64", thr=1e-9, tau=0.005)
    g.close()


def test_fp64_warm_start_from_duals(dd):
    """pi0 from global Sinkhorn duals at eps0 = 2 eps (Section 5.3 warm start);
    the duals come from the oracle."""
    N, s = 32, 4
    mu, nu = inputs.mixture_small(N=N, seed=1005)
    mu, nu = mu.ravel(), nu.ravel()
    geo = odd.Geometry(N, s)
    eps = (1 / N) ** 2
    a0, b0, _, _ = uot.full_sinkhorn(mu, nu, odd.full_cost(geo), 2 * eps, 1.0, err=1e-6, ti=True)
    g, st = run_pair(dd, N, s, mu, nu, eps, 1.0, 2, "fp64", init_duals=(a0, b0, 2 * eps),
                     tols=(1e-9, 1e-9, 1e-8))
    g.close()


@pytest.mark.parametrize("cell_ctas", [0, 1, 4])
def test_fp32_fixed_iterations_match_oracle(dd, cell_ctas):
    """FP32 cell arithmetic with exactly 12 cell iterations per solve: same
    decisions; scores and marginals within FP32 error of the FP64 oracle."""
    mu, nu = inputs.mixture_small(N=32, seed=1000)
    g, st = run_pair(dd, 32, 4, mu, nu, (1 / 32) ** 2, 1.0, 2, "fp32", err=-1.0, maxit=12,
                     tols=(1e-6, 1e-5, 1e-4), tol_box=None, cell_ctas=cell_ctas)
    g.close()


@pytest.mark.parametrize("cell_ctas", [0, 1])
def test_fp64_translation_step_matches_oracle(dd, cell_ctas):
    """Cell Sinkhorn with the translation step (cell_ti = 1) from a global
    Sinkhorn warm start at 2 eps with eps << lam: FP64 sweeps match the
    oracle's ti=True sweeps (decisions, iteration counts, state)."""
    N, s = 32, 4
    mu, nu = inputs.mixture_blobs(N=N, seed=1010)
    mu, nu = mu.ravel(), nu.ravel()
    geo = odd.Geometry(N, s)
    eps = (1 / N) ** 2
    a0, b0, _, _ = uot.full_sinkhorn(mu, nu, odd.full_cost(geo), 2 * eps, 1.0, err=1e-6, ti=True)
    g, st = run_pair(dd, N, s, mu, nu, eps, 1.0, 3, "fp64", err=1e-7, maxit=5000, init_duals=(a0, b0, 2 * eps),
                     tols=(1e-9, 1e-9, 1e-8), cell_ctas=cell_ctas, ti=1)
    g.close()


def test_fp32_translation_step_converges_to_oracle_optimum(dd):
    """FP32 cells with the translation step reach the oracle's optimum within
    the stated tolerances (relative score 1e-6, marginal L1 1e-5)."""
    N, s = 32, 4
    mu, nu = inputs.mixture_small(N=N, seed=1006)
    mu, nu = mu.ravel(), nu.ravel()
    eps, lam = (1 / N) ** 2, 1.0
    pi, Eopt = global_optimum(N, 1006, eps, lam)
    g = dd.DomDec(mu, nu, eps, lam, s, precision="fp32", err=1e-12, maxit=2000, tau=0.0, cell_ti=1)
    g.iterate(30)
    g.sync()
    E = g.score()[0]
    PX, PY = g.marginals()
    assert abs(E - Eopt) <= 1e-6 * Eopt, (E, Eopt)
    assert np.abs(PX - pi.sum(1)).sum() / mu.sum() <= 1e-5
    assert np.abs(PY - pi.sum(0)).sum() / mu.sum() <= 1e-5
    g.close()


def test_fp32_converges_to_oracle_optimum(dd):
    """DomDec in FP32 run to convergence reaches the unique UOT optimum computed
    by the oracle's global Sinkhorn: relative score <= 1e-6, marginal L1 <= 1e-5."""
    N, s = 32, 4
    mu, nu = inputs.mixture_small(N=N, seed=1006)
    mu, nu = mu.ravel(), nu.ravel()
    eps, lam = (1 / N) ** 2, 1.0
    pi, Eopt = global_optimum(N, 1006, eps, lam)
    g = dd.DomDec(mu, nu, eps, lam, s, precision="fp32", err=1e-12, maxit=2000, tau=0.0)
    g.iterate(30)
    g.sync()
    E = g.score()[0]
    PX, PY = g.marginals()
    ex = np.abs(PX - pi.sum(1)).sum() / mu.sum()
    ey = np.abs(PY - pi.sum(0)).sum() / mu.sum()
    assert abs(E - Eopt) <= 1e-6 * Eopt, (E, Eopt)
    assert ex <= 1e-5 and ey <= 1e-5, (ex, ey)
    cert = g.pd_gap()
    assert 0 <= cert[2] < 1e-5
    g.close()


def test_certificate_matches_oracle(dd):
    mu, nu = inputs.mixture_small(N=16, seed=1007)
    g, st = run_pair(dd, 16, 2, mu, nu, (1 / 16) ** 2, 0.7, 2, "fp64")
    P, D, rel, beta = odd.pd_certificate(st)
    out, gb = g.pd_gap(with_beta=True)
    assert abs(out[0] - P) <= 1e-10 * abs(P)
    assert abs(out[1] - D) <= 1e-10 * abs(D)
    assert np.abs(gb - beta).max() <= 1e-9 * (1 + np.abs(beta).max())
    ex, ey = odd.marginal_errors(st, beta)
    assert abs(out[3] - ex) <= 1e-9 and abs(out[4] - ey) <= 1e-9
    g.close()


@pytest.mark.parametrize("variant,precision,tol", [(1, 1, 1e-10), (0, 1, 1e-10), (1, 0, 2e-3), (0, 0, 2e-3),
                                                   (5, 1, 1e-10), (4, 1, 1e-10), (5, 0, 2e-3), (1, 2, 1e-6),
                                                   (5, 2, 1e-6)])
def test_full_sinkhorn_matches_oracle(dd, variant, precision, tol):
    """Global Sinkhorn (Eq. sinkhorn-iters-ot): separable and dense evaluation,
    FP64, FP32 and mixed (float exponentials of double exponents: ~1e-7 relative
    per log-sum-exp, so 1e-6 here), with and without the translation step
    (variant bit 4), against the oracle with the same iteration count."""
    N = 16
    mu, nu = inputs.mixture_small(N=N, seed=1008)
    mu, nu = mu.ravel(), nu.ravel()
    geo = odd.Geometry(N, 2)
    eps, lam = (2 / N) ** 2, 1.5
    a_ref, b_ref, it_ref, gap_ref = uot.full_sinkhorn(mu, nu, odd.full_cost(geo), eps, lam, err=-1, maxit=40,
                                                      ti=bool(variant & 4))
    alpha, beta = np.empty(N * N), np.empty(N * N)
    it, gap, P, D, rc = dd.domdec_full_sinkhorn(mu, nu, N, eps, lam, variant=variant, precision=precision,
                                                maxit=40, err=-1.0, check_every=40, alpha=alpha, beta=beta)
    assert it == 40
    scale = 1 + np.abs(a_ref).max()
    assert np.abs(alpha - a_ref).max() <= tol * scale
    assert np.abs(beta - b_ref).max() <= tol * scale
    # relative agreement, plus an absolute floor of 1e-16 |mu| for the rounding
    # of a KL sum whose terms are ~1e-8 (the translation step converges far)
    assert abs(gap - gap_ref) <= max(tol, 1e-12) * max(gap_ref, 1e-12) * (1 if precision == 1 else 1e3) + 1e-16
    assert P >= D


def test_error_states_are_reported_and_sticky(dd):
    """A cell Y-box larger than the kernel capacity (one CTA per cell, no spill
    slots) is reported by the kernel (no fault), then the handle refuses
    further work."""
    mu, nu = inputs.mixture_small(N=32, seed=1009)
    g = dd.DomDec(mu, nu, (1 / 32) ** 2, 1.0, 4, precision="fp32", max_ny=256, spill_slots=-1, cell_ctas=1)
    g.iterate(1)
    with pytest.raises(dd.DomDecError) as e:
        g.sync()
    assert e.value.code == dd.DOMDEC_ETOOBIG
    with pytest.raises(dd.DomDecError) as e:
        g.iterate(1)
    assert e.value.code == dd.DOMDEC_ESTATE
    g.close()
    bad = mu.copy()
    bad[3] = -1.0
    with pytest.raises(dd.DomDecError) as e:
        dd.DomDec(bad, nu, (1 / 32) ** 2, 1.0, 4)
    assert e.value.code == dd.DOMDEC_EINVAL


@pytest.mark.parametrize("cell_ctas", [0, 1])
def test_fp64_spilled_boxes_match_oracle(dd, cell_ctas):
    """Cells whose Y-box exceeds one CTA's capacity (here every cell of the
    first sweeps: 32 x 32 boxes > max_ny = 256): with one CTA per cell (1) they
    run from global spill slots; automatically (0) they go to a cluster, whose
    new marginals exceed the per-cell buffer and take a spill slot."""
    mu, nu = inputs.mixture_small(N=32, seed=1000)
    geo = odd.Geometry(32, 4)
    mu, nu = mu.ravel(), nu.ravel()
    eps = (1 / 32) ** 2
    traj = oracle_run(32, 4, mu, nu, eps, 1.0, 2, "staggered", 2e-5, 2000, 0.0, 1e-15, None, 0, 0)
    g = dd.DomDec(mu, nu, eps, 1.0, 4, precision="fp64", max_ny=256, spill_slots=4, cell_ctas=cell_ctas)
    for k in range(2):
        st = traj[k + 1][1]
        g.iterate(1)
        g.sync()
        if cell_ctas == 1:
            assert (g.cell_log()[:, 7] >= 0).any() or k > 0
        compare_state(g, st, 1e-10, 1e-10, 1e-8, tol_box=1e-8)
    g.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_batch_of_instances_matches_single_runs(dd, precision, tol):
    """Many-instance batching: three different problems (grid, cell size, eps,
    lam) swept together give the states of the same problems swept alone (in
    FP32 within the stated plan-marginal tolerance: the batch and the single
    handles may solve a cell with different kernels, one CTA or a cluster)."""
    specs = [(32, 4, (1 / 32) ** 2, 1.0, 1000), (16, 2, (2 / 16) ** 2, 0.5, 1001), (24, 3, (1 / 24) ** 2, 5.0, 1002)]
    alone, batched = [], []
    for N, s, eps, lam, seed in specs:
        mu, nu = inputs.mixture_small(N=N, seed=seed)
        for lst in (alone, batched):
            lst.append(dd.DomDec(mu, nu, eps, lam, s, precision=precision))
    for g in alone:
        g.iterate(3)
        g.sync()
    B = dd.DomDecBatch(batched)
    B.iterate(3)
    assert B.sync() in (0, 1)
    for g1, g2 in zip(alone, batched):
        s1, s2 = g1.score(), g2.score()
        assert abs(s1[0] - s2[0]) <= tol * abs(s1[0])
        np.testing.assert_array_equal(g1.decisions()[:, 3], g2.decisions()[:, 3])
        PX1, PY1 = g1.marginals()
        PX2, PY2 = g2.marginals()
        assert np.abs(PX1 - PX2).sum() <= tol * PX1.sum()
        assert np.abs(PY1 - PY2).sum() <= tol * PY1.sum()
        assert g1.stats()["cell_iters"] == g2.stats()["cell_iters"] or precision == "fp32"
    C, f = B.autotune()
    assert C in (1, 2, 4) and f in (1.0, 2.0, 4.0)
    B.iterate(1)
    B.sync()
    B.close()
    for g in alone + batched:
        g.close()


def test_maxit_warning(dd):
    mu, nu = inputs.mixture_small(N=16, seed=1010)
    g = dd.DomDec(mu, nu, (1 / 16) ** 2, 1.0, 2, precision="fp32", err=1e-12, maxit=2)
    g.iterate(1)
    assert g.sync() == dd.DOMDEC_WNOTCONV
    n_maxit = g.stats()["maxit_cells"]
    assert n_maxit > 0
    # the warning covers the solves since the previous sync only: with a loose
    # tolerance every cell converges within the cap and the next sync is clean
    assert g.sync() == dd.DOMDEC_OK
    g.set_tolerance(1e30)
    g.iterate(1)
    assert g.sync() == dd.DOMDEC_OK
    assert g.stats()["maxit_cells"] == n_maxit
    g.set_tolerance(1e-12)
    g.iterate(1)
    assert g.sync() == dd.DOMDEC_WNOTCONV
    g.close()


@pytest.mark.parametrize("with_duals", [False, True])
def test_reset_reuses_the_handle(dd, with_duals):
    """domdec_reset loads a new problem into an existing handle: the sweeps
    that follow equal those of a fresh handle on that problem (same decisions,
    iteration counts and state), and counters, sweep count and eps restart."""
    N, s = 32, 4
    eps, lam = (1 / N) ** 2, 1.0
    probs = [inputs.mixture_small(N=N, seed=1020 + k) for k in range(2)]
    geo = odd.Geometry(N, s)
    duals = []
    for mu, nu in probs:
        if with_duals:
            a0, b0, _, _ = uot.full_sinkhorn(mu.ravel(), nu.ravel(), odd.full_cost(geo), 2 * eps, lam, err=1e-6, ti=True)
            duals.append(dict(alpha0=a0, beta0=b0, eps_init=2 * eps))
        else:
            duals.append({})
    g = dd.DomDec(probs[0][0], probs[0][1], eps, lam, s, precision="fp64", **duals[0])
    g.iterate(2)
    g.set_eps(2 * eps)
    g.iterate(1)
    g.sync()
    for k in (1, 0):
        mu, nu = probs[k]
        g.reset(mu.ravel(), nu.ravel(), **duals[k])
        assert g.stats()["sweeps"] == 0 and g.stats()["cell_iters"] == 0
        ref = dd.DomDec(mu, nu, eps, lam, s, precision="fp64", **duals[k])
        for h in (g, ref):
            h.iterate(3)
            h.sync()
        np.testing.assert_array_equal(g.decisions()[:, 3], ref.decisions()[:, 3])
        assert g.stats()["cell_iters"] == ref.stats()["cell_iters"]
        assert abs(g.score()[0] - ref.score()[0]) <= 1e-12 * abs(ref.score()[0])
        PX1, PY1 = g.marginals()
        PX2, PY2 = ref.marginals()
        assert np.abs(PY1 - PY2).sum() <= 1e-12 * PY2.sum()
        ref.close()
    g.close()


def test_batch_instances_match_their_oracle_runs(dd):
    """Many-instance batching against the oracle: four different problems
    (64 x 64 with s = 8 and lam = 1; 32 x 32, lam = 5; the ragged 24 x 24 with
    s = 3; 16 x 16) swept together in FP64 for two sweeps; after every sweep
    each instance has its own oracle run's decisions, cell iteration counts and
    state (the 64 x 64 instance after the first)."""
    specs = [(64, 8, (2 / 64) ** 2, 1.0, 1030), (32, 4, (1 / 32) ** 2, 5.0, 1031),
             (24, 3, (1 / 24) ** 2, 0.5, 1032), (16, 2, (2 / 16) ** 2, 1.0, 1033)]
    # the oracle runs, one process per problem; the 64 x 64 one (dense 256 x 4096 cell
    # problems from pi0 = mu x nu, minutes of NumPy per sweep) for the first sweep only
    trajs = oracle_pool.mixture_trajectories(specs, [1, 2, 2, 2])
    hs = []
    for N, s, eps, lam, seed in specs:
        mu, nu = inputs.mixture_small(N=N, seed=seed)
        hs.append(dd.DomDec(mu.ravel(), nu.ravel(), eps, lam, s, precision="fp64"))
    B = dd.DomDecBatch(hs)
    nrec = [0] * len(hs)
    its = [0] * len(hs)
    for k in range(2):
        B.iterate(1)
        assert B.sync() in (0, 1)
        for j, g in enumerate(hs):
            if k >= len(trajs[j]):
                continue
            log, st = trajs[j][k]
            dec = g.decisions()
            assert len(dec) == nrec[j] + len(log)
            for rec, d in zip(log, dec[nrec[j]:]):
                assert d[3] == rec["theta"], (j, k, d, rec)
            nrec[j] += len(log)
            its[j] += sum(sum(r["iters"]) for r in log)
            assert g.stats()["cell_iters"] == its[j], j
            compare_state(g, st, 1e-10, 1e-10, 1e-8, tol_box=1e-8)
    B.close()
    for g in hs:
        g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_arena_overflow_grows_and_reruns(dd, precision):
    """A box arena far too small for the sweeps (arena_factor tiny: capacity =
    the initial plan): the first sub-batch whose new boxes do not fit halts the
    enqueued sweeps before changing anything, the next synchronisation grows
    the arena and reruns what was skipped -- same decisions, iteration counts
    and scores as with the default arena, no error."""
    mu, nu = inputs.mixture_small(N=32, seed=1040)
    eps, lam = (1 / 32) ** 2, 1.0
    ref = dd.DomDec(mu, nu, eps, lam, 4, precision=precision)
    small = dd.DomDec(mu, nu, eps, lam, 4, precision=precision, arena_factor=1e-9)
    for g in (ref, small):
        g.iterate(4)
        assert g.sync() in (0, 1)
    assert small.stats()["arena_regrows"] >= 1 and ref.stats()["arena_regrows"] == 0
    np.testing.assert_array_equal(small.decisions()[:, 3], ref.decisions()[:, 3])
    if precision == "fp64":   # FP32 iteration counts may differ by round-off in P_Y's atomic sums
        assert small.stats()["cell_iters"] == ref.stats()["cell_iters"]
    assert small.stats()["sweeps"] == ref.stats()["sweeps"] == 4
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert abs(small.score()[0] - ref.score()[0]) <= tol * abs(ref.score()[0])
    small.iterate(2)
    ref.iterate(2)
    assert small.sync() in (0, 1) and ref.sync() in (0, 1)
    assert abs(small.score()[0] - ref.score()[0]) <= tol * abs(ref.score()[0])
    for g in (ref, small):
        g.close()


def test_autotune_keeps_the_iterates(dd):
    """domdec_autotune times one sweep per candidate launch shape (cluster size,
    split threshold) and keeps the fastest: in FP64 the cell results do not
    depend on the launch shape, so the tuned handle follows the untuned one
    sweep for sweep (same decisions, iteration counts and state)."""
    mu, nu = inputs.mixture_small(N=64, seed=1050)
    eps, lam = (2 / 64) ** 2, 1.0
    g = dd.DomDec(mu, nu, eps, lam, 8, precision="fp64")
    ref = dd.DomDec(mu, nu, eps, lam, 8, precision="fp64")
    C, f = g.autotune()
    assert C in (1, 2, 4, 8) and f in (0.5, 1.0, 2.0)
    n = g.stats()["sweeps"]
    assert n >= 1
    g.iterate(2)
    ref.iterate(n + 2)
    assert g.sync() in (0, 1) and ref.sync() in (0, 1)
    np.testing.assert_array_equal(g.decisions()[:, 3], ref.decisions()[:, 3])
    assert g.stats()["cell_iters"] == ref.stats()["cell_iters"]
    assert abs(g.score()[0] - ref.score()[0]) <= 1e-12 * abs(ref.score()[0])
    PX1, PY1 = g.marginals()
    PX2, PY2 = ref.marginals()
    assert np.abs(PY1 - PY2).sum() <= 1e-12 * PY2.sum()
    for h in (g, ref):
        h.close()


def test_too_small_launch_cluster_regroups(dd):
    """A launch shape that cannot hold the cells (one CTA per cell while every
    box exceeds max_ny = 256 and no spill slot exists): the sweep halts before
    its cell solves, the next synchronisation reruns it with the layout's
    largest cluster -- the same sweeps as the oracle, no error."""
    mu, nu = inputs.mixture_small(N=32, seed=1000)
    geo = odd.Geometry(32, 4)
    mu, nu = mu.ravel(), nu.ravel()
    eps = (1 / 32) ** 2
    traj = oracle_run(32, 4, mu, nu, eps, 1.0, 2, "staggered", 2e-5, 2000, 0.0, 1e-15, None, 0, 0)
    g = dd.DomDec(mu, nu, eps, 1.0, 4, precision="fp64", max_ny=256, spill_slots=-1)
    assert g.set_launch(1, 2.0) == 1
    for k in range(2):
        st = traj[k + 1][1]
        g.iterate(1)
        assert g.sync() in (0, 1)
        compare_state(g, st, 1e-10, 1e-10, 1e-8, tol_box=1e-8)
    assert g.stats()["cluster_regroups"] >= 1
    assert g.stats()["sweeps"] == 2
    g.close()
