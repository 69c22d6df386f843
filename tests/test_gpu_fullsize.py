"""Full-size checks in the benchmark's launch configuration (FP32 cells, the
automatic choice of one CTA or a cluster per cell, staggered swift, warm start
by global Sinkhorn to 2 eps):

* blobs256 (256 x 256, s = 8, eps = (1/256)^2) at lam = 0.1, 1, 10: every cell
  of the first staggered sub-batch against the FP64 oracle solving the same
  cell problems from the GPU's state with the same number of cell iterations,
  and the step size against the oracle's own decision; at lam = 0.1 also both
  converged to a cell tolerance of 1e-7;
* lognormal1024 (1024 x 1024, s = 16, eps = (2/1024)^2): the largest and some
  random cells of that sub-batch with the same number of iterations;
* invariants that hold at any size: P_Y equals the sum of the basic-cell
  marginals, |P_X| = |P_Y|, the tracked score does not increase over sweeps,
  and weak duality of the certificate.
"""
import numpy as np
import pytest

import oracle_pool
from oracle import domdec as odd
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


def oracle_state(g, geo, mu, nu, eps, lam):
    """An oracle State holding the GPU handle's current plan data."""
    st = odd.State(geo, mu, nu, eps, lam, 1e-15)
    st.alpha = g.duals()
    st.PX, st.PY = g.marginals()
    st.Cc, st.Hh = g.basic_costs()
    box, vals = g.basic_marginals()
    pos = 0
    for i in range(geo.nbasic):
        k0, l0, H, W = (int(v) for v in box[i])
        st.lo[i] = (k0, l0)
        st.hi[i] = (k0 + H, l0 + W)
        st.vals[i] = vals[pos:pos + H * W].reshape(H, W).copy()
        pos += H * W
    return st


def warm_started(dd, torch, name, quick):
    mu, nu, spec = inputs.workload(name)
    N, s = spec["N"], spec["s"]
    eps, lam = spec["eps"], spec["lam"]
    mu, nu = mu.ravel(), nu.ravel()
    md = torch.from_numpy(mu.copy()).cuda()
    nd = torch.from_numpy(nu.copy()).cuda()
    a0 = torch.empty(N * N, dtype=torch.float64, device="cuda")
    b0 = torch.empty_like(a0)
    dd.domdec_full_sinkhorn(md, nd, N, 2 * eps, lam, eps_start=1.0, variant=dd.SINKHORN_SEPARABLE,
                            precision=dd.MIXED, maxit=300 if quick else 4000, err=2e-5 if quick else 5e-6,
                            check_every=10, alpha=a0, beta=b0)
    return mu, nu, N, s, eps, lam, md, nd, a0, b0


def check_invariants(dd, g, mu, nu, N, s):
    geo_nbasic = (N // s) ** 2
    PX, PY = g.marginals()
    box, vals = g.basic_marginals()
    acc = np.zeros(N * N)
    pos = 0
    for i in range(geo_nbasic):
        k0, l0, H, W = (int(v) for v in box[i])
        if H * W:
            v = vals[pos:pos + H * W].reshape(H, W)
            acc.reshape(N, N)[k0:k0 + H, l0:l0 + W] += v
        pos += H * W
    assert np.abs(acc - PY).sum() <= 1e-12 * PY.sum()
    assert abs(PX.sum() - PY.sum()) <= 1e-6 * PY.sum()
    cert = g.pd_gap()
    assert cert[1] <= cert[0] + 1e-12 * abs(cert[0])   # weak duality: D <= E_hat


def compare_subbatch(dd, torch, name, lam, ncheck, err, maxit, report):
    """One sweep of partition A in FP32 from the warm start, cells solved to the
    tolerance `err` on both sides; the cells of staggered sub-batch 0 (all of
    them, or the `ncheck` largest and `ncheck` random ones) are solved again by
    the FP64 oracle from the GPU's state before the sweep.  Compares every
    checked cell's potentials on X_J and its members' new marginals after the
    mixing with the GPU's theta; with all cells, also theta against the
    oracle's own GetWeights decision.  Returns the error figures."""
    mu, nu, spec = inputs.workload(name)
    N, s, eps = spec["N"], spec["s"], spec["eps"]
    mu, nu = mu.ravel(), nu.ravel()
    md = torch.from_numpy(mu.copy()).cuda()
    nd = torch.from_numpy(nu.copy()).cuda()
    a0 = torch.empty(N * N, dtype=torch.float64, device="cuda")
    b0 = torch.empty_like(a0)
    dd.domdec_full_sinkhorn(md, nd, N, 2 * eps, lam, eps_start=1.0, variant=dd.SINKHORN_SEPARABLE,
                            precision=dd.MIXED, maxit=4000, err=5e-6, check_every=10, alpha=a0, beta=b0)
    # the bench's launch configuration (automatic cluster choice), tighter cell tolerance
    g = dd.DomDec(md, nd, eps, lam, s, alpha0=a0, beta0=b0, eps_init=2 * eps, precision="fp32", tau=0.0,
                  err=err, maxit=maxit)
    geo = odd.Geometry(N, s)
    st = oracle_state(g, geo, mu, nu, eps, lam)
    g.iterate(1)
    g.sync()
    theta = g.decisions()[0][3]
    box, vals = g.basic_marginals()
    starts = np.concatenate([[0], np.cumsum(box[:, 2] * box[:, 3])])
    alpha_new = g.duals()
    g.close()
    cells = [c for c in geo.parts["A"] if c["sub"] == 0]
    probs_all = [odd.cell_problem(st, c) for c in cells]
    if ncheck is None:
        picks = list(range(len(cells)))
    else:
        size = [0 if p is None else p["Y"].size for p in probs_all]
        order = list(np.argsort(size)[::-1])
        rng = np.random.default_rng(7)
        rest = order[ncheck:]
        picks = order[:ncheck] + list(rng.choice(rest, min(ncheck, len(rest)), replace=False))
    picks = [ci for ci in picks if probs_all[ci] is not None]
    sols = [None] * len(cells)
    for ci, sol in zip(picks, oracle_pool.solve_cells(st, [(cells[ci], probs_all[ci]) for ci in picks], err, maxit)):
        sols[ci] = sol
    l1_num, mass_tot, worst_cell, worst_alpha, worst_shift = 0.0, 0.0, 0.0, 0.0, 0.0
    for ci in picks:
        cell, prob, sol = cells[ci], probs_all[ci], sols[ci]
        a_ref = sol["alpha"]
        # alpha = (the cell's shift along the mass mode (alpha + t, beta - t), which
        # leaves the plan unchanged) + the rest; compared separately
        d = alpha_new[cell["X"]] - a_ref
        worst_shift = max(worst_shift, float(abs(d.mean())))
        worst_alpha = max(worst_alpha, float(np.abs(d - d.mean()).max() / eps))
        lo, hi = prob["lo"], prob["hi"]
        for i in cell["members"]:
            exp_full = np.zeros((N, N))
            mixed = (1 - theta) * st.embed(i, lo, hi) + theta * sol["nut"][i]
            exp_full[lo[0]:hi[0], lo[1]:hi[1]] = np.where(mixed < st.thr, 0.0, mixed)
            got_full = np.zeros((N, N))
            k0, l0, H, W = (int(v) for v in box[i])
            got_full[k0:k0 + H, l0:l0 + W] = vals[starts[i]:starts[i] + H * W].reshape(H, W)
            d = np.abs(got_full - exp_full).sum()
            m = max(exp_full.sum(), 1e-300)
            l1_num += d
            mass_tot += m
            worst_cell = max(worst_cell, d / m)
    out = {"name": name, "lam": lam, "cells": len(picks), "theta": theta, "l1_rel": l1_num / mass_tot,
           "worst_cell_l1_rel": worst_cell, "alpha_max_over_eps": worst_alpha, "alpha_shift": worst_shift,
           "shift_bound": 2 * lam * np.sqrt(err) if err > 0 else 1e-3 * eps}
    if ncheck is None:
        th_ref, E0, Eg, Es = odd.get_weights(st, cells, probs_all, sols, "staggered", 0.0)
        out["theta_oracle"] = th_ref
        out["E_greedy_minus_safe_rel"] = (Eg - Es) / abs(E0)
    report.append(out)
    print("full-size parity:", out)
    return out


@pytest.mark.parametrize("lam", [0.1, 1.0, 10.0])
def test_blobs256_all_cells_of_a_subbatch_fixed_iterations(dd, lam):
    """blobs256 (256 x 256, s = 8, eps = (1/256)^2): every cell of the first
    staggered sub-batch solved with exactly 20 cell iterations by the FP32 GPU
    kernels (in the bench's launch configuration) and by the FP64 oracle from the
    same state: the same iterates up to FP32 arithmetic, so the new marginals
    agree to <= 1e-5 of their mass in L1 over the sub-batch (the stated
    plan-marginal tolerance), and theta equals the oracle's decision unless
    greedy and safe tie within the FP32 error of the score (1e-6).  Per cell the
    FP32 error accumulates over the iterations (the mass mode is damped only by
    about 1 - eps/lam per iteration): measured up to 6e-5 of a cell's mass and
    1.6e-3 eps in the potentials at lam = 1, bounded here by 2e-4 and 5e-3 eps."""
    import torch
    r = compare_subbatch(dd, torch, "blobs256", lam, None, -1.0, 20, [])
    assert r["l1_rel"] <= 1e-5, r
    assert r["worst_cell_l1_rel"] <= 2e-4, r
    assert r["alpha_max_over_eps"] <= 5e-3, r
    assert r["alpha_shift"] <= r["shift_bound"], r
    assert r["theta"] == r["theta_oracle"] or abs(r["E_greedy_minus_safe_rel"]) <= 1e-6, r


def test_blobs256_all_cells_of_a_subbatch_converged(dd):
    """blobs256 at lam = 0.1: every cell of the first staggered sub-batch, FP32
    GPU against the FP64 oracle, both solved to a cell tolerance of 1e-7.  The
    new marginals agree to <= 1e-5 of their mass in L1 over the sub-batch (the
    stated plan-marginal tolerance), each cell to <= 5e-5, the potentials to
    1e-3 eps apart from a constant per cell, and theta equals the oracle's
    decision unless greedy and safe tie within the FP32 error of the score.

    The constant: (alpha + t, beta - t) leaves the cell plan unchanged, so only
    the two marginal penalties fix t; their dual terms are concave in t with
    curvature (|P_X pi| + |P_Y pi|) / lam ~ 2 |mu_J| / lam, and a solve stopped
    at PD <= err lam |mu_J| is within lam sqrt(err) of the optimal t -- two solves
    within 2 lam sqrt(err) of each other."""
    import torch
    r = compare_subbatch(dd, torch, "blobs256", 0.1, None, 1e-7, 3000, [])
    assert r["l1_rel"] <= 1e-5, r
    assert r["worst_cell_l1_rel"] <= 5e-5, r
    assert r["alpha_max_over_eps"] <= 1e-3, r
    assert r["alpha_shift"] <= r["shift_bound"], r
    assert r["theta"] == r["theta_oracle"] or abs(r["E_greedy_minus_safe_rel"]) <= 1e-6, r


def test_lognormal1024_largest_and_random_cells_fixed_iterations(dd):
    """lognormal1024 (1024 x 1024, s = 16, eps = (2/1024)^2): the 3 largest cells
    of the first sub-batch (Y boxes of tens of thousands of points, solved by
    thread-block clusters) and 3 random ones (one CTA each), exactly 10 cell
    iterations by the FP32 GPU kernels and by the FP64 oracle from the same
    state: new marginals within 1e-5 of their mass in L1 over the checked cells,
    per cell and in the potentials the FP32 bounds of the blobs256 test (2e-4,
    5e-3 eps)."""
    import torch
    r = compare_subbatch(dd, torch, "lognormal1024", 1.0, 3, -1.0, 10, [])
    assert r["l1_rel"] <= 1e-5, r
    assert r["worst_cell_l1_rel"] <= 2e-4, r
    assert r["alpha_max_over_eps"] <= 5e-3, r
    assert r["alpha_shift"] <= r["shift_bound"], r


@pytest.mark.parametrize("name", ["blobs256", "lognormal1024"])
def test_invariants_over_sweeps(dd, name):
    """At full size in the bench's configuration (cell tolerance 2e-5): P_Y is
    the sum of the basic-cell marginals, |P_X| = |P_Y|, the tracked score does
    not increase over sweeps (staggered swift, no leniency), weak duality."""
    import torch
    mu, nu, N, s, eps, lam, md, nd, a0, b0 = warm_started(dd, torch, name, False)
    g = dd.DomDec(md, nd, eps, lam, s, alpha0=a0, beta0=b0, eps_init=2 * eps, precision="fp32", tau=0.0,
                  err=2e-5)
    scores = [g.score()[0]]
    for _ in range(4):
        g.iterate(1)
        g.sync()
        scores.append(g.score()[0])
    assert all(b <= a + 1e-7 * abs(a) for a, b in zip(scores, scores[1:])), scores
    check_invariants(dd, g, mu, nu, N, s)
    g.close()
