"""The parallel oracle runs used by the GPU tests give exactly the sequential
oracle's results (same cells, same order, bit-equal arrays)."""
import numpy as np

import oracle_pool
from oracle import domdec as odd
from paper_2410_08859_gb300 import inputs


def test_pool_cell_solves_equal_sequential_ones():
    mu, nu = inputs.mixture_small(N=16, seed=1003)
    geo = odd.Geometry(16, 2)
    st = odd.init_product(geo, mu.ravel(), nu.ravel(), (1 / 16) ** 2, 1.0)
    odd.sweep(st, "A", "staggered")
    cells = [c for c in geo.parts["B"] if c["sub"] == 0]
    jobs = [(c, p) for c in cells for p in [odd.cell_problem(st, c)] if p is not None]
    par = oracle_pool.solve_cells(st, jobs, 1e-7, 500, workers=2)
    seq = [odd.solve_cell(st, c, p, err=1e-7, maxit=500) for c, p in jobs]
    assert len(par) == len(seq) == len(jobs)
    for a, b in zip(par, seq):
        np.testing.assert_array_equal(a["alpha"], b["alpha"])
        for i in b["nut"]:
            np.testing.assert_array_equal(a["nut"][i], b["nut"][i])


def test_pool_trajectories_equal_sequential_sweeps():
    specs = [(16, 2, (2 / 16) ** 2, 1.0, 1033), (16, 4, (1 / 16) ** 2, 0.5, 1034)]
    trajs = oracle_pool.mixture_trajectories(specs, [1, 2])
    assert [len(t) for t in trajs] == [1, 2]
    for (N, s, eps, lam, seed), traj in zip(specs, trajs):
        mu, nu = inputs.mixture_small(N=N, seed=seed)
        st = odd.init_product(odd.Geometry(N, s), mu.ravel(), nu.ravel(), eps, lam)
        for k, (log, got) in enumerate(traj):
            ref = odd.sweep(st, "AB"[k % 2], "staggered")
            assert [r["theta"] for r in log] == [r["theta"] for r in ref]
            np.testing.assert_array_equal(got.PY, st.PY)
            np.testing.assert_array_equal(got.alpha, st.alpha)
