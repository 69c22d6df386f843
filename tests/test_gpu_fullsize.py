"""Full-size checks in the benchmark's launch configuration (FP32 cells, one CTA
or a 2-CTA cluster per cell, staggered swift, warm start by global Sinkhorn to
2 eps):

* blobs256 (256 x 256, s = 8, eps = (1/256)^2) and lognormal1024 (1024 x 1024,
  s = 16, eps = (2/1024)^2): sampled cells of the first staggered sub-batch
  against the oracle solving the same cell problems one by one from the GPU's
  state (fixed iteration count, so that only FP32 against FP64 arithmetic
  differs), and invariants that hold at any size: P_Y equals the sum of the
  basic-cell marginals, |P_X| = |P_Y|, the tracked score does not increase over
  sweeps, and weak duality of the certificate.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("name,ncheck,quick", [("blobs256", 8, False), ("lognormal1024", 4, False)])
def test_sampled_cells_and_invariants(dd, name, ncheck, quick):
    import torch
    mu, nu, N, s, eps, lam, md, nd, a0, b0 = warm_started(dd, torch, name, quick)
    iters = 20
    g = dd.DomDec(md, nd, eps, lam, s, alpha0=a0, beta0=b0, eps_init=2 * eps, precision="fp32", tau=0.0,
                  err=-1.0, maxit=iters)
    geo = odd.Geometry(N, s)
    st = oracle_state(g, geo, mu, nu, eps, lam)
    scores = [g.score()[0]]
    g.iterate(1)                     # partition A; sub-batch 0 saw exactly the state read above
    g.sync()
    scores.append(g.score()[0])
    theta = g.decisions()[0][3]
    box, vals = g.basic_marginals()
    starts = np.concatenate([[0], np.cumsum(box[:, 2] * box[:, 3])])
    alpha_new = g.duals()
    cells = [c for c in geo.parts["A"] if c["sub"] == 0]
    rng = np.random.default_rng(5)
    picks = rng.choice(len(cells), ncheck, replace=False)
    for ci in picks:
        cell = cells[ci]
        prob = odd.cell_problem(st, cell)
        if prob is None:
            continue
        sol = odd.solve_cell(st, cell, prob, err=-1.0, maxit=iters)
        # the cell's potentials after the solve (kept whatever theta, R7)
        a_ref = sol["alpha"]
        assert np.abs(alpha_new[cell["X"]] - a_ref).max() <= 1e-4 * (eps + np.abs(a_ref).max()) + 2e-3 * eps
        for i in cell["members"]:
            exp_full = np.zeros((N, N))
            lo, hi = prob["lo"], prob["hi"]
            mixed = (1 - theta) * st.embed(i, lo, hi) + theta * sol["nut"][i]
            mixed = np.where(mixed < st.thr, 0.0, mixed)
            exp_full[lo[0]:hi[0], lo[1]:hi[1]] = mixed
            got_full = np.zeros((N, N))
            k0, l0, H, W = (int(v) for v in box[i])
            got_full[k0:k0 + H, l0:l0 + W] = vals[starts[i]:starts[i] + H * W].reshape(H, W)
            mass = max(exp_full.sum(), 1e-300)
            # FP32 cell arithmetic: a plan entry carries ~2^-24 x |exponent| relative error, with
            # exponents up to ~1e3 in the cell frame, over 20 iterations: 2e-4 of the cell's mass
            err = np.abs(got_full - exp_full).sum() / mass
            assert err <= 2e-4, (name, ci, i, err)
    # a few more sweeps: invariants and a non-increasing tracked score
    for _ in range(3):
        g.iterate(1)
        g.sync()
        scores.append(g.score()[0])
    assert all(b <= a + 1e-7 * abs(a) for a, b in zip(scores, scores[1:])), scores
    check_invariants(dd, g, mu, nu, N, s)
    g.close()
