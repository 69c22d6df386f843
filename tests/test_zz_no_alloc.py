"""The allocation-free global Sinkhorn entry point (for callers that cannot
allocate device memory while it runs) gives the same result as the regular,
allocating entry point, on two calls in a row that share its static scratch
array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2410_08859_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_08859_gb300 import domdec
    return torch, domdec


@pytest.mark.parametrize("variant,precision,tol", [(1, 1, 1e-10), (0, 1, 1e-10), (1, 0, 2e-3)])
def test_noalloc_matches_allocating_entry_point_twice(env, variant, precision, tol):
    torch, dd = env
    N = 32
    mu, nu = inputs.mixture_small(N=N, seed=1011)
    mu_d = torch.from_numpy(mu.ravel().copy()).cuda()
    nu_d = torch.from_numpy(nu.ravel().copy()).cuda()
    eps, lam = (2.0 / N) ** 2, 1.5
    a_ref = torch.empty(N * N, dtype=torch.float64, device="cuda")
    b_ref = torch.empty_like(a_ref)
    ref = dd.domdec_full_sinkhorn(mu_d, nu_d, N, eps, lam, eps_start=0.05, variant=variant,
                                  precision=precision, maxit=60, err=1e-6, check_every=5,
                                  alpha=a_ref, beta=b_ref)
    scale = 1.0 + float(a_ref.abs().max())
    for call in range(2):
        a = torch.full_like(a_ref, np.nan)
        b = torch.full_like(a_ref, np.nan)
        got = dd.domdec_full_sinkhorn_noalloc(mu_d, nu_d, N, eps, lam, a, b, eps_start=0.05, variant=variant,
                                              precision=precision, maxit=60, err=1e-6, check_every=5)
        torch.cuda.synchronize()
        assert got[0] == ref[0], (call, got, ref)
        assert float((a - a_ref).abs().max()) <= tol * scale, call
        assert float((b - b_ref).abs().max()) <= tol * scale, call
        for k in (1, 2, 3):
            assert abs(got[k] - ref[k]) <= tol * max(abs(ref[k]), 1e-12), (call, k, got, ref)


def test_noalloc_rejects_grids_beyond_its_capacity(env):
    torch, dd = env
    N = 512
    mu = torch.ones(N * N, dtype=torch.float64, device="cuda")
    a = torch.empty_like(mu)
    b = torch.empty_like(mu)
    with pytest.raises(dd.DomDecError) as e:
        dd.domdec_full_sinkhorn_noalloc(mu, mu, N, 1e-3, 1.0, a, b, maxit=1)
    assert e.value.code == dd.DOMDEC_ETOOBIG
