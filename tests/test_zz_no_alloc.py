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


def test_noalloc_rejects_host_memory_before_any_launch(env):
    """Host arrays never reach the kernels: the binding raises on NumPy input
    and on CPU tensors, and the C entry point itself returns DOMDEC_EINVAL for
    host pointers (pageable and pinned) before it enqueues anything."""
    import ctypes
    torch, dd = env
    N = 16
    mu, nu = inputs.mixture_small(N=N, seed=1012)
    mu, nu = mu.ravel().copy(), nu.ravel().copy()
    a = torch.empty(N * N, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    with pytest.raises(TypeError):
        dd.domdec_full_sinkhorn_noalloc(mu, nu, N, 1e-2, 1.0, a, b, maxit=1)
    with pytest.raises(TypeError):
        dd.domdec_full_sinkhorn_noalloc(torch.from_numpy(mu), torch.from_numpy(nu), N, 1e-2, 1.0, a, b, maxit=1)
    mu_d = torch.from_numpy(mu).cuda()
    nu_d = torch.from_numpy(nu).cuda()
    pinned = torch.from_numpy(mu).pin_memory()
    out = (ctypes.c_double * 4)()
    L = dd.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for m_ptr, n_ptr, a_ptr in ((mu.ctypes.data, nu_d.data_ptr(), a.data_ptr()),
                                (mu_d.data_ptr(), nu_d.data_ptr(), mu.ctypes.data),
                                (pinned.data_ptr(), nu_d.data_ptr(), a.data_ptr())):
        a.fill_(7.0)
        rc = L.domdec_full_sinkhorn_noalloc(m_ptr, n_ptr, N, 1e-2, 1e-2, 1.0, 1, 1, 1, 1e-6, 1, None,
                                            a_ptr, b.data_ptr(), out, stream)
        torch.cuda.synchronize()
        assert rc == dd.DOMDEC_EINVAL
        assert bool((a == 7.0).all())   # nothing was written
