"""The library's own device math against CUDA's: the table-driven double
logarithm used by the step-size decision (Tang's method) is within a few ulp
of CUDA's log over normal and subnormal inputs and the edges of its table."""
import numpy as np
import pytest

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


def test_table_log_matches_cuda_log(env):
    torch, dd = env
    rng = np.random.default_rng(11)
    x = np.concatenate([
        np.exp(rng.uniform(-740.0, 709.0, 200000)),            # the whole normal range
        rng.uniform(0.5, 2.0, 200000),                         # around 1, both sides of the j = 128 fold
        1.0 + (np.arange(-2000, 2001) / 2.0 ** 20),            # next to 1
        (1.0 + np.arange(129) / 128.0) * (1 + 1e-15),          # the table points c_j
        (1.0 + (np.arange(128) + 0.5) / 128.0),                # half-way between table points
        np.array([5e-324, 1e-310, 2.2250738585072014e-308, 1e-300, 1e300, 1.7976931348623157e308]),
    ])
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    dd.domdec_probe_log(xd, y)
    ref = torch.log(xd)
    err = (y - ref).abs() / torch.clamp(ref.abs(), min=1e-300)
    ulp = torch.from_numpy(np.spacing(np.abs(ref.cpu().numpy()))).cuda()
    err_ulp = ((y - ref).abs() / ulp).max().item()
    assert err_ulp <= 4.0, err_ulp
    assert torch.isfinite(y).all()
    assert float(err.max()) <= 1e-15
