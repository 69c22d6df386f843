"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/domdec.h declares; argument validation that needs no
device runs on the CPU."""
import ctypes
import os
import re

import pytest

from paper_2410_08859_gb300 import build as B

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "domdec.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(domdec_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_default_params_and_error_strings():
    from paper_2410_08859_gb300 import domdec as dd
    p = dd.domdec_default_params()
    assert p.err == 2e-5 and p.trunc_thr == 1e-15 and p.strategy == dd.STAGGERED
    assert p.basic_cell == 4 and p.precision == dd.FP32
    # the paper's plain iteration by default: no translation step, no balancing
    assert p.cell_ti == 0 and p.balance == 0 and p.cell_ctas == 0
    assert dd.domdec_default_params(strategy="staggered_line").strategy == dd.STAGGERED_LINE == 5
    assert dd.error_string(dd.DOMDEC_EINVAL) == "invalid argument"
    assert "arena" in dd.error_string(dd.DOMDEC_EARENA)


@pytest.mark.parametrize("bad", [dict(N=30, s=4), dict(N=32, s=0), dict(N=32, s=4, eps=-1.0),
                                 dict(N=32, s=4, lam=float("inf")), dict(N=32, s=4, strategy=7),
                                 dict(N=32, s=4, strategy=6), dict(N=32, s=4, cell_ctas=3),
                                 dict(N=32, s=4, cell_ti=2), dict(N=32, s=4, balance=-1)])
def test_init_rejects_bad_parameters_before_touching_the_device(bad):
    import numpy as np

    from paper_2410_08859_gb300 import domdec as dd
    N = bad.pop("N")
    s = bad.pop("s")
    kw = dict(eps=1e-3, lam=1.0)
    kw.update(bad)
    p = dd.domdec_default_params(basic_cell=s, **kw)
    mu = np.ones(N * N)
    with pytest.raises(dd.DomDecError) as e:
        dd.domdec_init(mu, mu, N, p, stream=0)
    assert e.value.code == dd.DOMDEC_EINVAL
