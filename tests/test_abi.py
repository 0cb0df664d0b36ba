"""The C-ABI library loads and exports every function include/ys.h declares;
argument validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ys_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02300_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared("ys.h")
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_validation_without_gpu():
    from paper_1905_02300_gb300 import ys
    bad = [dict(R1=0.0, R2=1.0), dict(R1=1.0, R2=0.5), dict(dt=0.0), dict(Nr=4), dict(Nph=10, Nth=16),
           dict(chi=0.0), dict(Nth=13, Nph=13, Nr=8)]   # last: too coarse for the exchange
    for b in bad:
        kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=1e-3, Nr=16, Nth=16, Nph=48)
        kw.update(b)
        with pytest.raises(ys.YSError) as e:
            ys.Solver(**kw)
        assert e.value.code == ys.YS_EINVAL, (b, e.value)


def test_strerror_and_defaults():
    from paper_1905_02300_gb300 import ys
    assert ys.lib.ys_strerror(ys.YS_EDIVERGED) == b"diverged (NaN/Inf)"
    p = ys.default_params()
    assert p.chi == 1.0 and p.overlap == 2 and p.step7 == 1 and p.precision == ys.YS_FP64
