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


def test_invalid_radial_half_points_rejected_without_gpu():
    """Non-uniform radial grids: radii that do not increase, or do not start at
    R1 / end at R2, are rejected before any device work (YS_EINVAL); a wrong
    count is caught by the binding."""
    import numpy as np
    from paper_1905_02300_gb300 import ys, workloads as W
    kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=1e-3, Nr=16, Nth=16, Nph=48)
    good = np.array(W.stretched_radii(0.5, 1.0, 16, 0.5))
    bad = [good[::-1].copy(), good + 0.01, np.concatenate([good[:5], good[5:6], good[5:-1]])]
    for b in bad:
        with pytest.raises(ys.YSError) as e:
            ys.Solver(**kw, r_half=b)
        assert e.value.code == ys.YS_EINVAL
    with pytest.raises(ValueError):
        ys.Solver(**kw, r_half=good[:-1])

