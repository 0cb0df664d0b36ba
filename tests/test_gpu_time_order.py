"""Second order in time on the GPU (the time study of the 32 x 32 x 96 shell).

The discrete manufactured solution of tests/discrete_mms.py (exact for the
spatially discrete problem, so every error is a time error) on the
32 x 32 x 96-per-patch shell, R1 = 0.5, R2 = 1, Pr = 1, Ra = 1e3, dt halved
from 4e-3 to 5e-4 to t = 0.08 (20, 40, 80, 160 steps), Schwarz iterated to
1e-12, FP64, through the C ABI.  The errors against the exact grid functions
fall by 4 per halving for T, u_2 and p_2 (its mean over the support removed:
the constant pressure level of the overset grid drifts at O(dt) without
entering the velocity), the bootstrapped system; the first system u_1 falls
by 2 to 4 at these short times (its O(dt) part, chi dt d_t p, grows from 0
since d_t p vanishes at t = 0, so the O(dt^2) part still weighs in).
"""
import numpy as np
import pytest

from oracle.scheme import Params
from tests.discrete_mms import DiscreteMMS

pytestmark = pytest.mark.gpu


def _errors(ys, dt, N=32, Tf=0.08):
    prm = Params(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=dt, Nr=N, Nth=N, Nph=3 * N)
    mms = DiscreteMMS(prm)
    assert mms.div_max < 1e-10 and mms.yang_max == 0.0
    s = ys.Solver(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=dt, Nr=N, Nth=N, Nph=3 * N, schwarz_tol=1e-12)
    for lvl, t in ((0, 0.0), (1, -dt)):
        s.set_fields_dict(lvl, mms.at(t))
    for m, (tid, F) in enumerate(mms.modes):
        s.set_forcing(m, tid, *F)
    for _ in range(int(round(Tf / dt))):
        s.step(1, 400)
        # converged far below the time error (at dt = 4e-3 the increments
        # stall at rounding level above the 1e-12 tolerance)
        assert s.norms()[0].max() < 1e-9
    got, U = s.get_fields(0, aux=True), mms.U
    ex = mms.at(s.stats()["t"])
    e = {k: float(np.abs(got[k] - ex[k.rstrip("1")]).max() / np.abs(U[k.rstrip("1")]).max())
         for k in ("T", "ur", "uth", "uph", "ur1", "uth1", "uph1")}
    sup = mms.support()
    d = got["p"][0] - ex["p"][0]
    e["p_dm"] = float(np.abs(d - d[sup].mean())[sup].max() / np.abs(U["p"]).max())
    s.close()
    return e


def test_c2_time_study_second_order_on_the_gpu(gpu_lib):
    dts = (4e-3, 2e-3, 1e-3, 5e-4)
    res = [_errors(gpu_lib, dt) for dt in dts]
    ratios = {k: [res[i][k] / res[i + 1][k] for i in range(len(dts) - 1)] for k in res[0]}
    print(ratios)
    for k in ("T", "ur", "uth", "uph", "p_dm"):
        assert all(3.6 < q < 4.4 for q in ratios[k]), (k, ratios[k], res)
    for k in ("ur1", "uth1", "uph1"):
        assert all(1.7 < q < 4.4 for q in ratios[k]), (k, ratios[k], res)
