"""The manufactured solution of Sec. 5.1 on the CUDA path: u = cos t (2x^2yz,
-xy^2z, -xyz^2), p = cos t xyz, T = 2 cos t x^2yz, R1 = 1, R2 = 2,
Ra = Pr = 1, with its non-zero velocity and temperature on both walls
following cos t (ys_set_wall_data) and the forcing of the continuous
equations.

Parity against the FP64 oracle (same inputs, same wall data), element by
element: FP64 within 1e-11 after 10 steps, the mixed form within 1e-5 (a
velocity component against the vector's scale); and second-order space
convergence against the exact solution on grids the oracle would take
minutes for.
"""
import math

import numpy as np
import pytest

from oracle.scheme import Oracle, Params
from paper_1905_02300_gb300 import workloads as W
from tests.test_gpu_mixed import rel_errs as scaled_errs

pytestmark = pytest.mark.gpu

FIELDS = ("T", "ur", "uth", "uph", "p", "ur1", "uth1", "uph1", "p1")
LOCS = {"T": "c", "p": "c", "ur": "r", "uth": "t", "uph": "p"}


def paper_pair(ys, N, dt, precision=None, tol=0.0, with_oracle=True):
    spec = W.Spec(1.0, 2.0, N, N, 3 * N)
    ex = W.PaperShell(1.0, 2.0, 1.0, 1.0)
    f0, fm = W.sample_fields(ex, spec, 0.0), W.sample_fields(ex, spec, -dt)
    modes = W.forcing_modes(ex, spec)
    walls = dict(W.wall_velocity(ex, spec, 0.0), T=W.wall_temperature(ex, spec, 0.0))   # times cos t
    o = None
    if with_oracle:
        o = Oracle(Params(R1=1.0, R2=2.0, Pr=1.0, Ra=1.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, schwarz_tol=tol,
                          wall_mode=(ex.time_fn, walls)))
        for lvl, f in ((0, f0), (1, fm)):
            o.set_fields(lvl, f["T"], f["ur"], f["uth"], f["uph"], f["p"])
        for tid, F in modes:
            o.set_forcing(tid, F["T"], F["ur"], F["uth"], F["uph"])
    kw = dict(R1=1.0, R2=2.0, Pr=1.0, Ra=1.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, schwarz_tol=tol)
    if precision is not None:
        kw["precision"] = precision
    s = ys.Solver(**kw)
    s.set_wall_data(ex.time_fn, walls)
    for lvl, f in ((0, f0), (1, fm)):
        s.set_fields_dict(lvl, f)
    for m, (tid, F) in enumerate(modes):
        s.set_forcing(m, tid, F["T"], F["ur"], F["uth"], F["uph"])
    return o, s, spec, ex


def test_paper_mms_fp64_and_mixed_parity_after_10_steps(gpu_lib):
    ys = gpu_lib
    o, s, _, _ = paper_pair(ys, 16, 1e-3)
    _, sm, _, _ = paper_pair(ys, 16, 1e-3, precision=ys.YS_MIXED, with_oracle=False)
    o.step(10, 3)
    s.step(10, 3)
    sm.step(10, 3)
    ref = o.get_fields(0, aux=True)
    g = s.get_fields(0, aux=True)
    e = {k: np.abs(g[k] - ref[k]).max() / max(np.abs(ref[k]).max(), 1e-300) for k in FIELDS}
    assert max(e.values()) <= 1e-11, e
    em = scaled_errs(sm.get_fields(0, aux=True), ref)
    print(e, em)
    assert max(em.values()) <= 1e-5, em


def test_paper_mms_wall_data_follows_cos_t(gpu_lib):
    """The wall faces of u_r hold cos(t) times the wall data at every stored
    level: at t = 0 after set-up, and at t = 5 dt after 5 steps."""
    ys = gpu_lib
    o, s, spec, ex = paper_pair(ys, 12, 1e-3, with_oracle=False)
    for t in (0.0, None):
        if t is None:
            s.step(5, 3)
            t = s.stats()["t"]
        g = s.get_fields(0)
        w = W.wall_velocity(ex, spec, t)
        assert np.abs(g["ur"][:, 0] - w["ur"][0]).max() <= 1e-13 * np.abs(w["ur"]).max()
        assert np.abs(g["ur"][:, -1] - w["ur"][1]).max() <= 1e-13 * np.abs(w["ur"]).max()


def test_paper_mms_space_convergence_second_order(gpu_lib):
    """Second order in space at 24 -> 48 cells (dt = 2e-3 to t = 0.04, Schwarz
    to 1e-9): the near-wall error of a cell-centred Dirichlet condition needs
    t >> h^2 to settle at its O(h^2) profile, so the run is not shorter.  T
    and the velocity converge at second order (measured 1.94 to 2.02).  The
    pressure error also carries the artificial-compressibility transient that
    the O(h^2) discrete divergence of the sampled initial velocity starts (the
    oscillations Sec. 5.1 attributes to the AC algorithm); at this dt and t it
    falls by 2.2 from 24 to 48 cells (order 1.1), at dt = 1e-3 by 4.3, so the
    test asks of it only that it fall by more than 2."""
    ys = gpu_lib
    errs = []
    for N in (24, 48):
        _, s, spec, ex = paper_pair(ys, N, 2e-3, tol=1e-9, with_oracle=False)
        s.step(20, 200)
        g = s.get_fields(0)
        exact = W.sample_fields(ex, spec, s.stats()["t"])
        e = {}
        for k, loc in LOCS.items():
            r, th, _ = spec.coords(loc)
            w = np.broadcast_to(r * r * np.sin(th), g[k].shape)
            d = g[k] - exact[k]
            e[k] = math.sqrt(np.sum(w * d * d) / np.sum(w))
        errs.append(e)
    print(errs)
    for k in ("T", "ur", "uth", "uph"):
        assert math.log2(errs[0][k] / errs[1][k]) > 1.8, (k, errs)
    assert errs[0]["p"] / errs[1]["p"] > 2.0, errs
