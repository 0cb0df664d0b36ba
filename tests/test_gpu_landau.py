"""Landau's jet (Sec. 5.1) on the CUDA path: Dirichlet wall velocity from the
formula, no forcing, no buoyancy, started from the exact steady state.

Parity against the FP64 oracle (same inputs, same wall data) and second-order
space convergence against the exact solution on grids the oracle would take
minutes for.
"""
import math

import numpy as np
import pytest

from oracle.scheme import Oracle, Params
from paper_1905_02300_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("T", "ur", "uth", "uph", "p", "ur1", "uth1", "uph1", "p1")
LOCS = {"p": "c", "ur": "r", "uth": "t", "uph": "p"}


def landau_pair(ys, N, dt, precision=None, tol=0.0, with_oracle=True):
    spec = W.Spec(0.5, 1.0, N, N, 3 * N)
    ex = W.LandauJet(0.5, 1.0, 1.0, 0.0)
    f = W.sample_fields(ex, spec, 0.0)
    walls = W.wall_velocity(ex, spec)
    o = None
    if with_oracle:
        o = Oracle(Params(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, schwarz_tol=tol,
                          wall_u=walls))
        for lvl in (0, 1):
            o.set_fields(lvl, f["T"], f["ur"], f["uth"], f["uph"], f["p"])
    kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, schwarz_tol=tol)
    if precision is not None:
        kw["precision"] = precision
    s = ys.Solver(**kw)
    s.set_wall_velocity(walls)
    for lvl in (0, 1):
        s.set_fields_dict(lvl, f)
    return o, s, spec, f


def rel_errs(s, o):
    g = s.get_fields(0, aux=True)
    r = o.get_fields(0, aux=True)
    return {k: np.abs(g[k] - r[k]).max() / max(np.abs(r[k]).max(), 1e-300) for k in FIELDS}


def l2(spec, loc, e):
    r, th, _ = spec.coords(loc)
    w = np.broadcast_to(r * r * np.sin(th), e.shape)
    return math.sqrt(np.sum(w * e * e) / np.sum(w))


def test_landau_fp64_parity_after_10_steps(gpu_lib):
    o, s, _, _ = landau_pair(gpu_lib, 12, 1e-4)
    o.step(10, 3)
    s.step(10, 3)
    e = rel_errs(s, o)
    assert max(e.values()) <= 1e-11, e


def test_landau_wall_data_reaches_the_stored_levels(gpu_lib):
    """After set_fields, the wall faces of u_r hold the wall velocity."""
    o, s, spec, f = landau_pair(gpu_lib, 12, 1e-4)
    g = s.get_fields(0)
    walls = W.wall_velocity(W.LandauJet(0.5, 1.0, 1.0, 0.0), spec)
    assert np.array_equal(g["ur"][:, 0], walls["ur"][0])
    assert np.array_equal(g["ur"][:, -1], walls["ur"][1])
    e = rel_errs(s, o)
    assert max(e.values()) <= 1e-14, e


def test_landau_mixed_vs_oracle(gpu_lib):
    o, s, _, _ = landau_pair(gpu_lib, 12, 1e-4, precision=gpu_lib.YS_MIXED)
    o.step(10, 3)
    s.step(10, 3)
    e = rel_errs(s, o)
    print("mixed landau errors", e)
    assert max(e.values()) <= 1e-5, e


def test_landau_space_convergence_second_order(gpu_lib):
    """Sec. 5.1: the Landau runs converge at second order in space; here
    24 -> 48 cells per direction unit (Nph = 3 N), Schwarz to tolerance."""
    errs = []
    for N in (24, 48):
        _, s, spec, f = landau_pair(gpu_lib, N, 5e-5, tol=1e-9, with_oracle=False)
        s.step(20, 40)
        g = s.get_fields(0)
        errs.append({k: l2(spec, LOCS[k], g[k] - f[k]) for k in LOCS})
    for k in errs[0]:
        order = math.log(errs[0][k] / errs[1][k]) / math.log(2.0)
        assert order > 1.8, (k, errs, order)


def test_step4_parity_and_zero_boundary_flux(gpu_lib):
    """Algorithm step 4 on both sides (oracle: conjugate gradients on J; CUDA:
    its closed-form minimiser): FP64 parity after 10 steps, and the stored
    level's boundary velocity carries no net flux through either patch's
    boundary (discrete Gauss weights)."""
    ys = gpu_lib
    N, dt = 12, 1e-4
    spec = W.Spec(0.5, 1.0, N, N, 3 * N)
    ex = W.LandauJet(0.5, 1.0, 1.0, 0.0)
    f = W.sample_fields(ex, spec, 0.0)
    walls = W.wall_velocity(ex, spec)
    o = Oracle(Params(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, wall_u=walls, step4=True))
    s = ys.Solver(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, step4=1)
    s.set_wall_velocity(walls)
    for lvl in (0, 1):
        o.set_fields(lvl, f["T"], f["ur"], f["uth"], f["uph"], f["p"])
        s.set_fields_dict(lvl, f)
    o.step(10, 3)
    s.step(10, 3)
    e = rel_errs(s, o)
    assert max(e.values()) <= 1e-11, e
    g = s.get_fields(0)
    r = 0.5 + (np.arange(N) + 0.5) * spec.hr
    thf = spec.th0 + np.arange(N + 1) * spec.hth
    thc = spec.th0 + (np.arange(N) + 0.5) * spec.hth
    for p in (0, 1):
        terms = [-r[:, None] * math.sin(thf[0]) * spec.hr * spec.hph * g["uth"][p, :, 0, :],
                 r[:, None] * math.sin(thf[N]) * spec.hr * spec.hph * g["uth"][p, :, N, :],
                 -r[:, None] * spec.hr * spec.hth * g["uph"][p, :, :, 0],
                 r[:, None] * spec.hr * spec.hth * g["uph"][p, :, :, 3 * N],
                 -0.25 * np.sin(thc)[:, None] * spec.hth * spec.hph * g["ur"][p, 0],
                 1.0 * np.sin(thc)[:, None] * spec.hth * spec.hph * g["ur"][p, N]]
        flux = sum(np.sum(t) for t in terms)
        scale = sum(np.sum(np.abs(t)) for t in terms[:4])
        # eps = 1e-8 shrinks the flux by 1 + |w|^2 / (eps |dOmega|^2) (~2e3 here)
        assert abs(flux) <= 1e-6 * scale, (p, flux, scale)
