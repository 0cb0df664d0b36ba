"""The line-operator coefficient tables the library builds on the host (CPU,
no GPU): through ys_line_coefficients, the row (L0 + a LA, D0, U0 - a LA) of
(I - dt/2 Ahat_d) that the factorisation kernels form equals the oracle's line
operator (oracle.operators.factor) at every interior row, for T, u_r,
u_theta, u_phi along r, theta, phi, on a uniform and on a stretched radial
grid.  The first and last row of every line, which the kernels and the oracle
close with the wall and line-end conditions, are left out."""
import ctypes

import numpy as np
import pytest

from oracle import operators as ops
from oracle.grid import C, PH, R, TH, Grid
from paper_1905_02300_gb300 import workloads as W

LOCS = (C, R, TH, PH)


def tables(ys, kw):
    p = ys.default_params(**kw)
    n = ctypes.c_size_t(0)
    assert ys.lib.ys_line_coefficients(ctypes.byref(p), None, 0, ctypes.byref(n)) == ys.YS_OK
    out = np.zeros(n.value)
    assert ys.lib.ys_line_coefficients(ctypes.byref(p), out.ctypes.data, n.value, ctypes.byref(n)) == ys.YS_OK
    return out.reshape(4, 3, kw["Nr"] + 2, kw["Nth"] + 2, 4)


@pytest.mark.parametrize("beta", [None, 0.5])
def test_host_line_coefficients_match_the_oracle_operators(beta):
    from paper_1905_02300_gb300 import ys
    Nr, Nt, Np, dt, Pr, chi = 8, 12, 36, 0.02, 0.7, 1.3
    rh = None if beta is None else W.stretched_radii(0.5, 1.0, Nr, beta)
    kw = dict(R1=0.5, R2=1.0, Pr=Pr, Ra=0.0, dt=dt, Nr=Nr, Nth=Nt, Nph=Np, chi=chi, r_half=rh)
    tab = tables(ys, kw)
    g = Grid(0.5, 1.0, Nr, Nt, Np, r_half=rh)
    rng = np.random.default_rng(7)
    A = [rng.uniform(-2.0, 2.0, size=g.shape) for _ in range(3)]
    for li, loc in enumerate(LOCS):
        i0, i1, j0, j1, _, _ = g.region(loc)
        nu = 1.0 if loc == C else Pr
        adv = ops.advecting(g, loc, A)
        for di, d in enumerate("rtp"):
            lo, dg, up = ops.factor(g, loc, d, A, dt, nu, chi)
            rec = tab[li, di, i0 + 1:i1 + 1, j0 + 1:j1 + 1][None, :, :, None, :]
            a = adv[di]
            lo_t = rec[..., 0] + a * rec[..., 3]
            dg_t = np.broadcast_to(rec[..., 1], dg.shape)
            up_t = rec[..., 2] - a * rec[..., 3]
            ax = 1 + di
            inner = [slice(None)] * 4
            inner[ax] = slice(1, -1)
            inner = tuple(inner)
            for name, got, ref in (("lo", lo_t, lo), ("di", dg_t, dg), ("up", up_t, up)):
                got, ref = np.broadcast_to(got, ref.shape)[inner], ref[inner]
                err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
                assert err <= 1e-13, (loc, d, name, err)


def test_line_coefficients_argument_checks():
    from paper_1905_02300_gb300 import ys
    kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=1e-3, Nr=8, Nth=12, Nph=36)
    p = ys.default_params(**kw)
    n = ctypes.c_size_t(0)
    assert ys.lib.ys_line_coefficients(ctypes.byref(p), None, 0, None) == ys.YS_EINVAL
    assert ys.lib.ys_line_coefficients(ctypes.byref(p), None, 0, ctypes.byref(n)) == ys.YS_OK
    small = np.zeros(8)
    assert ys.lib.ys_line_coefficients(ctypes.byref(p), small.ctypes.data, 8, ctypes.byref(n)) == ys.YS_EINVAL


def residual_table(ys, kw, table):
    p = ys.default_params(**kw)
    n, m = ctypes.c_size_t(0), ctypes.c_int(0)
    assert ys.lib.ys_residual_coefficients(ctypes.byref(p), table, None, 0, ctypes.byref(n), ctypes.byref(m)) == 0
    out = np.zeros(n.value)
    assert ys.lib.ys_residual_coefficients(ctypes.byref(p), table, out.ctypes.data, n.value, ctypes.byref(n),
                                           ctypes.byref(m)) == 0
    return out.reshape(kw["Nr"] + 2, kw["Nth"] + 2, m.value)


@pytest.mark.parametrize("beta", [None, 0.5])
def test_host_residual_records_match_the_oracle_operators(beta):
    """The temperature and divergence records (Sec. 3.3), applied as the
    kernels apply them to the two-level sums S, give dt Rate_T(S/2) and
    div(S/2)/chi of the oracle at every cell, and the divergence record's norm
    weight is the oracle's midpoint-rule weight, on a uniform and a stretched
    radial grid."""
    from oracle.grid import view
    from paper_1905_02300_gb300 import ys
    Nr, Nt, Np, dt, Pr, chi = 8, 12, 36, 0.02, 0.7, 1.3
    rh = None if beta is None else W.stretched_radii(0.5, 1.0, Nr, beta)
    kw = dict(R1=0.5, R2=1.0, Pr=Pr, Ra=0.0, dt=dt, Nr=Nr, Nth=Nt, Nph=Np, chi=chi, r_half=rh)
    g = Grid(0.5, 1.0, Nr, Nt, Np, r_half=rh)
    rng = np.random.default_rng(9)
    S = rng.normal(size=g.shape)
    A = [rng.uniform(-2.0, 2.0, size=g.shape) for _ in range(3)]
    reg = g.region(C)
    i0, i1, j0, j1, _, _ = reg
    # temperature: diffusion minus advection with the 2-point sums of a
    c = residual_table(ys, kw, 0)[i0 + 1:i1 + 1, j0 + 1:j1 + 1][None, :, :, None, :]
    v = lambda a, di=0, dj=0, dk=0: view(a, reg, di, dj, dk)
    S0 = v(S)
    diff = (c[..., 0] * (v(S, 1) - S0) - c[..., 1] * (S0 - v(S, -1)) + c[..., 2] * (v(S, 0, 1) - S0)
            - c[..., 3] * (S0 - v(S, 0, -1)) + c[..., 4] * (v(S, 0, 0, 1) - 2 * S0 + v(S, 0, 0, -1)))
    sAr, sAt, sAp = v(A[0]) + v(A[0], 1), v(A[1]) + v(A[1], 0, 1), v(A[2]) + v(A[2], 0, 0, 1)
    adv = (c[..., 5] * sAr * (v(S, 1) - v(S, -1)) + c[..., 6] * sAt * (v(S, 0, 1) - v(S, 0, -1))
           + c[..., 7] * sAp * (v(S, 0, 0, 1) - v(S, 0, 0, -1)))
    ref = dt * ops.rate_T(g, 0.5 * S, A, np.zeros_like(S0))
    assert np.abs((diff - adv) - ref).max() <= 1e-12 * np.abs(ref).max()
    # divergence over chi, and the norm weight
    U = [rng.normal(size=g.shape) for _ in range(3)]
    d = residual_table(ys, kw, 4)[i0 + 1:i1 + 1, j0 + 1:j1 + 1][None, :, :, None, :]
    D = ((d[..., 0] * v(U[0], 1) - d[..., 1] * v(U[0])) + (d[..., 2] * v(U[1], 0, 1) - d[..., 3] * v(U[1]))
         + d[..., 4] * (v(U[2], 0, 0, 1) - v(U[2])))
    ref = ops.divergence(g, [0.5 * u for u in U]) / chi
    assert np.abs(D - ref).max() <= 1e-12 * np.abs(ref).max()
    w = g.weight(C) / (g.hr * g.hth * g.hph)
    assert np.abs(np.broadcast_to(d[..., 5], w.shape) - w).max() <= 1e-13 * np.abs(w).max()
