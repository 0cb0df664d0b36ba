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
