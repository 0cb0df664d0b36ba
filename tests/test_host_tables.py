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


@pytest.mark.parametrize("beta", [None, 0.5])
def test_host_velocity_records_match_the_oracle_rates(beta):
    """The u_r, u_theta, u_phi records applied as the residual kernels apply
    them (two-level sums S of the three components, the 4-point sums of the
    advecting velocity, the pressure entering the row and, for u_r, the
    temperature sum) give dt times the oracle's rates (vector Laplacian,
    advection with curvature terms, -grad P, grad div / (2 chi), buoyancy) at
    every unknown, on a uniform and a stretched radial grid."""
    from oracle.grid import view
    from paper_1905_02300_gb300 import ys
    Nr, Nt, Np, dt, Pr, Ra, chi = 8, 12, 36, 0.02, 0.7, 3.0, 1.3
    rh = None if beta is None else W.stretched_radii(0.5, 1.0, Nr, beta)
    kw = dict(R1=0.5, R2=1.0, Pr=Pr, Ra=Ra, dt=dt, Nr=Nr, Nth=Nt, Nph=Np, chi=chi, r_half=rh)
    g = Grid(0.5, 1.0, Nr, Nt, Np, r_half=rh)
    rng = np.random.default_rng(11)
    Sr, St, Sp, ST, P = (rng.normal(size=g.shape) for _ in range(5))
    A = [rng.uniform(-2.0, 2.0, size=g.shape) for _ in range(3)]
    U = [0.5 * Sr, 0.5 * St, 0.5 * Sp]
    D = ops.padded(g, ops.divergence(g, U))

    def records(table, loc):
        i0, i1, j0, j1, _, _ = g.region(loc)
        c = residual_table(ys, kw, table)[i0 + 1:i1 + 1, j0 + 1:j1 + 1][None, :, :, None, :]
        return lambda m: c[..., m]

    def diff(c, v, X):
        S0 = v(X)
        return (c(0) * (v(X, 1) - S0) - c(1) * (S0 - v(X, -1)) + c(2) * (v(X, 0, 1) - S0)
                - c(3) * (S0 - v(X, 0, -1)) + c(4) * (v(X, 0, 0, 1) - 2 * S0 + v(X, 0, 0, -1)))

    def sum4(a):
        return ((a[0] + a[1]) + a[2]) + a[3]

    checks = []
    # u_r at r-faces: own S_r, S_th and S_ph around the face, T sums
    v = lambda a, di=0, dj=0, dk=0: view(a, g.region(R), di, dj, dk)
    c = records(1, R)
    y1, y0, ym1, ym0 = v(St, 0, 1), v(St), v(St, -1, 1), v(St, -1)
    z1, z0, zm1, zm0 = v(Sp, 0, 0, 1), v(Sp), v(Sp, -1, 0, 1), v(Sp, -1)
    sAt = sum4([v(A[1], -1), v(A[1], -1, 1), v(A[1]), v(A[1], 0, 1)])
    sAp = sum4([v(A[2], -1), v(A[2], -1, 0, 1), v(A[2]), v(A[2], 0, 0, 1)])
    out = (diff(c, v, Sr) + c(5) * v(Sr, 1) + c(6) * v(Sr) + c(7) * v(Sr, -1)
           + c(8) * y1 + c(9) * y0 + c(10) * ym1 + c(11) * ym0 + c(12) * (z1 - z0) + c(13) * (zm1 - zm0)
           - c(14) * v(A[0]) * (v(Sr, 1) - v(Sr, -1))
           + sAt * (c(17) * sum4([ym0, ym1, y0, y1]) - c(15) * (v(Sr, 0, 1) - v(Sr, 0, -1)))
           + sAp * (c(17) * sum4([zm0, zm1, z0, z1]) - c(16) * (v(Sr, 0, 0, 1) - v(Sr, 0, 0, -1)))
           - c(18) * (v(P) - v(P, -1)) + c(19) * (v(ST, -1) + v(ST)))
    checks.append(("ur", out, dt * ops.rate_ur(g, U, A, P, D, 0.5 * ST, 0.0, Pr, chi, Pr * Ra)))
    # u_theta at theta-faces: own S_th, S_r and S_ph around the face
    v = lambda a, di=0, dj=0, dk=0: view(a, g.region(TH), di, dj, dk)
    c = records(2, TH)
    w1, w0, wm1, wm0 = v(Sr, 1), v(Sr), v(Sr, 1, -1), v(Sr, 0, -1)
    z1, z0, zm1, zm0 = v(Sp, 0, 0, 1), v(Sp), v(Sp, 0, -1, 1), v(Sp, 0, -1)
    sAr = sum4([v(A[0], 0, -1), v(A[0], 1, -1), v(A[0]), v(A[0], 1)])
    sAp = sum4([v(A[2], 0, -1), v(A[2], 0, -1, 1), v(A[2]), v(A[2], 0, 0, 1)])
    at = v(A[1])
    out = (diff(c, v, St) + c(5) * v(St, 0, 1) + c(6) * v(St) + c(7) * v(St, 0, -1)
           + c(8) * w1 + c(9) * w0 + c(10) * wm1 + c(11) * wm0 + c(12) * (z1 - z0) + c(13) * (zm1 - zm0)
           - c(14) * sAr * (v(St, 1) - v(St, -1))
           - at * (c(15) * (v(St, 0, 1) - v(St, 0, -1)) + c(17) * sum4([wm0, wm1, w0, w1]))
           + sAp * (c(18) * sum4([zm0, zm1, z0, z1]) - c(16) * (v(St, 0, 0, 1) - v(St, 0, 0, -1)))
           - c(19) * (v(P) - v(P, 0, -1)))
    checks.append(("ut", out, dt * ops.rate_ut(g, U, A, P, D, 0.0, Pr, chi)))
    # u_phi at phi-faces: own S_ph, S_r and S_th around the face
    v = lambda a, di=0, dj=0, dk=0: view(a, g.region(PH), di, dj, dk)
    c = records(3, PH)
    w1, w0, wm1, wm0 = v(Sr, 1), v(Sr), v(Sr, 1, 0, -1), v(Sr, 0, 0, -1)
    y1, y0, ym1, ym0 = v(St, 0, 1), v(St), v(St, 0, 1, -1), v(St, 0, 0, -1)
    sAr = sum4([v(A[0], 0, 0, -1), v(A[0], 1, 0, -1), v(A[0]), v(A[0], 1)])
    sAt = sum4([v(A[1], 0, 0, -1), v(A[1], 0, 1, -1), v(A[1]), v(A[1], 0, 1)])
    ap = v(A[2])
    out = (diff(c, v, Sp) + c(5) * v(Sp) + c(6) * w1 + c(7) * w0 + c(8) * wm1 + c(9) * wm0
           + c(10) * y1 + c(11) * y0 + c(12) * ym1 + c(13) * ym0
           - c(14) * sAr * (v(Sp, 1) - v(Sp, -1)) - c(15) * sAt * (v(Sp, 0, 1) - v(Sp, 0, -1))
           - ap * (c(16) * (v(Sp, 0, 0, 1) - v(Sp, 0, 0, -1)) + c(17) * sum4([wm0, wm1, w0, w1])
                   + c(18) * sum4([ym0, ym1, y0, y1]))
           - c(19) * (v(P) - v(P, 0, 0, -1)))
    checks.append(("up", out, dt * ops.rate_up(g, U, A, P, D, 0.0, Pr, chi)))
    for name, got, ref in checks:
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= 1e-12, (name, err)


XKINDS = ("T", "ur", "uth", "uph", "p")


def exchange_table(ys, kw, kind):
    p = ys.default_params(**kw)
    n = ctypes.c_size_t(0)
    rc = ys.lib.ys_exchange_table(ctypes.byref(p), kind, None, 0, ctypes.byref(n))
    if rc != ys.YS_OK:
        return rc, None
    out = np.zeros(n.value)
    assert ys.lib.ys_exchange_table(ctypes.byref(p), kind, out.ctypes.data, n.value, ctypes.byref(n)) == ys.YS_OK
    return rc, out.reshape(-1, 12)


def same_stencil(got, ref, name):
    """Bilinear stencils (j0, k0, wj, wk) agree: the donor coordinates
    j0 + wj and k0 + wk, which fix the interpolated value, to rounding; the
    bases exactly, except where a coordinate falls on a grid line to rounding,
    where base j0 with weight 1 and base j0 + 1 with weight 0 are the same
    stencil (the floor of the two sides may break that tie either way)."""
    for a in (0, 1):
        b, w = got[:, a], got[:, 2 + a]
        rb, rw = ref[a], ref[2 + a]
        assert np.abs((b + w) - (rb + rw)).max() <= 1e-12, name
        tie = b != rb
        assert np.all(np.abs(b - rb)[tie] == 1), name
        assert np.all(np.minimum(np.abs(w[tie]), np.abs(1 - w[tie])) <= 1e-12), name
        assert tie.sum() <= 2, (name, int(tie.sum()))


@pytest.mark.parametrize("dims", [(8, 12, 36, 2), (8, 17, 41, 2), (9, 20, 60, 3), (8, 9, 27, 1)])
def test_host_exchange_tables_match_the_oracle(dims):
    """Target points, donor stencil bases (exact), bilinear weights and the
    2x2 rotation rows of the host-built Yin <-> Yang tables equal the oracle's
    ExchangeTables (Sec. 4), kind by kind, in the oracle's point order; the
    rotation rows are unit vectors (the target's tangent basis vector lies in
    the plane of the donor's mapped tangent basis at the same point)."""
    from oracle.exchange import ExchangeTables
    from paper_1905_02300_gb300 import ys
    Nr, Nt, Np, ov = dims
    kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=1e-3, Nr=Nr, Nth=Nt, Nph=Np, overlap=ov)
    ref = ExchangeTables(Grid(0.5, 1.0, Nr, Nt, Np, overlap=ov)).tab
    for kind, name in enumerate(XKINDS):
        rc, t = exchange_table(ys, kw, kind)
        assert rc == ys.YS_OK, (name, rc)
        e = ref[name]
        assert t.shape[0] == len(e["j"]), name
        np.testing.assert_array_equal(t[:, 0], e["j"])
        np.testing.assert_array_equal(t[:, 1], e["k"])
        sa, sb = (e["s"], None) if "s" in e else (e["st"], e["sp"])
        same_stencil(t[:, 2:6], sa, name)
        if sb is None:
            assert np.all(t[:, 6:10] == 0) and np.all(t[:, 10] == 1) and np.all(t[:, 11] == 0), name
        else:
            same_stencil(t[:, 6:10], sb, name)
            assert np.abs(t[:, 10] - e["rot"][0]).max() <= 1e-13, name
            assert np.abs(t[:, 11] - e["rot"][1]).max() <= 1e-13, name
            assert np.abs(np.hypot(t[:, 10], t[:, 11]) - 1.0).max() <= 1e-13, name
        assert np.all((t[:, 4:6] >= 0) & (t[:, 4:6] < 1)), name


def test_exchange_table_argument_checks():
    from paper_1905_02300_gb300 import ys
    kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=1e-3, Nr=8, Nth=12, Nph=36)
    p = ys.default_params(**kw)
    n = ctypes.c_size_t(0)
    assert ys.lib.ys_exchange_table(ctypes.byref(p), 0, None, 0, None) == ys.YS_EINVAL
    assert ys.lib.ys_exchange_table(ctypes.byref(p), 5, None, 0, ctypes.byref(n)) == ys.YS_EINVAL
    assert ys.lib.ys_exchange_table(ctypes.byref(p), -1, None, 0, ctypes.byref(n)) == ys.YS_EINVAL
    assert ys.lib.ys_exchange_table(ctypes.byref(p), 4, None, 0, ctypes.byref(n)) == ys.YS_OK
    small = np.zeros(12)
    assert ys.lib.ys_exchange_table(ctypes.byref(p), 4, small.ctypes.data, 12, ctypes.byref(n)) == ys.YS_EINVAL
