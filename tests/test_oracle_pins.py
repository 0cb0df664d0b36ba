"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the
paper's printed coordinate maps, continuous operators computed in Cartesian
coordinates by automatic differentiation, dense LU solves, closed-form and
manufactured solutions, symmetry, and the paper's stated properties of the
iteration (fixed point, first iterate = factored scheme, stability).
"""
import math

import numpy as np
import pytest

from oracle import exchange as xch
from oracle import operators as ops
from oracle.grid import C, PH, R, TH, Grid, M, view
from oracle.linesolve import solve_factored, thomas
from oracle.scheme import Oracle, Params
from paper_1905_02300_gb300 import workloads as W
from tests.exact_padded import padded_exact


# ------------------------------------------------------------------ geometry
def yang_local_angles(x, y, z):
    """Yang-local angles of a global point, from the printed Yang map
    x = -r sin(t) cos(p), y = r cos(t), z = r sin(t) sin(p)  (Sec. 2)."""
    r = np.sqrt(x * x + y * y + z * z)
    return np.arccos(y / r), np.arctan2(z, -x)


def test_yang_map_is_yin_composed_with_M():
    rng = np.random.default_rng(0)
    th, ph = rng.uniform(0.2, 3.0, 50), rng.uniform(-3, 3, 50)
    yin = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
    yang = np.stack([-np.sin(th) * np.cos(ph), np.cos(th), np.sin(th) * np.sin(ph)], -1)
    assert np.allclose(yin @ M.T, yang, atol=1e-15)
    assert np.allclose(M @ M, np.eye(3)) and abs(np.linalg.det(M) - 1) < 1e-15
    # round trip through the printed inverse
    t2, p2 = yang_local_angles(*yang.T)
    assert np.allclose(t2, th) and np.allclose(np.cos(p2 - ph), 1.0)


def test_nominal_regions_cover_the_sphere():
    rng = np.random.default_rng(1)
    v = rng.normal(size=(20000, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    def nominal(th, ph):
        return (th >= np.pi / 4) & (th <= 3 * np.pi / 4) & (np.abs(ph) <= 0.75 * np.pi)
    in_yin = nominal(np.arccos(v[:, 2]), np.arctan2(v[:, 1], v[:, 0]))
    in_yang = nominal(*yang_local_angles(*v.T))
    assert (in_yin | in_yang).all()


def test_exchange_tables_valid_and_too_coarse_rejected():
    g = Grid(0.5, 1.0, 4, 16, 48)
    xch.ExchangeTables(g)           # raises if a donor stencil leaves the interior
    with pytest.raises(ValueError):
        xch.ExchangeTables(Grid(0.5, 1.0, 4, 12, 8))


def test_rotation_orthogonal():
    g = Grid(0.5, 1.0, 4, 16, 48)
    tab = xch.ExchangeTables(g).tab
    # the (e_th, e_ph) target rows at the same points form an orthogonal matrix:
    # for u_th targets, (R_tt, R_tp) is a unit row
    for kind in ("uth", "uph"):
        a, b = tab[kind]["rot"]
        assert np.allclose(a * a + b * b, 1.0, atol=1e-14)


# ------------------------------------------------------------------ interpolation
def _donor_angles_of_targets(g, patch, loc, j, k):
    th = g.th_f(j) if loc == TH else g.th_c(j)
    ph = g.ph_f(k) if loc == PH else g.ph_c(k)
    xl, yl, zl = np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)
    if patch == 0:       # target Yin: donor Yang
        return yang_local_angles(xl, yl, zl)
    # target Yang: global = printed Yang map of the local angles; donor Yin
    x, y, z = -np.sin(th) * np.cos(ph), np.cos(th), np.sin(th) * np.sin(ph)
    return np.arccos(z), np.arctan2(y, x)


def _state(g):
    z = g.zeros
    return {"T": z(), "u1": [z(), z(), z()], "u2": [z(), z(), z()]}


def test_scalar_interpolation_exact_for_bilinear_functions():
    g = Grid(0.5, 1.0, 3, 16, 48)
    tables = xch.ExchangeTables(g)
    f = lambda th, ph: 0.7 + 1.3 * th - 0.4 * ph + 0.9 * th * ph
    st = _state(g)
    jj, kk = np.arange(-1, g.Nth + 1), np.arange(-1, g.Nph + 1)
    TH_, PH_ = np.meshgrid(g.th_c(jj), g.ph_c(kk), indexing="ij")
    st["T"][:] = f(TH_, PH_)[None, None]
    xch.exchange_into(tables, st, st, (0, 1))
    e = tables.tab["T"]
    for p in (0, 1):
        tt, pp = _donor_angles_of_targets(g, p, C, e["j"], e["k"])
        got = st["T"][p][1:g.Nr + 1, e["j"] + 1, e["k"] + 1]
        assert np.abs(got - f(tt, pp)[None]).max() < 1e-13


def test_pressure_ring_exact_for_bilinear_functions_and_blind_to_the_donor_ring():
    """Algorithm step 7: the ring of outermost interior pressure cells is
    refilled from the other patch.  A pressure bilinear in the donor's local
    (theta, phi) is reproduced exactly at each ring cell's own position
    (mapped into the donor frame); the donor stencils stay off the donor's
    own ring, so garbage there does not reach the result, and both patches
    can be refilled at once; cells off the ring are left alone."""
    g = Grid(0.5, 1.0, 3, 16, 48)
    tables = xch.ExchangeTables(g)
    f = lambda th, ph: -0.3 + 0.8 * th + 0.5 * ph - 0.6 * th * ph
    jj, kk = np.arange(-1, g.Nth + 1), np.arange(-1, g.Nph + 1)
    TH_, PH_ = np.meshgrid(g.th_c(jj), g.ph_c(kk), indexing="ij")
    P = g.zeros()
    P[:] = f(TH_, PH_)[None, None]
    e = tables.tab["p"]
    ring = np.zeros((g.Nth + 2, g.Nph + 2), bool)
    ring[e["j"] + 1, e["k"] + 1] = True
    assert ring.sum() == 2 * g.Nph + 2 * g.Nth - 4
    rng = np.random.default_rng(3)
    for p in (0, 1):       # garbage on every ring cell and in the ghosts of both patches
        P[p][:, ring] = rng.uniform(-1e3, 1e3, size=P[p][:, ring].shape)
        P[p][:, 0, :] = P[p][:, -1, :] = P[p][:, :, 0] = P[p][:, :, -1] = np.nan
    inner = P[:, 1:g.Nr + 1].copy()
    xch.pressure_ring(tables, P, (0, 1))
    for p in (0, 1):
        tt, pp = _donor_angles_of_targets(g, p, C, e["j"], e["k"])
        got = P[p][1:g.Nr + 1, e["j"] + 1, e["k"] + 1]
        assert np.abs(got - f(tt, pp)[None]).max() < 1e-13
        off = ~ring
        off[0, :] = off[-1, :] = off[:, 0] = off[:, -1] = False
        np.testing.assert_array_equal(P[p][1:g.Nr + 1][:, off], inner[p][:, off])


def test_constant_scalar_exact_and_vector_field_second_order():
    errs = []
    for N in (16, 32):
        g = Grid(0.5, 1.0, 2, N, 3 * N)
        tables = xch.ExchangeTables(g)
        st = _state(g)
        st["T"][:] = 2.5
        v = np.array([0.3, -0.5, 0.7])     # constant global Cartesian vector
        # local components on each patch at each staggered location
        jj, kk = np.arange(-1, g.Nth + 1), np.arange(-1, g.Nph + 1)
        for comp, loc in ((0, R), (1, TH), (2, PH)):
            th = g.th_f(jj) if loc == TH else g.th_c(jj)
            ph = g.ph_f(kk) if loc == PH else g.ph_c(kk)
            TT, PP = np.meshgrid(th, ph, indexing="ij")
            basis = [np.stack([np.sin(TT) * np.cos(PP), np.sin(TT) * np.sin(PP), np.cos(TT)], -1),
                     np.stack([np.cos(TT) * np.cos(PP), np.cos(TT) * np.sin(PP), -np.sin(TT)], -1),
                     np.stack([-np.sin(PP), np.cos(PP), 0 * PP], -1)][comp]
            exact = [basis @ v, basis @ (M @ v)]       # Yang local = M global
            for p in (0, 1):
                st["u1"][comp][p][:] = exact[p][None]
        ref = {c: [a.copy() for a in st["u1"][c]] for c in range(3)} if False else [a.copy() for a in st["u1"]]
        xch.exchange_into(tables, st, st, (0, 1))
        assert np.abs(st["T"][:, 1:g.Nr + 1] - 2.5).max() < 1e-14
        err = 0.0
        for kind, comp in (("ur", 0), ("uth", 1), ("uph", 2)):
            e = tables.tab[kind]
            ii = slice(2, g.Nr + 1) if comp == 0 else slice(1, g.Nr + 1)
            d = st["u1"][comp][:, ii][:, :, e["j"] + 1, e["k"] + 1] - ref[comp][:, ii][:, :, e["j"] + 1, e["k"] + 1]
            err = max(err, np.abs(d).max())
        errs.append(err)
    assert errs[0] < 5e-3 and errs[0] / errs[1] > 3.5, errs


# ------------------------------------------------------------------ line solves
def test_thomas_matches_dense_lu():
    rng = np.random.default_rng(2)
    n, lines = 17, 9
    lo = rng.uniform(-1, 1, (n, lines))
    up = rng.uniform(-1, 1, (n, lines))
    di = 2.5 + rng.uniform(0, 1, (n, lines))
    b = rng.normal(size=(n, lines))
    x = thomas(lo, di, up, b, 0)
    for l in range(lines):
        A = np.diag(di[:, l]) + np.diag(lo[1:, l], -1) + np.diag(up[:-1, l], 1)
        assert np.abs(x[:, l] - np.linalg.solve(A, b[:, l])).max() < 1e-13


def _dense_of(op, shape):
    n = int(np.prod(shape))
    Mx = np.empty((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        Mx[:, i] = op(e.reshape(shape)).ravel()
    return Mx


@pytest.mark.parametrize("loc", [C, R, TH, PH])
def test_factored_solve_matches_dense_product(loc):
    """Three sweeps in the stated order invert the product of the factors
    (each factor applied as a matrix-vector product, assembled densely)."""
    g = Grid(0.5, 1.0, 4, 12, 14)
    rng = np.random.default_rng(3)
    A = [rng.uniform(-1, 1, g.shape) for _ in range(3)]
    fac = {d: ops.factor(g, loc, d, A, 0.01, 1.0, 1.0) for d in "rtp"}
    shape = view(g.zeros(), g.region(loc)).shape
    order = ops.ORDER[loc]
    axes = {"r": 1, "t": 2, "p": 3}

    def Pop(x):
        y = x
        for d in reversed(order):          # P = F1 F2 F3 applied right to left
            y = ops.apply_factor(*fac[d], y, axes[d])
        return y
    b = rng.normal(size=shape)
    x = solve_factored(fac, order, b)
    Pd = _dense_of(Pop, shape)
    xd = np.linalg.solve(Pd, b.ravel()).reshape(shape)
    assert np.abs(x - xd).max() < 1e-12 * max(1.0, np.abs(xd).max())


# ------------------------------------------------------------------ operators
class GradCurlShell(W.Exact):
    """A non-solenoidal field (curl part + gradient part) with a smooth T and
    p, for operator pins: u = CurlShell u + grad(s(r)^2 x y)."""
    name = "gradcurl"

    def fields(self, x, y, z, F):
        U, P, Th = W.CurlShell(self.R1, self.R2, self.Pr, self.Ra).fields(x, y, z, F)
        r = F.sqrt(x * x + y * y + z * z)
        L = self.R2 - self.R1
        s = F.sin((r - self.R1) * (math.pi / L))
        ds = F.cos((r - self.R1) * (math.pi / L)) * (math.pi / L)
        q = s * s
        dq = 2.0 * s * ds / r
        g_ = [dq * x * x * y + q * y, dq * y * x * y + q * x, dq * z * x * y]
        return [U[m] + g_[m] for m in range(3)], P, Th


def _operator_errors(N, beta=None):
    rh = None if beta is None else W.stretched_radii(0.5, 1.0, N, beta)
    g = Grid(0.5, 1.0, N, N, 3 * N, r_half=rh)
    spec = W.Spec(0.5, 1.0, N, N, 3 * N, r_half=rh)
    ex = GradCurlShell(0.5, 1.0, 1.0, 1.0)
    aex = W.TrigShell(0.5, 1.0, 1.0, 1.0)
    t = 0.3
    F = padded_exact(g, ex, t)
    Fa = padded_exact(g, aex, t)
    U = [F["ur"], F["ut"], F["up"]]
    A = [Fa["ur"], Fa["ut"], Fa["up"]]
    Z = [g.zeros(), g.zeros(), g.zeros()]
    D = ops.padded(g, ops.divergence(g, U))
    errs = {}
    out = {}
    for loc in (C, R, TH, PH):
        out[loc] = W.exact_rates(ex, spec, {C: "c", R: "r", TH: "t", PH: "p"}[loc], t, 1.0, 1.0, 1.0, a_ex=aex)

    def user(loc, a):          # exact values at the unknowns of loc
        i0, i1, j0, j1, k0, k1 = g.region(loc)
        return a[:, i0:i1, j0:j1, k0:k1]
    zc = np.zeros(view(g.zeros(), g.region(C)).shape)
    errs["div"] = np.abs(ops.divergence(g, U) - user(C, out[C]["div"])).max()
    errs["lapT"] = np.abs(ops.rate_T(g, F["T"], Z, zc) - user(C, out[C]["lapT"])).max()
    errs["advT"] = np.abs(ops.rate_T(g, F["T"], A, zc, kappa=0.0) + user(C, out[C]["advT"])).max()
    calls = {R: lambda **kw: ops.rate_ur(g, kw["U"], kw["A"], kw["P"], kw["D"], kw["Tb"], 0.0, kw["nu"], 1.0, kw["PrRa"]),
             TH: lambda **kw: ops.rate_ut(g, kw["U"], kw["A"], kw["P"], kw["D"], 0.0, kw["nu"], 1.0),
             PH: lambda **kw: ops.rate_up(g, kw["U"], kw["A"], kw["P"], kw["D"], 0.0, kw["nu"], 1.0)}
    z = g.zeros()
    for comp, loc in ((0, R), (1, TH), (2, PH)):
        f = calls[loc]
        ex_ = out[loc]
        errs[f"vlap{comp}"] = np.abs(f(U=U, A=Z, P=z, D=z, Tb=z, nu=1.0, PrRa=0.0) - user(loc, ex_["vlap"][comp])).max()
        errs[f"adv{comp}"] = np.abs(f(U=U, A=A, P=z, D=z, Tb=z, nu=0.0, PrRa=0.0) + user(loc, ex_["adv"][comp])).max()
        errs[f"gradp{comp}"] = np.abs(f(U=Z, A=Z, P=F["p"], D=z, Tb=z, nu=0.0, PrRa=0.0) + user(loc, ex_["gradp"][comp])).max()
        errs[f"graddiv{comp}"] = np.abs(f(U=Z, A=Z, P=z, D=D, Tb=z, nu=0.0, PrRa=0.0) - 0.5 * user(loc, ex_["graddiv"][comp])).max()
    errs["buoy"] = np.abs(calls[R](U=Z, A=Z, P=z, D=z, Tb=F["T"], nu=0.0, PrRa=1.0) - user(R, out[R]["buoy"][0])).max()
    return errs


def test_discrete_operators_converge_to_continuous_at_second_order():
    e1, e2 = _operator_errors(12), _operator_errors(24)
    for k in e1:
        ratio = e1[k] / max(e2[k], 1e-300)
        assert ratio > 3.3, (k, e1[k], e2[k], ratio)


def test_stretched_radial_grid_operators_converge_at_second_order():
    """Sec. 4 (centred differences on a non-uniform grid): on a smoothly
    stretched radial grid (cells 3x finer at the walls than mid-shell) every
    discrete operator still converges to its continuous value at second order."""
    e1, e2 = _operator_errors(12, 0.5), _operator_errors(24, 0.5)
    for k in e1:
        ratio = e1[k] / max(e2[k], 1e-300)
        assert ratio > 3.3, (k, e1[k], e2[k], ratio)


def test_uniform_half_points_give_the_uniform_operators():
    """A radial grid given by the half points of the uniform grid is the
    uniform grid: the same rates and line factors to rounding."""
    N = 8
    rh = tuple((0.5 + 0.5 * np.arange(2 * N + 1) / (2 * N)).tolist())
    g0, g1 = Grid(0.5, 1.0, N, 12, 36), Grid(0.5, 1.0, N, 12, 36, r_half=rh)
    rng = np.random.default_rng(3)
    X = rng.normal(size=g0.shape)
    U = [rng.normal(size=g0.shape) for _ in range(3)]
    A = [rng.normal(size=g0.shape) for _ in range(3)]
    P, D, Tb = (rng.normal(size=g0.shape) for _ in range(3))
    zc = np.zeros(view(g0.zeros(), g0.region(C)).shape)
    for g in (g0, g1):
        g.out = [ops.rate_T(g, X, A, zc), ops.divergence(g, U),
                 ops.rate_ur(g, U, A, P, D, Tb, 0.0, 0.7, 1.3, 2.0), ops.rate_ut(g, U, A, P, D, 0.0, 0.7, 1.3),
                 ops.rate_up(g, U, A, P, D, 0.0, 0.7, 1.3)]
        g.out += [np.stack(ops.factor(g, loc, "r", A, 0.01, 0.7, 1.3)) for loc in (C, R, TH, PH)]
        g.out.append(g.weight(R))
        g.out.append(g.weight(C))
    for a, b in zip(g0.out, g1.out):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_factors_hold_the_one_direction_terms_of_the_rates():
    """(I - dt/2 Ahat_d) y = y - dt/2 (d-part of the rate) for data varying
    along d only; theta/phi diffusion carries the modified metric
    r^2/R1^2 and r^2 sin^2(theta)/(R1^2 sin^2 theta_1) (Sec. 3.2)."""
    for beta in (None, 0.5):
        _factor_rate_consistency(None if beta is None else W.stretched_radii(0.5, 1.0, 8, beta))


def _factor_rate_consistency(rh):
    g = Grid(0.5, 1.0, 8, 12, 36, r_half=rh)
    dt = 0.02
    rng = np.random.default_rng(5)
    ii, jj, kk = np.arange(-1, g.Nr + 1), np.arange(-1, g.Nth + 1), np.arange(-1, g.Nph + 1)
    zc = np.zeros(view(g.zeros(), g.region(C)).shape)
    Z = [g.zeros(), g.zeros(), g.zeros()]
    rC, sC = g.r_c(np.arange(g.Nr))[None, :, None, None], np.sin(g.th_c(np.arange(g.Nth)))[None, None, :, None]
    for d, ax, coord in (("r", 1, ii), ("t", 2, jj), ("p", 3, kk)):
        shp = [1, 1, 1, 1]
        shp[ax] = len(coord)
        y = np.broadcast_to(np.sin(0.7 * coord + 0.3).reshape(shp), g.shape).copy()
        a = np.broadcast_to(rng.uniform(-2, 2, len(coord)).reshape(shp), g.shape).copy()
        A = [g.zeros(), g.zeros(), g.zeros()]
        A["rtp".index(d)] = a
        diff = ops.rate_T(g, y, Z, zc)
        adv = ops.rate_T(g, y, A, zc, kappa=0.0)
        scale = {"r": 1.0, "t": rC ** 2 / g.R1 ** 2,
                 "p": rC ** 2 * sC ** 2 / (g.R1 ** 2 * np.sin(g.theta1) ** 2)}[d]
        expect = view(y, g.region(C)) - 0.5 * dt * (scale * diff + adv)
        lo, di, up = ops.factor(g, C, d, A, dt, 1.0, 1.0)
        got = ops.apply_factor(lo, di, up, view(y, g.region(C)), ax)
        inner = [slice(None)] * 4
        inner[ax] = slice(1, -1)
        assert np.abs(got - expect)[tuple(inner)].max() < 1e-12
    # u_r along r: every own-direction term (diffusion, curvature, grad-div, advection)
    y = np.broadcast_to(np.sin(1.3 * ii + 0.2).reshape(1, -1, 1, 1), g.shape).copy()
    a = np.broadcast_to(rng.uniform(-2, 2, len(ii)).reshape(1, -1, 1, 1), g.shape).copy()
    A = [a, g.zeros(), g.zeros()]
    U = [y, g.zeros(), g.zeros()]
    D = ops.padded(g, ops.divergence(g, U))
    rate = ops.rate_ur(g, U, A, g.zeros(), D, g.zeros(), 0.0, 0.7, 1.3, 0.0)
    lo, di, up = ops.factor(g, R, "r", A, dt, 0.7, 1.3)
    got = ops.apply_factor(lo, di, up, view(y, g.region(R)), 1)
    assert np.abs(got - (view(y, g.region(R)) - 0.5 * dt * rate))[:, 1:-1].max() < 1e-11


# ------------------------------------------------------------------ the iteration
def _random_state(o, rng):
    g = o.g
    for L in o.lev:
        L.T = rng.normal(size=g.shape)
        L.u1 = [rng.normal(size=g.shape) for _ in range(3)]
        L.u2 = [rng.normal(size=g.shape) for _ in range(3)]
        L.p1 = rng.normal(size=g.shape)
        L.p2 = rng.normal(size=g.shape)


def test_fixed_point_is_the_crank_nicolson_ac_system():
    """With frozen boundary values, the defect-correction iteration (Eq. er,
    read as P(psi^k - psi^{k-1}) = -F(psi^{k-1})) converges to the solution of
    the coupled Crank-Nicolson AC system for T, u1, p1, u2, p2, obtained here
    by a dense solve."""
    prm = Params(R1=1.0, R2=2.0, Pr=0.8, Ra=3.0, dt=0.01, Nr=3, Nth=9, Nph=6, chi=1.0, step7=False)
    o = Oracle(prm, exchange=False)
    g = o.g
    rng = np.random.default_rng(7)
    _random_state(o, rng)
    n, nm1 = o.lev
    A = [0.1 * (1.5 * n.u2[m] - 0.5 * nm1.u2[m]) for m in range(3)]
    f = o.forcing(0.0)
    f = {k: rng.normal(size=v.shape) for k, v in f.items()}
    it = n.copy()
    it.T = it.T + 0.1 * rng.normal(size=g.shape)
    regs = [("T", None, C), ("u1", 0, R), ("u1", 1, TH), ("u1", 2, PH), ("p1", None, C),
            ("u2", 0, R), ("u2", 1, TH), ("u2", 2, PH), ("p2", None, C)]

    def get(L, key, comp):
        return getattr(L, key) if comp is None else getattr(L, key)[comp]

    def pack(L):
        return np.concatenate([view(get(L, k, c), g.region(loc)).ravel() for k, c, loc in regs])

    def unpack(L, v):
        o_ = 0
        for k, c, loc in regs:
            blk = view(get(L, k, c), g.region(loc))
            blk[...] = v[o_:o_ + blk.size].reshape(blk.shape)
            o_ += blk.size

    def residual(v):
        L = it.copy()
        unpack(L, v)
        dt, chi, nu = prm.dt, prm.chi, prm.Pr
        out = []
        Th = 0.5 * (L.T + n.T)
        out.append(view(L.T, g.region(C)) - view(n.T, g.region(C)) - dt * ops.rate_T(g, Th, A, f["T"]))
        for s in (1, 2):
            U, Un = (L.u1, n.u1) if s == 1 else (L.u2, n.u2)
            P = n.p1 if s == 1 else n.p2 + 0.5 * (L.p1 - n.p1)
            Uh = [0.5 * (U[m] + Un[m]) for m in range(3)]
            D = ops.padded(g, ops.divergence(g, Uh))
            rr = ops.rate_ur(g, Uh, A, P, D, Th, f["ur"], nu, chi, prm.Pr * prm.Ra)
            rt = ops.rate_ut(g, Uh, A, P, D, f["uth"], nu, chi)
            rp = ops.rate_up(g, Uh, A, P, D, f["uph"], nu, chi)
            for comp, loc, rate in ((0, R, rr), (1, TH, rt), (2, PH, rp)):
                out.append(view(U[comp], g.region(loc)) - view(Un[comp], g.region(loc)) - dt * rate)
            div = ops.divergence(g, Uh)
            if s == 1:
                out.append(view(L.p1, g.region(C)) - view(n.p1, g.region(C)) + div / chi)
            else:
                out.append(view(L.p2, g.region(C)) - view(n.p2, g.region(C))
                           - (view(L.p1, g.region(C)) - view(n.p1, g.region(C))) + div / chi)
        return np.concatenate([a.ravel() for a in out])

    v0 = pack(it)
    G0 = residual(np.zeros_like(v0))
    J = np.empty((v0.size, v0.size))
    for i in range(v0.size):
        e = np.zeros_like(v0)
        e[i] = 1.0
        J[:, i] = residual(e) - G0
    vstar = np.linalg.solve(J, -G0)
    fac = o._factors(A)
    for _ in range(150):
        o._iterate(it, n, A, f, fac, (0, 1))
    got = pack(it)
    assert np.abs(got - vstar).max() < 1e-10 * max(1.0, np.abs(vstar).max())


def _heat_first_iterate_gap(dt):
    prm = Params(R1=1.0, R2=2.0, Pr=1.0, Ra=0.0, dt=dt, Nr=6, Nth=12, Nph=14, step7=False)
    o = Oracle(prm, exchange=False)
    g = o.g
    ii, jj, kk = np.meshgrid(np.arange(-1, g.Nr + 1), np.arange(-1, g.Nth + 1), np.arange(-1, g.Nph + 1), indexing="ij")
    base = np.sin(0.5 * ii + 0.3) * np.cos(0.4 * jj) * np.sin(0.3 * kk + 0.1)
    base = np.stack([base, 0.5 * base])
    Tn, Tnm1 = base * 1.0, base * (1.0 + 0.7 * dt)
    z = g.zeros
    for L, T in zip(o.lev, (Tn, Tnm1)):
        L.T = T.copy()
        L.u1, L.u2 = [z(), z(), z()], [z(), z(), z()]
        L.p1, L.p2 = z(), z()
    n, nm1 = o.lev
    A = [z(), z(), z()]
    f = o.forcing(0.0)
    fac = o._factors(A)
    it = n.copy()
    it.T = 2 * n.T - nm1.T
    o._iterate(it, n, A, f, fac, (0, 1))
    # literal Eq. HeatDouglas: P dT/dt = lap T* - 1/2 lap_hat (T^n - T^{n-1})
    reg = g.region(C)
    zc = np.zeros(view(z(), reg).shape)
    Tstar = 1.5 * n.T - 0.5 * nm1.T
    dTn = view(n.T - nm1.T, reg)
    lap_hat = sum(-(2.0 / dt) * (ops.apply_factor(*fac[C][d], dTn, ax) - dTn) for d, ax in (("r", 1), ("t", 2), ("p", 3)))
    rhs = ops.rate_T(g, Tstar, A, zc) - 0.5 * lap_hat
    T_douglas = view(n.T, reg) + dt * solve_factored(fac[C], "rtp", rhs)
    return np.abs(view(it.T, reg) - T_douglas).max()


def test_first_iterate_is_the_factored_douglas_scheme_to_third_order():
    e1, e2 = _heat_first_iterate_gap(2e-3), _heat_first_iterate_gap(1e-3)
    assert 6.0 < e1 / e2 < 10.0, (e1, e2)


def test_heat_first_iterate_stable_for_large_dt():
    """Sec. 3.2 theorem: the factored heat scheme is unconditionally stable.
    Sanity check at dt = 10 >> h^2, one iterate per step."""
    prm = Params(R1=1.0, R2=2.0, Pr=1.0, Ra=0.0, dt=10.0, Nr=6, Nth=12, Nph=14, step7=False)
    o = Oracle(prm, exchange=False)
    rng = np.random.default_rng(9)
    g = o.g
    reg = g.region(C)
    T0 = g.zeros()
    view(T0, reg)[...] = rng.normal(size=view(T0, reg).shape)
    for L in o.lev:
        L.T = T0.copy()
    z = g.zeros
    A = [z(), z(), z()]
    norms = []
    for _ in range(30):
        n, nm1 = o.lev
        it = n.copy()
        it.T = 2 * n.T - nm1.T
        # zero Dirichlet data on the frozen boundary values
        it.T[:, :, 0] = it.T[:, :, -1] = it.T[:, :, :, 0] = it.T[:, :, :, -1] = 0.0
        it.T[:, 0] = -it.T[:, 1]
        it.T[:, -1] = -it.T[:, -2]
        o._iterate(it, n, A, o.forcing(0.0), o._factors(A), (0, 1))
        o.lev = [it, n]
        norms.append(np.abs(view(it.T, reg)).max())
    assert np.isfinite(norms).all() and max(norms) <= 1.5 * np.abs(view(T0, reg)).max()


# ------------------------------------------------------------------ convergence
def _run(kind, N, dt, nsteps, tol=1e-9, maxit=40, mode="additive", R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, beta=None):
    rh = None if beta is None else W.stretched_radii(R1, R2, N, beta)
    spec = W.Spec(R1, R2, N, N, 3 * N, r_half=rh)
    ex = W.EXACT[kind](R1, R2, Pr, Ra)
    wall_mode = None
    if kind == "paper":     # non-zero walls following the solution's cos t
        wall_mode = (ex.time_fn, dict(W.wall_velocity(ex, spec, 0.0), T=W.wall_temperature(ex, spec, 0.0)))
    prm = Params(R1=R1, R2=R2, Pr=Pr, Ra=Ra, dt=dt, Nr=N, Nth=N, Nph=3 * N, schwarz_tol=tol, schwarz_mode=mode,
                 r_half=rh, wall_mode=wall_mode)
    o = Oracle(prm)
    f0, fm = W.sample_fields(ex, spec, 0.0), W.sample_fields(ex, spec, -dt)
    o.set_fields(0, f0["T"], f0["ur"], f0["uth"], f0["uph"], f0["p"])
    o.set_fields(1, fm["T"], fm["ur"], fm["uth"], fm["uph"], fm["p"])
    if kind != "radial_heat":
        for tid, F in W.forcing_modes(ex, spec):
            o.set_forcing(tid, F["T"], F["ur"], F["uth"], F["uph"])
    o.step(nsteps, maxit)
    return o, spec, ex


def _l2(spec, loc, e):
    r, th, _ = spec.coords(loc)
    w = np.broadcast_to(r * r * np.sin(th), e.shape)
    return math.sqrt(np.sum(w * e * e) / np.sum(w))


LOCS = {"T": "c", "p": "c", "ur": "r", "uth": "t", "uph": "p"}


def _errors(o, spec, ex, ref=None):
    got = o.get_fields(0)
    exact = W.sample_fields(ex, spec, o.t) if ref is None else ref
    return {k: _l2(spec, LOCS[k], got[k] - exact[k]) for k in LOCS}


@pytest.mark.parametrize("kind", ["trig", "curl"])
def test_space_convergence_second_order(kind):
    """Sec. 5.1: second order in space on a manufactured solution (here with
    homogeneous walls; Schwarz converged to a tolerance, Eq. er on)."""
    errs = []
    for N in (12, 20):
        o, spec, ex = _run(kind, N, 5e-4, 4)
        errs.append(_errors(o, spec, ex))
    for k in errs[0]:
        if kind == "trig" and k == "ur":
            continue            # the exact u_r is zero for this solution
        order = math.log(errs[0][k] / errs[1][k]) / math.log(20 / 12)
        assert order > 1.7, (k, errs, order)


def test_paper_manufactured_solution_space_convergence_second_order():
    """Sec. 5.1's own manufactured solution u = cos t (2x^2yz, -xy^2z, -xyz^2),
    p = cos t xyz, T = 2 cos t x^2yz with its parameters R1 = 1, R2 = 2,
    Ra = Pr = 1: the velocity and temperature are non-zero on both walls and
    follow cos t there (time-dependent Dirichlet wall data at each new time
    level).  Second order in space for every field, Schwarz converged, as
    Sec. 5.1 reports: 12 -> 24 cells, dt = 2e-3 to t = 0.04.  The run is not
    shorter because the error of a cell-centred Dirichlet wall (reflection
    ghost) settles at its O(h^2) profile only after t >> h^2, and the step is
    not smaller because the artificial-compressibility pressure transient
    that the O(h^2) discrete divergence of the sampled initial velocity
    starts grows as dt shrinks."""
    errs = []
    for N in (12, 24):
        o, spec, ex = _run("paper", N, 2e-3, 20, R1=1.0, R2=2.0, Ra=1.0)
        errs.append(_errors(o, spec, ex))
    for k in errs[0]:
        order = math.log(errs[0][k] / errs[1][k]) / math.log(2.0)
        assert order > 1.8, (k, errs, order)


def test_stretched_radial_grid_space_convergence_second_order():
    """The whole scheme on a smoothly stretched radial grid (cells 3x finer at
    the walls than mid-shell): second order in space on the manufactured
    solution, as on the uniform grid."""
    errs = []
    for N in (12, 20):
        o, spec, ex = _run("trig", N, 5e-4, 4, beta=0.5)
        errs.append(_errors(o, spec, ex))
    for k in errs[0]:
        if k == "ur":
            continue            # the exact u_r is zero for this solution
        order = math.log(errs[0][k] / errs[1][k]) / math.log(20 / 12)
        assert order > 1.7, (k, errs, order)


def test_stretched_radial_heat_closed_form_second_order():
    """The radial heat closed form on the stretched grid: second order."""
    errs = []
    for N, dt in ((10, 2e-3), (20, 5e-4)):
        o, spec, ex = _run("radial_heat", N, dt, int(round(0.008 / dt)), Pr=1.0, Ra=0.0, beta=0.5)
        errs.append(_errors(o, spec, ex)["T"])
    assert math.log(errs[0] / errs[1]) / math.log(2.0) > 1.7, errs


def test_radial_heat_closed_form_second_order():
    """T = sin(pi (r - R1)/L)/r exp(-(pi/L)^2 t) solves the heat equation with
    homogeneous walls; both patches and the exchange are exercised."""
    errs = []
    for N, dt in ((12, 2e-3), (24, 5e-4)):
        o, spec, ex = _run("radial_heat", N, dt, int(round(0.008 / dt)), Pr=1.0, Ra=0.0)
        errs.append(_errors(o, spec, ex)["T"])
    assert math.log(errs[0] / errs[1]) / math.log(2.0) > 1.7, errs


def test_time_convergence_second_order():
    """Sec. 5.1: second order in time at a fixed grid, errors against the dt/4
    solution on the same grid (ratio 5 for a second-order method, 3 for first
    order).  Closed-form heat problem: no artificial-compressibility pressure
    transient, whose phase depends on dt and would mask the O(dt^2) error at
    the short final times a CPU test can afford."""
    N, Tf = 12, 0.016
    sols = {}
    for dt in (4e-3, 2e-3, 1e-3):
        o, spec, ex = _run("radial_heat", N, dt, int(round(Tf / dt)), tol=1e-12, maxit=80, Ra=0.0)
        sols[dt] = o.get_fields(0)["T"]
    e1 = _l2(spec, "c", sols[4e-3] - sols[1e-3])
    e2 = _l2(spec, "c", sols[2e-3] - sols[1e-3])
    assert 4.0 < e1 / e2 < 6.0, (e1, e2)


def _time_study_run(args):
    """One run of the discrete manufactured solution (tests/discrete_mms.py)
    to time Tf with Schwarz iterated to 1e-12: the errors against the exact
    grid functions (max-norm over both patches, relative to the field's
    scale), the pressures' errors with their mean over the support removed,
    and the largest discrete divergence of each velocity system."""
    dt, Tf, N = args
    from tests.discrete_mms import DiscreteMMS
    prm = Params(R1=1.0, R2=2.0, Pr=1.0, Ra=1.0, dt=dt, Nr=N[0], Nth=N[1], Nph=N[2], schwarz_tol=1e-12)
    mms = DiscreteMMS(prm)
    o = Oracle(prm)
    for lvl, t in ((0, 0.0), (1, -dt)):
        f = mms.at(t)
        o.set_fields(lvl, f["T"], f["ur"], f["uth"], f["uph"], f["p"])
    for tid, F in mms.modes:
        o.set_forcing(tid, *F)
    o.step(int(round(Tf / dt)), 200)
    got, ex, U = o.get_fields(0, aux=True), mms.at(o.t), mms.U
    out = {k: float(np.abs(got[k] - ex[k.rstrip("1")]).max() / np.abs(U[k.rstrip("1")]).max())
           for k in ("T", "ur", "uth", "uph", "ur1", "uth1", "uph1")}
    sup = mms.support()
    for k in ("p", "p1"):
        e = got[k][0] - ex["p"][0]
        out[k + "_dm"] = float(np.abs(e - e[sup].mean())[sup].max() / np.abs(U["p"]).max())
        out[k + "_mean"] = float(abs(e[sup].mean()) / np.abs(U["p"]).max())
    n = o.lev[0]
    out["div1"] = float(np.abs(ops.divergence(o.g, n.u1)).max())
    out["div2"] = float(np.abs(ops.divergence(o.g, n.u2)).max())
    out["premise"] = (mms.div_max, mms.yang_max)
    return out


def test_bootstrapped_ac_scheme_is_second_order_in_time():
    """Sec. 3.3 / Sec. 5.1: the bootstrapped artificial-compressibility scheme
    (Eq. ac2 on top of Eq. ac1) is second order in time for u_2, p_2 and T,
    while the first system (u_1, p_1) is first order; the discrete divergence
    of u_1 is O(dt) and that of u_2 O(dt^2) at a fixed time (Sec. 3.3: the
    continuity equations carry chi dt d_t p_1 and chi dt d_t(p_2 - p_1)).

    A discrete manufactured solution (tests/discrete_mms.py) removes the
    spatial error and the pressure transient that a sampled continuous
    solution would start, so each error is the time error alone: dt = 4e-3,
    2e-3, 1e-3 to t = 0.1 on an 8 x 20 x 60 shell (R1 = 1, R2 = 2, Ra = Pr = 1
    as in Sec. 5.1), Schwarz to 1e-12.  Ratios of successive errors: about 4
    for second order, 2 for first.  The pressures are compared after removing
    their mean over the support: the overset composite grid leaves the
    pressure's constant level weakly determined, and it drifts at O(dt) in
    both systems without entering the velocity (the mean is not part of the
    pin).  Planting any of these mistakes in a copy of the oracle fails the
    ratios: P_2 = p_2^n (no 1/2 (p_1 - p_1^n)), a factor 1 instead of 1/2
    there, a p_2 update without p_1 - p_1^n, a first-order advecting velocity,
    the temperature rate off the half level."""
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import get_context
    dts = (4e-3, 2e-3, 1e-3)
    with ProcessPoolExecutor(len(dts), mp_context=get_context("spawn")) as ex:
        res = list(ex.map(_time_study_run, [(dt, 0.1, (8, 20, 60)) for dt in dts]))
    for r in res:
        div0, yang = r.pop("premise")
        assert div0 < 1e-12 and yang == 0.0, (div0, yang)     # exact solenoidal data, Yang at rest
    ratios = {k: [res[i][k] / res[i + 1][k] for i in range(len(dts) - 1)] for k in res[0]}
    for k in ("T", "ur", "uth", "uph", "p_dm", "div2"):
        assert all(3.3 < q < 4.8 for q in ratios[k]), (k, ratios[k], res)
    for k in ("ur1", "uth1", "uph1", "p1_dm", "div1"):
        assert all(1.5 < q < 2.6 for q in ratios[k]), (k, ratios[k], res)
    # the bootstrapped pressure is the more accurate one at every step size
    assert all(r["p_dm"] < r["p1_dm"] for r in res), res


def test_yin_yang_congruence_bitwise():
    """M-invariant data stays identical on both patches under additive Schwarz."""
    N = 12
    prm = Params(R1=0.5, R2=1.0, Pr=1.0, Ra=100.0, dt=1e-3, Nr=N, Nth=N, Nph=3 * N)
    o = Oracle(prm)
    spec = W.Spec(0.5, 1.0, N, N, 3 * N)
    ex = W.SymmetricShell(0.5, 1.0, 1.0, 100.0)
    f0 = W.sample_fields(ex, spec, 0.0)
    for k in f0:
        f0[k][1] = f0[k][0]
    o.set_fields(0, f0["T"], f0["ur"], f0["uth"], f0["uph"], f0["p"])
    o.step(3, 3)
    got = o.get_fields(0, aux=True)
    for k, v in got.items():
        assert np.array_equal(v[0], v[1]), k
    assert np.abs(got["uth"][0]).max() > 1e-3


def test_multiplicative_and_additive_reach_the_same_step():
    """Both Schwarz variants (Sec. 4) converge to the same time step."""
    oa, spec, ex = _run("curl", 12, 1e-3, 1, tol=1e-12, maxit=80)
    om, _, _ = _run("curl", 12, 1e-3, 1, tol=1e-12, maxit=80, mode="multiplicative")
    a, m = oa.get_fields(0), om.get_fields(0)
    for k in a:
        assert np.abs(a[k] - m[k]).max() < 1e-8 * max(1.0, np.abs(a[k]).max()), k
    assert om.iters_done <= oa.iters_done


# ------------------------------------------------------------------ Landau jet
def _landau(N, dt, nsteps, tol=1e-9, maxit=20):
    """Oracle run of Landau's jet (Sec. 5.1) from the exact steady state, with
    the exact wall velocity, no forcing and no buoyancy."""
    spec = W.Spec(0.5, 1.0, N, N, 3 * N)
    ex = W.LandauJet(0.5, 1.0, 1.0, 0.0)
    f = W.sample_fields(ex, spec, 0.0)
    prm = Params(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, schwarz_tol=tol,
                 wall_u=W.wall_velocity(ex, spec))
    o = Oracle(prm)
    for lvl in (0, 1):
        o.set_fields(lvl, f["T"], f["ur"], f["uth"], f["uph"], f["p"])
    o.step(nsteps, maxit)
    return o, spec, f


def _div_l2(spec, f):
    """l2 norm of the discrete divergence (Sec. 3.3: conservative face
    differences with r^2 and sin(theta) at the faces) of user-layout velocity."""
    r, th, _ = spec.coords("c")
    rf = spec.R1 + np.arange(spec.Nr + 1) * spec.hr
    sf = np.sin(spec.th0 + np.arange(spec.Nth + 1) * spec.hth)
    ur, ut, up = f["ur"], f["uth"], f["uph"]
    s = np.sin(th)[0]
    d = ((rf[1:, None, None] ** 2 * ur[:, 1:] - rf[:-1, None, None] ** 2 * ur[:, :-1]) / (r[0] ** 2 * spec.hr)
         + (sf[None, 1:, None] * ut[:, :, 1:] - sf[None, :-1, None] * ut[:, :, :-1]) / (r[0] * s * spec.hth)
         + (up[..., 1:] - up[..., :-1]) / (r[0] * s * spec.hph))
    return _l2(spec, "c", d)


def test_landau_jet_is_a_steady_navier_stokes_solution():
    """The Landau jet fields (stream function 2 nu r sin^2 / (A - cos), pressure
    4 nu^2 (A cos - 1) / (r^2 (A - cos)^2)) solve the steady, unforced
    Navier-Stokes equations: the continuous rate nu lap u - (u.grad)u - grad p
    (AD in Cartesian coordinates) and div u vanish at every MAC point."""
    spec = W.Spec(0.5, 1.0, 12, 12, 36)
    ex = W.LandauJet(0.5, 1.0, 1.0, 0.0)
    for loc, comp in (("r", 0), ("t", 1), ("p", 2)):
        rt = W.exact_rates(ex, spec, loc, 0.0, 1.0, 0.0, 1.0)
        terms = (rt["vlap"][comp], rt["adv"][comp], rt["gradp"][comp])
        scale = max(np.abs(t).max() for t in terms)
        res = terms[0] - terms[1] - terms[2]
        assert np.abs(res).max() <= 1e-11 * scale, (loc, np.abs(res).max(), scale)
        assert np.abs(rt["div"]).max() <= 1e-11 * scale


def test_landau_jet_space_convergence_second_order():
    """Sec. 5.1: second order in space on Landau's jet with Dirichlet wall
    velocity from the formula (both patches carry the axisymmetric jet in
    rotated local bases), Schwarz converged to a tolerance."""
    errs = []
    for N in (12, 20):
        o, spec, f = _landau(N, 1e-4, 10)
        g = o.get_fields(0)
        errs.append({k: _l2(spec, LOCS[k], g[k] - f[k]) for k in ("ur", "uth", "uph", "p")})
    for k in errs[0]:
        order = math.log(errs[0][k] / errs[1][k]) / math.log(20 / 12)
        assert order > 1.8, (k, errs, order)


def _div_cells(spec, f):
    """Discrete divergence (Sec. 3.3) of user-layout velocity at every cell."""
    r, th, _ = spec.coords("c")
    rf = spec.R1 + np.arange(spec.Nr + 1) * spec.hr
    sf = np.sin(spec.th0 + np.arange(spec.Nth + 1) * spec.hth)
    ur, ut, up = f["ur"], f["uth"], f["uph"]
    s = np.sin(th)[0]
    return ((rf[1:, None, None] ** 2 * ur[:, 1:] - rf[:-1, None, None] ** 2 * ur[:, :-1]) / (r[0] ** 2 * spec.hr)
            + (sf[None, 1:, None] * ut[:, :, 1:] - sf[None, :-1, None] * ut[:, :, :-1]) / (r[0] * s * spec.hth)
            + (up[..., 1:] - up[..., :-1]) / (r[0] * s * spec.hph))


def test_landau_jet_divergence_decays():
    """Sec. 3.3, Eq. ac1: p1^{n+1} - p1^n = -div(u1^{n+1/2}) / chi, so as the
    steady run settles (delta p -> 0) the discrete divergence of every cell
    whose pressure the AC update owns decays.  The Step-7 ring cells are
    excluded: their pressure is interpolated from the other patch, not updated
    by Eq. ac1 (with Step 7 off every cell decays)."""
    spec = W.Spec(0.5, 1.0, 10, 10, 30)
    ex = W.LandauJet(0.5, 1.0, 1.0, 0.0)
    f = W.sample_fields(ex, spec, 0.0)
    o = Oracle(Params(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=1e-3, Nr=10, Nth=10, Nph=30,
                      wall_u=W.wall_velocity(ex, spec)))
    for lvl in (0, 1):
        o.set_fields(lvl, f["T"], f["ur"], f["uth"], f["uph"], f["p"])
    first = np.abs(_div_cells(spec, o.get_fields(0))[:, :, 1:-1, 1:-1]).max()
    o.step(300, 3)
    last = np.abs(_div_cells(spec, o.get_fields(0))[:, :, 1:-1, 1:-1]).max()
    assert last < first / 20, (first, last)


def test_landau_jet_divergence_is_second_order():
    """At a fixed early time the discrete divergence of the Landau run is at
    the O(h^2) level of the sampled exact field."""
    divs = []
    for N in (12, 20):
        o, spec, _ = _landau(N, 2e-4, 20, tol=0.0, maxit=3)
        divs.append(_div_l2(spec, o.get_fields(0)))
    assert math.log(divs[0] / divs[1]) / math.log(20 / 12) > 1.7, divs


def test_step4_zeroes_the_boundary_mass_flux():
    """Algorithm step 4: after the correction the net flux of each patch's
    boundary velocity through its boundary (discrete Gauss weights) vanishes,
    and the conjugate-gradient minimiser of J equals the closed-form
    minimiser u - alpha (w.u + c) / (1 + alpha w.w) w (Sherman-Morrison)."""
    N = 12
    spec = W.Spec(0.5, 1.0, N, N, 3 * N)
    ex = W.LandauJet(0.5, 1.0, 1.0, 0.0)
    f = W.sample_fields(ex, spec, 0.0)
    walls = W.wall_velocity(ex, spec)
    prm = Params(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=1e-3, Nr=N, Nth=N, Nph=3 * N, wall_u=walls)
    o = Oracle(prm)
    o.set_fields(0, f["T"], f["ur"], f["uth"], f["uph"], f["p"])
    g = o.g
    wt0, wt1, wp0, wp1, wr0, wr1 = xch.boundary_flux_weights(g)
    d = o.lev[0].as_dict()
    U = d["u2"]

    def parts(p):
        ut, up, ur = U[1][p], U[2][p], U[0][p]
        u = np.concatenate([ut[1:N + 1, 1, 1:3 * N + 1].ravel(), ut[1:N + 1, N + 1, 1:3 * N + 1].ravel(),
                            up[1:N + 1, 1:N + 1, 1].ravel(), up[1:N + 1, 1:N + 1, 3 * N + 1].ravel()])
        w = np.concatenate([wt0.ravel(), wt1.ravel(), wp0.ravel(), wp1.ravel()])
        c = np.sum(wr0 * ur[1, 1:N + 1, 1:3 * N + 1]) + np.sum(wr1 * ur[N + 1, 1:N + 1, 1:3 * N + 1])
        return u, w, c

    eps = 1e-8
    for p in (0, 1):
        u0, w, c = parts(p)
        assert abs(np.dot(w, u0) + c) > 1e-8       # interpolation leaves a flux to correct
        area = np.sum(np.abs(w)) + np.sum(np.abs(wr0)) + np.sum(np.abs(wr1))
        alpha = 1.0 / (eps * area * area)
        closed = u0 - alpha * (np.dot(w, u0) + c) / (1.0 + alpha * np.dot(w, w)) * w
        xch.mass_flux_correction(g, U, p, eps, 1e-13)
        u1, _, _ = parts(p)
        assert np.abs(u1 - closed).max() <= 1e-10 * np.abs(u0).max()
        assert abs(np.dot(w, u1) + c) <= 1e-6 * np.sum(np.abs(w * u0))


@pytest.mark.parametrize("ab", [(0.0, 1.0), (1.0, 0.5)])
def test_radial_heat_neumann_and_robin_walls_second_order(ab):
    """Sec. 1 (Neumann and Robin walls): T = sin(k (r - R1))/r exp(-k^2 t) with
    T = 0 at R1 and a T + b dT/dn = 0 at R2 (k the first root of the wall
    condition) converges at second order in space and time together."""
    a, b = ab
    errs = []
    for N, dt in ((12, 2e-3), (24, 5e-4)):
        spec = W.Spec(0.5, 1.0, N, N, 3 * N)
        ex = W.RadialHeatRobin(0.5, 1.0, 1.0, 0.0, a=a, b=b)
        o = Oracle(Params(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, Tbc_out=(a, b),
                          schwarz_tol=1e-8))
        f0, fm = W.sample_fields(ex, spec, 0.0), W.sample_fields(ex, spec, -dt)
        o.set_fields(0, f0["T"], f0["ur"], f0["uth"], f0["uph"], f0["p"])
        o.set_fields(1, fm["T"], fm["ur"], fm["uth"], fm["uph"], fm["p"])
        o.step(int(round(0.008 / dt)), 20)
        errs.append(_l2(spec, "c", o.get_fields(0)["T"] - W.sample_fields(ex, spec, o.t)["T"]))
    assert math.log(errs[0] / errs[1]) / math.log(2.0) > 1.8, errs


def test_robin_ghost_reduces_to_dirichlet_and_neumann():
    """The wall-condition ghost: Dirichlet (1, 0) gives 2 g - x0, Neumann (0, 1)
    gives x0 + h g (dT/dn = g)."""
    h = 0.03
    gam, dl = xch.robin_ghost(1.0, 0.0, h)
    assert gam == -1.0 and dl == 2.0
    gam, dl = xch.robin_ghost(0.0, 1.0, h)
    assert gam == pytest.approx(1.0) and dl == pytest.approx(h)


def test_printed_landau_grid_sizes_fix_the_patch_extents():
    """Sec. 2's patch extents are garbled; the reading taken (theta in
    [pi/4 - d, 3pi/4 + d], phi in [-3pi/4 - d, 3pi/4 + d], d the overlap angle)
    reproduces the grid sizes Sec. 5.1 prints for its Landau runs (R1 = 1,
    R2 = 2, d = 0.1) to every printed digit with whole cell counts (36, 104,
    136); the extents without the overlap, or with it on one side only, give
    no whole counts.  The oracle's grid has these extents."""
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "landau_grid_sizes.txt")):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            vals[k] = [float(x) for x in v]
    R1, R2, d = vals["R1"][0], vals["R2"][0], vals["overlap"][0]
    h_r, h_t, h_p = vals["h"]
    ext = {"r": R2 - R1, "t": math.pi / 2 + 2 * d, "p": 1.5 * math.pi + 2 * d}
    counts = {}
    for key, h in (("r", h_r), ("t", h_t), ("p", h_p)):
        n = round(ext[key] / h)
        assert abs(ext[key] / n - h) <= 5e-5 * h, (key, n, ext[key] / n, h)
        counts[key] = n
    assert counts == {"r": 36, "t": 104, "p": 136}
    # alternative readings of the theta extent give no whole count
    for alt in (math.pi / 2, math.pi / 2 + d):
        n = round(alt / h_t)
        assert abs(alt / n - h_t) > 5e-5 * h_t
    # the oracle's grid: theta and phi extents are pi/2 + 2 delta and 3 pi/2 + 2 delta
    g = Grid(1.0, 2.0, 36, 104, 136, overlap=6)
    assert abs(g.Nth * g.hth - (math.pi / 2 + 2 * g.delta)) < 1e-13
    assert abs(g.Nph * g.hph - (1.5 * math.pi + 2 * g.delta)) < 1e-13
    assert abs(g.th0 - (math.pi / 4 - g.delta)) < 1e-15 and abs(g.ph0 + 0.75 * math.pi + g.delta) < 1e-15


def test_stretched_radial_grid_robin_wall_second_order():
    """A Robin temperature wall (a, b) = (1, 0.5) at R2 on the stretched radial
    grid: its ghost uses the wall's own centre distance h_f, and the closed-form
    heat solution still converges at second order."""
    errs = []
    for N, dt in ((10, 2e-3), (20, 5e-4)):
        rh = W.stretched_radii(0.5, 1.0, N, 0.5)
        spec = W.Spec(0.5, 1.0, N, N, 3 * N, r_half=rh)
        ex = W.RadialHeatRobin(0.5, 1.0, 1.0, 0.0, a=1.0, b=0.5)
        o = Oracle(Params(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, Tbc_out=(1.0, 0.5),
                          schwarz_tol=1e-8, r_half=rh))
        f0, fm = W.sample_fields(ex, spec, 0.0), W.sample_fields(ex, spec, -dt)
        o.set_fields(0, f0["T"], f0["ur"], f0["uth"], f0["uph"], f0["p"])
        o.set_fields(1, fm["T"], fm["ur"], fm["uth"], fm["uph"], fm["p"])
        o.step(int(round(0.008 / dt)), 20)
        errs.append(_l2(spec, "c", o.get_fields(0)["T"] - W.sample_fields(ex, spec, o.t)["T"]))
    assert math.log(errs[0] / errs[1]) / math.log(2.0) > 1.8, errs
