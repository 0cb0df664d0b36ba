"""Discrete operators of the scheme (oracle; test infrastructure).

Everything here acts on padded arrays of one or both patches (see grid.py)
and returns compact arrays over the unknowns of one location type.

Continuous targets (Sec. 1 and Sec. 3.3, viscosity nu = Pr, conductivity 1):
  T     : lap T - a.grad T + f_T                                (Eq. Convect_Douglas)
  u_r   : nu[lap u_r - 2u_r/r^2 + (2/r^3) d_r(r^2 u_r)]
          - [a.grad u_r - (a_th b_th + a_ph b_ph)/r] - d_r P + (2chi)^-1 d_r(div b)
          + Pr Ra T + f_r                                       (Sec. 3.3.1)
  u_th  : nu[lap u_th - u_th/(r^2 s^2) + (2c/(r^2 s^2)) d_th(s u_th) + (2/r^2) d_th u_r
          + (2c/(r^3 s)) d_r(r^2 u_r)] - [a.grad u_th + (a_th b_r - a_ph b_ph cot)/r]
          - r^-1 d_th P + (2chi)^-1 r^-1 d_th(div b) + f_th     (Sec. 3.3.2)
  u_ph  : nu[lap u_ph - u_ph/(r^2 s^2) + (2/(r^2 s)) d_ph u_r + (2c/(r^2 s^2)) d_ph u_th]
          - [a.grad u_ph + (a_ph b_r + a_ph b_th cot)/r]
          - (r s)^-1 d_ph P + (2chi)^-1 (r s)^-1 d_ph(div b) + f_ph   (Sec. 3.3.3)
with s = sin(theta), c = cos(theta), b the velocity being advanced and a the
extrapolated advecting velocity u_2^{*,n+1/2} (Sec. 3.3).  The viscous rows use
the continuity-substituted forms printed in Sec. 3.3.1-3.3.2; the curvature
terms are the spherical components of the directional derivative (a.grad)b,
which reduce to the printed nonlinear terms when a = b = u.

Discretisation rules (second-order centred differences on the MAC grid, Sec. 4):
  * diffusion is conservative 3-point with the metric at the half points,
    e.g. D_rr x_m = r_m^-2 [r_{m+1/2}^2 (x_{m+1}-x_m)/h_{m+1/2}
                            - r_{m-1/2}^2 (x_m-x_{m-1})/h_{m-1/2}] / h_m;
  * a first derivative of a quantity stored half a cell away is a 2-point
    difference over the distance of the two points, otherwise a centred
    difference over 2 h of the point;
  * radial spacings are local (grid.py: h_c at centres, h_f at faces; both
    h_r on a uniform grid);
  * a quantity needed off its own location is the arithmetic mean of its 2 or
    4 nearest stored values (products are formed after averaging each factor);
  * metric factors are evaluated exactly at the point of the row.
"""
from __future__ import annotations

import numpy as np

from .grid import C, PH, R, TH, view


# ----------------------------------------------------------------- metric
def _rc(g, reg, d=0):
    return g.r_c(np.arange(reg[0] + d, reg[1] + d))[None, :, None, None]


def _rf(g, reg, d=0):
    return g.r_f(np.arange(reg[0] + d, reg[1] + d))[None, :, None, None]


def _hc(g, reg, d=0):
    """Radial cell widths h_c at centre indices reg[0] + d .. reg[1] + d."""
    return g.h_c(np.arange(reg[0] + d, reg[1] + d))[None, :, None, None]


def _hf(g, reg, d=0):
    """Radial centre distances h_f at face indices reg[0] + d .. reg[1] + d."""
    return g.h_f(np.arange(reg[0] + d, reg[1] + d))[None, :, None, None]


def _sc(g, reg, d=0):
    return np.sin(g.th_c(np.arange(reg[2] + d, reg[3] + d)))[None, None, :, None]


def _sf(g, reg, d=0):
    return np.sin(g.th_f(np.arange(reg[2] + d, reg[3] + d)))[None, None, :, None]


def _cc(g, reg, d=0):
    return np.cos(g.th_c(np.arange(reg[2] + d, reg[3] + d)))[None, None, :, None]


def _cf(g, reg, d=0):
    return np.cos(g.th_f(np.arange(reg[2] + d, reg[3] + d)))[None, None, :, None]


def _avg(a, reg, offs):
    return sum(view(a, reg, *o) for o in offs) / len(offs)


# 4-point neighbourhoods of other staggered components at each face type
# (offsets in logical index of the array being averaged)
NB = {
    # at u_r faces (face i, cell j, cell k)
    (R, TH): [(-1, 0, 0), (-1, 1, 0), (0, 0, 0), (0, 1, 0)],
    (R, PH): [(-1, 0, 0), (-1, 0, 1), (0, 0, 0), (0, 0, 1)],
    # at u_theta faces (cell i, face j, cell k)
    (TH, R): [(0, -1, 0), (1, -1, 0), (0, 0, 0), (1, 0, 0)],
    (TH, PH): [(0, -1, 0), (0, -1, 1), (0, 0, 0), (0, 0, 1)],
    # at u_phi faces (cell i, cell j, face k)
    (PH, R): [(0, 0, -1), (1, 0, -1), (0, 0, 0), (1, 0, 0)],
    (PH, TH): [(0, 0, -1), (0, 1, -1), (0, 0, 0), (0, 1, 0)],
    # at cell centres: the two faces of the cell
    (C, R): [(0, 0, 0), (1, 0, 0)],
    (C, TH): [(0, 0, 0), (0, 1, 0)],
    (C, PH): [(0, 0, 0), (0, 0, 1)],
}
COMP_LOC = (R, TH, PH)


def advecting(g, loc, A):
    """(a_r, a_th, a_ph) at the unknowns of ``loc``: own component as stored,
    the others averaged from their nearest stored values."""
    reg = g.region(loc)
    out = []
    for m, cl in enumerate(COMP_LOC):
        if cl == loc:
            out.append(view(A[m], reg))
        else:
            out.append(_avg(A[m], reg, NB[(loc, cl)]))
    return out


# ----------------------------------------------------------------- divergence
def divergence(g, U):
    """Discrete divergence at cell centres (compact, region C):
    (r+^2 u_r+ - r-^2 u_r-)/(r^2 h_r) + (s+ u_th+ - s- u_th-)/(r s h_th)
    + (u_ph+ - u_ph-)/(r s h_ph)."""
    reg = g.region(C)
    r, s = _rc(g, reg), _sc(g, reg)
    Ur, Ut, Up = U
    d_r = (_rf(g, reg, 1) ** 2 * view(Ur, reg, 1, 0, 0) - _rf(g, reg) ** 2 * view(Ur, reg)) / (r * r * _hc(g, reg))
    d_t = (_sf(g, reg, 1) * view(Ut, reg, 0, 1, 0) - _sf(g, reg) * view(Ut, reg)) / (r * s * g.hth)
    d_p = (view(Up, reg, 0, 0, 1) - view(Up, reg)) / (r * s * g.hph)
    return d_r + d_t + d_p


def padded(g, compact, loc=C):
    out = g.zeros()
    view(out, g.region(loc))[...] = compact
    return out


# ----------------------------------------------------------------- rates
def rate_T(g, X, A, f, kappa=1.0):
    """Rate of the temperature equation, kappa lap X - a.grad X + f, at centres."""
    reg = g.region(C)
    r, s = _rc(g, reg), _sc(g, reg)
    ht, hp = g.hth, g.hph
    X0 = view(X, reg)
    Xr_p, Xr_m = view(X, reg, 1, 0, 0), view(X, reg, -1, 0, 0)
    Xt_p, Xt_m = view(X, reg, 0, 1, 0), view(X, reg, 0, -1, 0)
    Xp_p, Xp_m = view(X, reg, 0, 0, 1), view(X, reg, 0, 0, -1)
    hc = _hc(g, reg)
    Drr = (_rf(g, reg, 1) ** 2 * (Xr_p - X0) / _hf(g, reg, 1) - _rf(g, reg) ** 2 * (X0 - Xr_m) / _hf(g, reg)) / (r * r * hc)
    Dtt = (_sf(g, reg, 1) * (Xt_p - X0) - _sf(g, reg) * (X0 - Xt_m)) / (r * r * s * ht * ht)
    Dpp = (Xp_p - 2.0 * X0 + Xp_m) / (r * r * s * s * hp * hp)
    ar, at, ap = advecting(g, C, A)
    adv = (ar * (Xr_p - Xr_m) / (2 * hc) + at * (Xt_p - Xt_m) / (2 * r * ht)
           + ap * (Xp_p - Xp_m) / (2 * r * s * hp))
    return kappa * (Drr + Dtt + Dpp) - adv + f


def rate_ur(g, U, A, P, D, Tb, f, nu, chi, PrRa):
    """Rate of the u_r equation at interior r-faces.  U: half-level velocity
    (padded), P: pressure entering the row (padded), D: divergence of U
    (padded), Tb: half-level temperature (padded)."""
    reg = g.region(R)
    r, s = _rf(g, reg), _sc(g, reg)
    ht, hp = g.hth, g.hph
    X = U[0]
    X0 = view(X, reg)
    Xr_p, Xr_m = view(X, reg, 1, 0, 0), view(X, reg, -1, 0, 0)
    Xt_p, Xt_m = view(X, reg, 0, 1, 0), view(X, reg, 0, -1, 0)
    Xp_p, Xp_m = view(X, reg, 0, 0, 1), view(X, reg, 0, 0, -1)
    hf = _hf(g, reg)
    Drr = (_rc(g, reg) ** 2 * (Xr_p - X0) / _hc(g, reg) - _rc(g, reg, -1) ** 2 * (X0 - Xr_m) / _hc(g, reg, -1)) / (r * r * hf)
    Dtt = (_sf(g, reg, 1) * (Xt_p - X0) - _sf(g, reg) * (X0 - Xt_m)) / (r * r * s * ht * ht)
    Dpp = (Xp_p - 2.0 * X0 + Xp_m) / (r * r * s * s * hp * hp)
    extra = (-2.0 * X0 / (r * r)
             + 2.0 / r ** 3 * (_rf(g, reg, 1) ** 2 * Xr_p - _rf(g, reg, -1) ** 2 * Xr_m) / (2 * hf))
    ar, at, ap = advecting(g, R, A)
    bt = _avg(U[1], reg, NB[(R, TH)])
    bp = _avg(U[2], reg, NB[(R, PH)])
    adv = (ar * (Xr_p - Xr_m) / (2 * hf) + at * (Xt_p - Xt_m) / (2 * r * ht)
           + ap * (Xp_p - Xp_m) / (2 * r * s * hp) - (at * bt + ap * bp) / r)
    gradP = (view(P, reg) - view(P, reg, -1, 0, 0)) / hf
    gdiv = (view(D, reg) - view(D, reg, -1, 0, 0)) / hf
    buoy = PrRa * 0.5 * (view(Tb, reg, -1, 0, 0) + view(Tb, reg))
    return nu * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv / (2 * chi) + buoy + f


def rate_ut(g, U, A, P, D, f, nu, chi):
    """Rate of the u_theta equation at interior theta-faces."""
    reg = g.region(TH)
    r, s, c = _rc(g, reg), _sf(g, reg), _cf(g, reg)
    ht, hp = g.hth, g.hph
    X, W = U[1], U[0]
    X0 = view(X, reg)
    Xr_p, Xr_m = view(X, reg, 1, 0, 0), view(X, reg, -1, 0, 0)
    Xt_p, Xt_m = view(X, reg, 0, 1, 0), view(X, reg, 0, -1, 0)
    Xp_p, Xp_m = view(X, reg, 0, 0, 1), view(X, reg, 0, 0, -1)
    hc = _hc(g, reg)
    Drr = (_rf(g, reg, 1) ** 2 * (Xr_p - X0) / _hf(g, reg, 1) - _rf(g, reg) ** 2 * (X0 - Xr_m) / _hf(g, reg)) / (r * r * hc)
    Dtt = (_sc(g, reg) * (Xt_p - X0) - _sc(g, reg, -1) * (X0 - Xt_m)) / (r * r * s * ht * ht)
    Dpp = (Xp_p - 2.0 * X0 + Xp_m) / (r * r * s * s * hp * hp)
    # u_r averaged to the r-centre, on theta-cells j and j-1
    W_j = 0.5 * (view(W, reg) + view(W, reg, 1, 0, 0))
    W_jm = 0.5 * (view(W, reg, 0, -1, 0) + view(W, reg, 1, -1, 0))
    dW_dth = (W_j - W_jm) / ht
    # d_r(r^2 u_r) at the r-centre on theta-cells j and j-1, averaged to the face
    q_j = (_rf(g, reg, 1) ** 2 * view(W, reg, 1, 0, 0) - _rf(g, reg) ** 2 * view(W, reg)) / hc
    q_jm = (_rf(g, reg, 1) ** 2 * view(W, reg, 1, -1, 0) - _rf(g, reg) ** 2 * view(W, reg, 0, -1, 0)) / hc
    dr_r2W = 0.5 * (q_j + q_jm)
    extra = (-X0 / (r * r * s * s)
             + 2.0 * c / (r * r * s * s) * (_sf(g, reg, 1) * Xt_p - _sf(g, reg, -1) * Xt_m) / (2 * ht)
             + 2.0 / (r * r) * dW_dth + 2.0 * c / (r ** 3 * s) * dr_r2W)
    ar, at, ap = advecting(g, TH, A)
    br = _avg(W, reg, NB[(TH, R)])
    bp = _avg(U[2], reg, NB[(TH, PH)])
    adv = (ar * (Xr_p - Xr_m) / (2 * hc) + at * (Xt_p - Xt_m) / (2 * r * ht)
           + ap * (Xp_p - Xp_m) / (2 * r * s * hp) + (at * br - ap * bp * c / s) / r)
    gradP = (view(P, reg) - view(P, reg, 0, -1, 0)) / (r * ht)
    gdiv = (view(D, reg) - view(D, reg, 0, -1, 0)) / (r * ht)
    return nu * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv / (2 * chi) + f


def rate_up(g, U, A, P, D, f, nu, chi):
    """Rate of the u_phi equation at interior phi-faces."""
    reg = g.region(PH)
    r, s, c = _rc(g, reg), _sc(g, reg), _cc(g, reg)
    ht, hp = g.hth, g.hph
    X, W, Y = U[2], U[0], U[1]
    X0 = view(X, reg)
    Xr_p, Xr_m = view(X, reg, 1, 0, 0), view(X, reg, -1, 0, 0)
    Xt_p, Xt_m = view(X, reg, 0, 1, 0), view(X, reg, 0, -1, 0)
    Xp_p, Xp_m = view(X, reg, 0, 0, 1), view(X, reg, 0, 0, -1)
    hc = _hc(g, reg)
    Drr = (_rf(g, reg, 1) ** 2 * (Xr_p - X0) / _hf(g, reg, 1) - _rf(g, reg) ** 2 * (X0 - Xr_m) / _hf(g, reg)) / (r * r * hc)
    Dtt = (_sf(g, reg, 1) * (Xt_p - X0) - _sf(g, reg) * (X0 - Xt_m)) / (r * r * s * ht * ht)
    Dpp = (Xp_p - 2.0 * X0 + Xp_m) / (r * r * s * s * hp * hp)
    W_k = 0.5 * (view(W, reg) + view(W, reg, 1, 0, 0))
    W_km = 0.5 * (view(W, reg, 0, 0, -1) + view(W, reg, 1, 0, -1))
    Y_k = 0.5 * (view(Y, reg) + view(Y, reg, 0, 1, 0))
    Y_km = 0.5 * (view(Y, reg, 0, 0, -1) + view(Y, reg, 0, 1, -1))
    extra = (-X0 / (r * r * s * s) + 2.0 / (r * r * s) * (W_k - W_km) / hp
             + 2.0 * c / (r * r * s * s) * (Y_k - Y_km) / hp)
    ar, at, ap = advecting(g, PH, A)
    br = _avg(W, reg, NB[(PH, R)])
    bt = _avg(Y, reg, NB[(PH, TH)])
    adv = (ar * (Xr_p - Xr_m) / (2 * hc) + at * (Xt_p - Xt_m) / (2 * r * ht)
           + ap * (Xp_p - Xp_m) / (2 * r * s * hp) + (ap * br + ap * bt * c / s) / r)
    gradP = (view(P, reg) - view(P, reg, 0, 0, -1)) / (r * s * hp)
    gdiv = (view(D, reg) - view(D, reg, 0, 0, -1)) / (r * s * hp)
    return nu * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv / (2 * chi) + f


# ----------------------------------------------------------------- 1-D factors
# Sweep order, first factor solved first (Sec. 4 for T; Eq. r_comp,
# theta_comp, phi_comp for the velocity components).
ORDER = {C: "rtp", R: "tpr", TH: "prt", PH: "rtp"}
# directions along which the correction has a reflection (cell-centred) wall
REFLECT_R = {C: True, R: False, TH: True, PH: True}


def factor(g, loc, d, A, dt, nu, chi, gamma=(-1.0, -1.0)):
    """Tridiagonal coefficients (lo, di, up) of (I - dt/2 Ahat_d) at the
    unknowns of ``loc`` along direction ``d`` in 'r', 't', 'p', with the
    homogeneous boundary rows of the correction already folded in (gamma:
    ghost factors of T at the two walls, see exchange.robin_ghost).

    Ahat_d (Sec. 3.2 modified operators; Eq. r_comp, theta_comp, phi_comp):
      diffusion: true D_rr along r; (R1^2 s)^-1 d_th(s d_th) along theta;
                 d_phph/(R1^2 sin^2 theta_1) along phi;
      advection: -a_r d_r, -(a_th/r) d_th, -(a_ph/(r s)) d_ph (centred);
      own-direction extras of the velocity rows:
        u_r along r : nu(-2/r^2 + 2 r^-3 d_r(r^2 .)) + (2chi)^-1 d_r(r^-2 d_r(r^2 .))
        u_th along t: nu(-1/(r^2 s^2) + 2c/(r^2 s^2) d_th(s .)) + (2chi)^-1 r^-1 d_th((r s)^-1 d_th(s .))
        u_ph along p: -nu/(r^2 s^2) + (2chi)^-1 (r s)^-2 d_phph."""
    reg = g.region(loc)
    ht, hp = g.hth, g.hph
    R1 = g.R1
    ar, at, ap = advecting(g, loc, A)
    r = _rf(g, reg) if loc == R else _rc(g, reg)
    s = _sf(g, reg) if loc == TH else _sc(g, reg)
    zero = 0.0
    if d == "r":
        # local spacings: h of the row's point, and of the half points on either side
        if loc == R:
            h, hp_, hm_ = _hf(g, reg), _hc(g, reg), _hc(g, reg, -1)
            cp_d = _rc(g, reg) ** 2 / (r * r * h * hp_)
            cm_d = _rc(g, reg, -1) ** 2 / (r * r * h * hm_)
        else:
            h, hp_, hm_ = _hc(g, reg), _hf(g, reg, 1), _hf(g, reg)
            cp_d = _rf(g, reg, 1) ** 2 / (r * r * h * hp_)
            cm_d = _rf(g, reg) ** 2 / (r * r * h * hm_)
        cm = nu * cm_d + ar / (2 * h)
        c0 = -nu * (cp_d + cm_d) + zero * ar
        cp = nu * cp_d - ar / (2 * h)
        if loc == R:
            cm = cm - nu * 2.0 * _rf(g, reg, -1) ** 2 / (r ** 3 * 2 * h)
            cp = cp + nu * 2.0 * _rf(g, reg, 1) ** 2 / (r ** 3 * 2 * h)
            c0 = c0 - nu * 2.0 / (r * r)
            k = 1.0 / (2 * chi)
            cm = cm + k * _rf(g, reg, -1) ** 2 / (_rc(g, reg, -1) ** 2 * hm_ * h)
            c0 = c0 - k * (_rf(g, reg) ** 2 / (_rc(g, reg) ** 2 * hp_ * h)
                           + _rf(g, reg) ** 2 / (_rc(g, reg, -1) ** 2 * hm_ * h))
            cp = cp + k * _rf(g, reg, 1) ** 2 / (_rc(g, reg) ** 2 * hp_ * h)
    elif d == "t":
        if loc == TH:
            cp_d = _sc(g, reg) / (R1 * R1 * s * ht * ht)
            cm_d = _sc(g, reg, -1) / (R1 * R1 * s * ht * ht)
        else:
            cp_d = _sf(g, reg, 1) / (R1 * R1 * s * ht * ht)
            cm_d = _sf(g, reg) / (R1 * R1 * s * ht * ht)
        cm = nu * cm_d + at / (2 * r * ht)
        c0 = -nu * (cp_d + cm_d) + zero * at
        cp = nu * cp_d - at / (2 * r * ht)
        if loc == TH:
            c = _cf(g, reg)
            q = 2.0 * c / (r * r * s * s) / (2 * ht)
            cm = cm - nu * q * _sf(g, reg, -1)
            cp = cp + nu * q * _sf(g, reg, 1)
            c0 = c0 - nu / (r * r * s * s)
            k = 1.0 / (2 * chi)
            cp = cp + k * _sf(g, reg, 1) / (r * r * _sc(g, reg) * ht * ht)
            c0 = c0 - k * (s / (r * r * _sc(g, reg) * ht * ht) + s / (r * r * _sc(g, reg, -1) * ht * ht))
            cm = cm + k * _sf(g, reg, -1) / (r * r * _sc(g, reg, -1) * ht * ht)
    elif d == "p":
        s1 = np.sin(g.theta1)
        cpm = 1.0 / (R1 * R1 * s1 * s1 * hp * hp)
        cm = nu * cpm + ap / (2 * r * s * hp)
        c0 = -2.0 * nu * cpm + zero * ap
        cp = nu * cpm - ap / (2 * r * s * hp)
        if loc == PH:
            c0 = c0 - nu / (r * r * s * s)
            k = 1.0 / (2 * chi)
            q = k / (r * r * s * s * hp * hp)
            cm, c0, cp = cm + q, c0 - 2.0 * q, cp + q
    else:
        raise ValueError(d)
    shp = view(A[0], reg).shape if loc == R else ar.shape
    lo = np.broadcast_to(-0.5 * dt * cm, shp).copy()
    di = np.broadcast_to(1.0 - 0.5 * dt * c0, shp).copy()
    up = np.broadcast_to(-0.5 * dt * cp, shp).copy()
    ax = {"r": 1, "t": 2, "p": 3}[d]
    first = [slice(None)] * 4
    last = [slice(None)] * 4
    first[ax] = 0
    last[ax] = -1
    first, last = tuple(first), tuple(last)
    if d == "r" and REFLECT_R[loc]:
        # correction ghost = gamma (first/last unknown) (homogeneous wall
        # condition; gamma = -1 for Dirichlet): fold into the diagonal
        g0, g1 = gamma if loc == C else (-1.0, -1.0)
        di[first] += g0 * lo[first]
        di[last] += g1 * up[last]
    lo[first] = 0.0
    up[last] = 0.0
    return lo, di, up


def apply_factor(lo, di, up, x, axis):
    """y = (lo, di, up) x along ``axis`` (boundary rows already folded)."""
    y = di * x
    xm = np.zeros_like(x)
    xp = np.zeros_like(x)
    sl_hi = [slice(None)] * 4
    sl_lo = [slice(None)] * 4
    sl_hi[axis] = slice(1, None)
    sl_lo[axis] = slice(None, -1)
    xm[tuple(sl_hi)] = x[tuple(sl_lo)]
    xp[tuple(sl_lo)] = x[tuple(sl_hi)]
    return y + lo * xm + up * xp
