"""Yin <-> Yang Schwarz boundary exchange (oracle; test infrastructure).

Sec. 4: the solution on each patch uses boundary data interpolated from the
currently available solution on the other patch (Algorithm steps 1, 3 and 7).
The interpolation order is not stated; the reading used is tensor bilinear
interpolation in the donor's local (theta', phi') at the same radius (both
patches share the radial grid), which is second-order accurate.

Geometry: a point with local unit vector x of one patch has local unit vector
M x in the other patch (M is its own inverse).  A vector with donor-local
spherical components (v_r, v_th', v_ph') has target components
v_r (radial directions coincide) and, tangentially,
  v_t = (e_t . M e_th') v_th' + (e_t . M e_ph') v_ph'   for e_t = e_th or e_ph.

Target points of each patch (logical indices, see grid.py):
  T      : theta-ghost rows j in {-1, Nth} (k interior) and phi-ghost
           columns k in {-1, Nph} (j interior), every radial cell;
  u_r    : the same (j, k) points, interior radial faces; wall faces carry
           the wall value;
  u_th   : edge faces j in {0, Nth} (k interior) and phi-ghosts k in {-1, Nph}
           at interior faces j in [1, Nth);
  u_ph   : edge faces k in {0, Nph} (j interior) and theta-ghosts j in {-1, Nth}
           at interior faces k in [1, Nph);
  p      : the outermost ring of interior cells (j in {0, Nth-1} or
           k in {0, Nph-1}), overwritten after the pressure update (step 7).
Radial ghosts of cell-centred quantities are reflections 2 g - x_0 about the
wall value g.  Every donor stencil lies strictly inside the donor's unknowns
(and, for the pressure ring, off the donor's ring); building a table checks
this and raises if the grid is too coarse for it.
"""
from __future__ import annotations

import math

import numpy as np

from .grid import C, PH, R, TH, M, e_phi, e_theta, sph_to_unit, unit_to_sph


def _target_points(g, kind):
    """Logical (j, k) target points in the (theta, phi) plane."""
    Nt, Np = g.Nth, g.Nph
    pts = []
    if kind in ("T", "ur"):
        pts += [(j, k) for j in (-1, Nt) for k in range(Np)]
        pts += [(j, k) for k in (-1, Np) for j in range(Nt)]
    elif kind == "uth":
        pts += [(j, k) for j in (0, Nt) for k in range(Np)]
        pts += [(j, k) for k in (-1, Np) for j in range(1, Nt)]
    elif kind == "uph":
        pts += [(j, k) for k in (0, Np) for j in range(Nt)]
        pts += [(j, k) for j in (-1, Nt) for k in range(1, Np)]
    elif kind == "p":
        ring = set()
        for k in range(Np):
            ring.add((0, k))
            ring.add((Nt - 1, k))
        for j in range(Nt):
            ring.add((j, 0))
            ring.add((j, Np - 1))
        pts = sorted(ring)
    else:
        raise ValueError(kind)
    return np.array([p[0] for p in pts]), np.array([p[1] for p in pts])


def _angles(g, loc, j, k):
    th = g.th_f(j) if loc == TH else g.th_c(j)
    ph = g.ph_f(k) if loc == PH else g.ph_c(k)
    return th, ph


def _stencil(g, loc, th, ph, strict_ring=False):
    """Bilinear stencil of donor quantity at ``loc`` for donor angles (th, ph):
    base indices (j0, k0) and weights (wj, wk) along theta and phi."""
    jf = (th - g.th0) / g.hth - (0.0 if loc == TH else 0.5)
    kf = (ph - g.ph0) / g.hph - (0.0 if loc == PH else 0.5)
    j0 = np.floor(jf).astype(np.int64)
    k0 = np.floor(kf).astype(np.int64)
    # allowed base ranges: the stencil (j0, j0+1) x (k0, k0+1) must be unknowns
    jlo, jhi = (1, g.Nth - 1) if loc == TH else (0, g.Nth - 1)
    klo, khi = (1, g.Nph - 1) if loc == PH else (0, g.Nph - 1)
    if strict_ring:
        jlo, jhi, klo, khi = jlo + 1, jhi - 1, klo + 1, khi - 1
    if (j0 < jlo).any() or (j0 + 1 > jhi).any() or (k0 < klo).any() or (k0 + 1 > khi).any():
        raise ValueError("exchange donor stencil leaves the donor interior: grid too coarse")
    return j0, k0, jf - j0, kf - k0


class ExchangeTables:
    """Per-target donor stencils and rotations; identical for both patches."""

    def __init__(self, g):
        self.g = g
        self.tab = {}
        for kind, loc in (("T", C), ("ur", R), ("uth", TH), ("uph", PH), ("p", C)):
            j, k = _target_points(g, kind)
            th, ph = _angles(g, loc, j, k)
            x = sph_to_unit(th, ph)
            xd = x @ M.T
            thd, phd = unit_to_sph(xd)
            entry = {"j": j, "k": k}
            if kind in ("T", "ur", "p"):
                entry["s"] = _stencil(g, C, thd, phd, strict_ring=(kind == "p"))
            else:
                entry["st"] = _stencil(g, TH, thd, phd)
                entry["sp"] = _stencil(g, PH, thd, phd)
                e_t = e_theta(th, ph) if kind == "uth" else e_phi(th, ph)
                Met = e_theta(thd, phd) @ M.T
                Mep = e_phi(thd, phd) @ M.T
                entry["rot"] = (np.sum(e_t * Met, axis=-1), np.sum(e_t * Mep, axis=-1))
            self.tab[kind] = entry


def _interp(a_donor, st, i_slice):
    """Bilinear interpolation of padded donor array a_donor[i, j, k] at the
    stencils st for every radial index of i_slice -> shape (ni, npts)."""
    j0, k0, wj, wk = st
    A = a_donor[i_slice]
    J, K = j0 + 1, k0 + 1
    return ((1 - wj) * (1 - wk) * A[:, J, K] + (1 - wj) * wk * A[:, J, K + 1]
            + wj * (1 - wk) * A[:, J + 1, K] + wj * wk * A[:, J + 1, K + 1])


def boundary_flux_weights(g):
    """Outward normal times face area of every boundary velocity value of a
    patch, from the discrete Gauss theorem of the divergence (Sec. 3.3: the
    sum over cells of div * r^2 sin(theta) h_c h_th h_ph telescopes to these
    face terms): theta-edge faces r_c sin(theta_f) h_c h_ph, phi-edge faces
    r_c h_c h_th, wall faces r_f^2 sin(theta_c) h_th h_ph (h_c the radial cell
    width, grid.py).  Returns
    (wt0, wt1, wp0, wp1, wr0, wr1) shaped like the faces' value blocks
    (Nr x Nph, Nr x Nph, Nr x Nth, Nr x Nth, Nth x Nph, Nth x Nph)."""
    Nr, Nt, Np = g.Nr, g.Nth, g.Nph
    rc = g.r_c(np.arange(Nr))[:, None]
    hc = g.h_c(np.arange(Nr))[:, None]
    sc = np.sin(g.th_c(np.arange(Nt)))
    ones_p = np.ones((1, Np))
    wt = lambda j: rc * math.sin(g.th_f(j)) * hc * g.hph * ones_p
    wp = rc * hc * g.hth * np.ones((1, Nt))
    wr = lambda i: g.r_f(i) ** 2 * sc[:, None] * g.hth * g.hph * ones_p
    return (-wt(0), wt(Nt), -wp, wp, -wr(0), wr(Nr))


def mass_flux_correction(g, U, p, eps, tol, maxit=50):
    """Algorithm step 4: if the net flux of patch p's boundary velocity
    through its boundary is at least tol, replace the interpolated normal
    components v on the theta and phi edges by the minimiser of
      J(v) = |v - u_bd|^2 / 2 + (flux_edges(v) + flux_walls(u_bd))^2 / (2 eps |dOmega|^2)
    found by the conjugate gradient method (the Hessian is I + alpha w w^T,
    alpha = 1 / (eps |dOmega|^2), w the edge weights).  U: padded velocity
    components [u_r, u_theta, u_phi] of both patches."""
    Nr, Nt, Np = g.Nr, g.Nth, g.Nph
    wt0, wt1, wp0, wp1, wr0, wr1 = boundary_flux_weights(g)
    ur, ut, up = U[0][p], U[1][p], U[2][p]
    cells_r = slice(1, Nr + 1)
    blocks = [(ut, (cells_r, 1, slice(1, Np + 1)), wt0), (ut, (cells_r, Nt + 1, slice(1, Np + 1)), wt1),
              (up, (cells_r, slice(1, Nt + 1), 1), wp0), (up, (cells_r, slice(1, Nt + 1), Np + 1), wp1)]
    u = np.concatenate([a[ix].ravel() for a, ix, _ in blocks])
    w = np.concatenate([wb.ravel() for _, _, wb in blocks])
    c = np.sum(wr0 * ur[1, 1:Nt + 1, 1:Np + 1]) + np.sum(wr1 * ur[Nr + 1, 1:Nt + 1, 1:Np + 1])
    if abs(np.dot(w, u) + c) < tol:
        return
    area = np.sum(np.abs(w)) + np.sum(np.abs(wr0)) + np.sum(np.abs(wr1))
    alpha = 1.0 / (eps * area * area)
    H = lambda x: x + alpha * w * np.dot(w, x)
    b = u - alpha * c * w
    x = u.copy()
    r = b - H(x)
    d = r.copy()
    rr = np.dot(r, r)
    for _ in range(maxit):
        if math.sqrt(rr) <= 1e-15 * math.sqrt(np.dot(b, b)):
            break
        Hd = H(d)
        a = rr / np.dot(d, Hd)
        x += a * d
        r -= a * Hd
        rr_new = np.dot(r, r)
        d = r + (rr_new / rr) * d
        rr = rr_new
    o = 0
    for a, ix, wb in blocks:
        a[ix] = x[o:o + wb.size].reshape(wb.shape)
        o += wb.size


def exchange_into(tables, target, fields, patches, T_walls=(0.0, 0.0), U_walls=None, step4=None,
                  T_robin=((1.0, 0.0), (1.0, 0.0))):
    """Fill the boundary values of the listed target ``patches`` from the other
    patch, for the state dict ``fields`` (padded arrays with keys 'T' and the
    velocity lists 'u1', 'u2').  Donor values are read from a snapshot taken
    before any write, so both patches may be filled at once (additive Schwarz)."""
    g = tables.g
    tab = tables.tab
    Nr = g.Nr
    src = {"T": fields["T"].copy(), "u1": [u.copy() for u in fields["u1"]],
           "u2": [u.copy() for u in fields["u2"]]}
    cells = slice(1, Nr + 1)          # logical i in [0, Nr)
    ifaces = slice(2, Nr + 1)         # logical r-faces i in [1, Nr)
    for p in patches:
        d = 1 - p
        e = tab["T"]
        target["T"][p][cells, e["j"] + 1, e["k"] + 1] = _interp(src["T"][d], e["s"], cells)
        for key in ("u1", "u2"):
            U, S = target[key], src[key]
            e = tab["ur"]
            U[0][p][ifaces, e["j"] + 1, e["k"] + 1] = _interp(S[0][d], e["s"], ifaces)
            for kind, comp in (("uth", 1), ("uph", 2)):
                e = tab[kind]
                vt = _interp(S[1][d], e["st"], cells)
                vp = _interp(S[2][d], e["sp"], cells)
                U[comp][p][cells, e["j"] + 1, e["k"] + 1] = e["rot"][0] * vt + e["rot"][1] * vp
    wall_ghosts(g, target, patches, T_walls, U_walls, T_robin)
    if step4 is not None:   # (eps, tol): Algorithm step 4 on both systems' boundary velocity
        for p in patches:
            for key in ("u1", "u2"):
                mass_flux_correction(g, target[key], p, step4[0], step4[1])


def robin_ghost(a, b, h):
    """Ghost x_g = gamma x_0 + delta of a cell-centred quantity for the wall
    condition a x + b dx/dn = g (Sec. 1: Dirichlet, Neumann or Robin walls),
    with x = (x_g + x_0)/2 and dx/dn = (x_g - x_0)/h on the wall, h the
    distance of the ghost centre from the first one (h_f of the wall face):
    returns (gamma, delta per unit g).  Dirichlet (1, 0): (-1, 2)."""
    den = 0.5 * a + b / h
    return -(0.5 * a - b / h) / den, 1.0 / den


def wall_ghosts(g, fields, patches, T_walls=(0.0, 0.0), U_walls=None, T_robin=((1.0, 0.0), (1.0, 0.0))):
    """Radial wall data (Sec. 2): u_r on the wall faces is the wall value;
    u_theta, u_phi get the reflection ghost 2 g - x_0 about the wall velocity g;
    T gets the ghost of its wall condition a T + b dT/dn = T_wall (T_robin
    gives (a, b) per wall; (1, 0) = Dirichlet: 2 T_wall - T_0); T_walls[w]
    is a constant or per point, [2 patches][Nth][Nph].
    U_walls: None (no-slip) or wall velocities as in Params.wall_u."""
    Nr, Nt, Np = g.Nr, g.Nth, g.Nph
    gi, di_ = robin_ghost(T_robin[0][0], T_robin[0][1], float(g.h_f(0)))
    go, do_ = robin_ghost(T_robin[1][0], T_robin[1][1], float(g.h_f(Nr)))

    def wall_T(w, p):   # a constant, or per point [2 patches][Nth][Nph]
        a = np.asarray(T_walls[w], dtype=np.float64)
        return a[p] if a.ndim == 3 else a

    for p in patches:
        T = fields["T"][p]
        T[0, 1:Nt + 1, 1:Np + 1] = gi * T[1, 1:Nt + 1, 1:Np + 1] + di_ * wall_T(0, p)
        T[Nr + 1, 1:Nt + 1, 1:Np + 1] = go * T[Nr, 1:Nt + 1, 1:Np + 1] + do_ * wall_T(1, p)
        if U_walls is None:
            gr = (0.0, 0.0)
            gt = (0.0, 0.0)
            gp = (0.0, 0.0)
        else:
            gr = (U_walls["ur"][0][p], U_walls["ur"][1][p])
            gt = (U_walls["uth"][0][p][1:Nt, :], U_walls["uth"][1][p][1:Nt, :])
            gp = (U_walls["uph"][0][p][:, 1:Np], U_walls["uph"][1][p][:, 1:Np])
        for key in ("u1", "u2"):
            U = fields[key]
            U[0][p][1, :, :] = 0.0
            U[0][p][Nr + 1, :, :] = 0.0
            U[0][p][1, 1:Nt + 1, 1:Np + 1] = gr[0]
            U[0][p][Nr + 1, 1:Nt + 1, 1:Np + 1] = gr[1]
            ut = U[1][p]
            ut[0, 2:Nt + 1, 1:Np + 1] = 2.0 * gt[0] - ut[1, 2:Nt + 1, 1:Np + 1]
            ut[Nr + 1, 2:Nt + 1, 1:Np + 1] = 2.0 * gt[1] - ut[Nr, 2:Nt + 1, 1:Np + 1]
            up = U[2][p]
            up[0, 1:Nt + 1, 2:Np + 1] = 2.0 * gp[0] - up[1, 1:Nt + 1, 2:Np + 1]
            up[Nr + 1, 1:Nt + 1, 2:Np + 1] = 2.0 * gp[1] - up[Nr, 1:Nt + 1, 2:Np + 1]


def pressure_ring(tables, P, patches):
    """Step 7: overwrite the outermost ring of interior pressure cells of each
    listed patch by interpolation of the other patch's pressure (padded array
    P of both patches).  Donor stencils avoid the donor's ring, so both patches
    may be updated at once."""
    g = tables.g
    e = tables.tab["p"]
    cells = slice(1, g.Nr + 1)
    src = P.copy()
    for p in patches:
        P[p][cells, e["j"] + 1, e["k"] + 1] = _interp(src[1 - p], e["s"], cells)
