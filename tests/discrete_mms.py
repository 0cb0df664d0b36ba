"""A discrete manufactured solution for time-convergence studies (test
infrastructure; used by the oracle pins and the GPU time study).

The fields are fixed grid functions times functions of time,
    u(t) = cos t U,  T(t) = cos t Theta,  p(t) = cos t P,
where U is discretely divergence-free on the MAC grid and every field is
supported inside the part of the Yin patch that the Yang patch does not
cover, at a distance from its edge larger than the interpolation stencils.
The Yang patch therefore holds zeros, every boundary value the Schwarz
exchange interpolates is exactly zero, and the wall values are those of the
scheme's own wall rules.  The forcing is the semi-discrete residual of these
fields, taken from the oracle's spatial rates (each pinned separately
against continuous operators):
    f(t) = du/dt - Rate_h(u(t); a = u(t)),
split into the separable time modes sin t, cos t and cos^2 t (the advection
is quadratic).  The grid functions are then an exact solution of the
spatially discrete incompressible problem, so a run's error against them is
its time-discretisation error alone: no spatial error, and no acoustic
transient of the artificial compressibility started by a discrete
divergence of the initial data.

Construction of U (Stokes' theorem on the MAC cells): line integrals E of a
smooth vector potential along the cell edges (midpoint rule), face fluxes as
the circulation around each face, velocities as flux / face area with the
face areas of the discrete divergence
    (r_f^2 sin th_c h_th h_ph, r_c sin th_f h_r h_ph, r_c h_r h_th),
so that the divergence of every cell is a sum in which each edge integral
appears twice with opposite signs: zero up to rounding.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import operators as ops
from oracle.grid import C, PH, R, TH, view
from oracle.scheme import Oracle, Params

# time functions of the forcing modes (their ids in set_forcing)
TAU_COS, TAU_SIN, TAU_COS2 = 1, 2, 3


def _fields(g, rho0):
    """U, Theta, P of one patch in the user layouts (Yin; Yang is zero)."""
    Nr, Nt, Np = g.Nr, g.Nth, g.Nph
    rc, rf = g.r_c(np.arange(Nr)), g.r_f(np.arange(Nr + 1))
    tc, tf = g.th_c(np.arange(Nt)), g.th_f(np.arange(Nt + 1))
    pc, pf = g.ph_c(np.arange(Np)), g.ph_f(np.arange(Np + 1))
    L = g.R2 - g.R1

    def shape(r, th, ph, a, b, c):
        Rr, Tt, Pp = np.meshgrid(r, th, ph, indexing="ij")
        radial = np.sin(np.pi * (Rr - g.R1) / L) ** 2
        # angular distance from the Yin patch centre (theta = pi/2, phi = 0)
        rho = np.arccos(np.clip(np.sin(Tt) * np.cos(Pp), -1.0, 1.0))
        bump = np.where(rho < rho0, np.cos(0.5 * np.pi * rho / rho0) ** 4, 0.0)
        return radial * bump * (a + b * np.sin(2 * Tt + 0.3) + c * np.cos(3 * Pp - 0.2))

    # edge line integrals of the potential: along r at (r_c, th_f, ph_f), along
    # theta at (r_f, th_c, ph_f), along phi at (r_f, th_f, ph_c)
    Er = shape(rc, tf, pf, 0.7, 0.4, 0.3) * g.hr
    Et = shape(rf, tc, pf, -0.5, 0.6, 0.2) * rf[:, None, None] * g.hth
    Ep = shape(rf, tf, pc, 0.8, -0.3, 0.5) * (rf[:, None, None] * np.sin(tf)[None, :, None]) * g.hph
    # circulations around the faces (right-handed about +r, +theta, +phi)
    Fr = Et[:, :, :-1] + Ep[:, 1:, :] - Et[:, :, 1:] - Ep[:, :-1, :]
    Ft = Ep[:-1, :, :] + Er[:, :, 1:] - Ep[1:, :, :] - Er[:, :, :-1]
    Fp = Er[:, :-1, :] + Et[1:, :, :] - Er[:, 1:, :] - Et[:-1, :, :]
    Ar = (rf ** 2)[:, None, None] * np.sin(tc)[None, :, None] * g.hth * g.hph
    At = rc[:, None, None] * np.sin(tf)[None, :, None] * g.hr * g.hph
    Ap = rc[:, None, None] * g.hr * g.hth
    return {"ur": Fr / Ar, "uth": Ft / At, "uph": Fp / Ap,
            "T": shape(rc, tc, pc, 0.6, 0.5, -0.4), "p": shape(rc, tc, pc, 0.3, -0.7, 0.5)}


def _to_user(g, loc, compact):
    a = g.zeros()
    view(a, g.region(loc))[...] = compact
    return a[g.user_slices(loc)]


class DiscreteMMS:
    """The grid functions (user layouts, both patches) and the forcing modes
    for the shell of ``prm`` (uniform radial grid)."""

    def __init__(self, prm: Params, rho0: float = 0.35):
        if prm.r_half is not None:
            raise ValueError("uniform radial grids only")
        o = Oracle(prm)
        g = o.g
        yin = _fields(g, rho0)
        self.U = {k: np.stack([v, np.zeros_like(v)]) for k, v in yin.items()}
        # the state with every boundary value filled by the scheme's own
        # exchange, wall and ring rules
        o.set_fields(0, *(self.U[k] for k in ("T", "ur", "uth", "uph", "p")))
        L = o.lev[0]
        self.div_max = float(np.abs(ops.divergence(g, L.u2)).max())
        self.yang_max = max(float(np.abs(a[1]).max()) for a in (L.T, L.p2, *L.u2))
        z = g.zeros
        zero_A = [z(), z(), z()]
        D = ops.padded(g, ops.divergence(g, L.u2))
        fz = {loc: np.zeros(view(z(), g.region(loc)).shape) for loc in (C, R, TH, PH)}
        nu, chi, PrRa = prm.Pr, prm.chi, prm.Pr * prm.Ra

        def rates(A):
            return {"T": ops.rate_T(g, L.T, A, fz[C], prm.kappa),
                    "ur": ops.rate_ur(g, L.u2, A, L.p2, D, L.T, fz[R], nu, chi, PrRa),
                    "uth": ops.rate_ut(g, L.u2, A, L.p2, D, fz[TH], nu, chi),
                    "uph": ops.rate_up(g, L.u2, A, L.p2, D, fz[PH], nu, chi)}

        lin = rates(zero_A)                  # linear in the fields: time function cos t
        full = rates([a.copy() for a in L.u2])
        locs = {"T": C, "ur": R, "uth": TH, "uph": PH}
        keys = ("T", "ur", "uth", "uph")
        # f = -sin t U - cos t Rate_lin - cos^2 t (Rate_full - Rate_lin)
        self.modes = [(TAU_SIN, [-self.U[k] for k in keys]),
                      (TAU_COS, [_to_user(g, locs[k], -lin[k]) for k in keys]),
                      (TAU_COS2, [_to_user(g, locs[k], -(full[k] - lin[k])) for k in keys])]

    def at(self, t):
        """Exact fields at time t (user layouts)."""
        c = math.cos(t)
        return {k: c * v for k, v in self.U.items()}

    def support(self):
        """Yin cells where the pressure grid function is non-zero."""
        return np.abs(self.U["p"][0]) > 0
