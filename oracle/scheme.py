"""The AC time step with Schwarz iterations (oracle; test infrastructure).

Time discretisation (Sec. 3.3): Crank-Nicolson artificial compressibility with
bootstrapping.  System 1 (Eq. ac1) and system 2 (Eq. ac2) are advanced with
the same advecting velocity a = u_2^{*,n+1/2} = 1.5 u_2^n - 0.5 u_2^{n-1}, so
both share one set of line-solve matrices.  Eliminating p^{n+1} gives
  p_1^{n+1} = p_1^n - chi^-1 div u_1^{n+1/2}                       (Eq. nst_Mass1)
  p_2^{n+1} = p_2^n + (p_1^{n+1} - p_1^n) - chi^-1 div u_2^{n+1/2}  (Eq. ac2)
and the momentum rows see P_1 = p_1^n, P_2 = p_2^n + (p_1^{n+1} - p_1^n)/2
plus the grad-div term (2chi)^-1 grad div u_s^{n+1/2}.

Splitting-error reduction (Eq. er): every line-solved unknown psi is advanced
by the defect correction
  P_psi (psi^k - psi^{k-1}) = -F_psi(psi^{k-1}),
  F_psi(psi) = (psi - psi^n) - dt Rate_psi((psi + psi^n)/2),
with P_psi the product of the 1-D factors (I - dt/2 Ahat_d).  The equation
as printed has the fixed point (I - L) d = -G; the reading used is the one
whose fixed point is the Crank-Nicolson AC system and whose first iterate,
from psi^0 = 2 psi^n - psi^{n-1}, is the factored scheme of Eq. HeatDouglas /
Eq. Convect_Douglas up to O(dt^3).  The velocity components are advanced in
the Gauss-Seidel order r, theta, phi (Sec. 3.3 grad-div splitting), each with
the newest values of the others; T is advanced first.

Schwarz iteration (Sec. 4): additive (both patches from the previous
iterate, the default) or multiplicative (Algorithm: Yin then Yang, each from
the other's newest data).  Step 4 (mass-flux correction) is skipped, as in
all of the paper's results; step 7 (pressure exchange) is on.  After the last
iteration the boundary values are refreshed from the final iterate, so the
stored time levels are functions of their interior values only.

The l2 norm (Sec. 5.1) is the midpoint rule with weight r^2 sin(theta).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import exchange as xch
from . import operators as ops
from .grid import C, PH, R, TH, Grid, view
from .linesolve import solve_factored

FIELD_NAMES = ("T", "u1r", "u1t", "u1p", "p1", "u2r", "u2t", "u2p", "p2")


@dataclass
class Params:
    R1: float
    R2: float
    Pr: float
    Ra: float
    dt: float
    Nr: int
    Nth: int
    Nph: int
    chi: float = 1.0
    overlap: int = 2
    schwarz_mode: str = "additive"
    schwarz_tol: float = 0.0
    T_in: float = 0.0
    T_out: float = 0.0
    # temperature wall condition a T + b dT/dn = T_in / T_out per wall (Sec. 1:
    # Dirichlet (1, 0), Neumann (0, 1) or Robin)
    Tbc_in: tuple = (1.0, 0.0)
    Tbc_out: tuple = (1.0, 0.0)
    step7: bool = True
    kappa: float = 1.0
    # Dirichlet velocity on the walls r = R1, R2 (steady), in each patch's local
    # basis: dict 'ur' [2 walls][2 patches][Nth][Nph], 'uth' [..][Nth+1][Nph],
    # 'uph' [..][Nth][Nph+1]; None = no-slip
    wall_u: Optional[dict] = None
    # Algorithm step 4 (mass-flux correction of the interpolated boundary
    # velocity); the paper skips it for its results, so it is off by default
    step4: bool = False
    step4_eps: float = 1e-8
    step4_tol: float = 1e-13
    # radii of the 2 Nr + 1 radial half points (faces at even, centres at odd
    # positions; grid.py); None = uniform radial grid
    r_half: Optional[tuple] = None
    # time-dependent Dirichlet wall data tau(t) W (the manufactured solution
    # of Sec. 5.1 has non-zero, time-dependent walls): (time function id,
    # dict with any of 'T' [2 walls][2 patches][Nth][Nph] added to T_in /
    # T_out, and 'ur', 'uth', 'uph' as in wall_u, added to it); None = none
    wall_mode: Optional[tuple] = None


def _time_fn(tid, t):
    import math
    return {0: 1.0, 1: math.cos(t), 2: math.sin(t), 3: math.cos(t) ** 2,
            4: math.sin(t) * math.cos(t)}[tid]


@dataclass
class Level:
    T: np.ndarray
    u1: list
    u2: list
    p1: np.ndarray
    p2: np.ndarray

    def copy(self):
        return Level(self.T.copy(), [u.copy() for u in self.u1], [u.copy() for u in self.u2],
                     self.p1.copy(), self.p2.copy())

    def as_dict(self):
        return {"T": self.T, "u1": self.u1, "u2": self.u2}


class Oracle:
    def __init__(self, prm: Params, exchange=True):
        self.prm = prm
        self.g = Grid(prm.R1, prm.R2, prm.Nr, prm.Nth, prm.Nph, prm.overlap, prm.r_half)
        # exchange=False: a single-patch problem with frozen boundary values
        self.tables = xch.ExchangeTables(self.g) if exchange else None
        g = self.g
        z = g.zeros
        self.lev = [Level(z(), [z(), z(), z()], [z(), z(), z()], z(), z()) for _ in range(2)]
        self.t = 0.0
        self.steps_done = 0
        self.modes = []           # list of (tid, {'T','ur','uth','uph'} compact arrays)
        self.last_norms = np.zeros(len(FIELD_NAMES))
        self.iters_done = 0
        self.level1_set = False
        ring_off = np.ones((1, 1, self.g.Nth, self.g.Nph))
        ring_off[:, :, 0, :] = ring_off[:, :, -1, :] = 0.0
        ring_off[:, :, :, 0] = ring_off[:, :, :, -1] = 0.0
        self._ring_off = ring_off

    # ------------------------------------------------------------ state io
    def _to_padded(self, loc, a):
        out = self.g.zeros()
        out[self.g.user_slices(loc)] = a
        return out

    def set_fields(self, level, T, ur, uth, uph, p, aux=None):
        """User layout in (see workloads.py).  Sets u1 = u2 = u and p1 = p2 = p
        unless ``aux`` = (ur1, uth1, uph1, p1) is given, then fills every
        boundary value by the exchange (and the pressure ring, if step 7 is on)."""
        L = self.lev[level]
        L.T = self._to_padded(C, T)
        u = [self._to_padded(R, ur), self._to_padded(TH, uth), self._to_padded(PH, uph)]
        L.u2 = [a.copy() for a in u]
        L.p2 = self._to_padded(C, p)
        if aux is None:
            L.u1 = [a.copy() for a in u]
            L.p1 = L.p2.copy()
        else:
            L.u1 = [self._to_padded(R, aux[0]), self._to_padded(TH, aux[1]), self._to_padded(PH, aux[2])]
            L.p1 = self._to_padded(C, aux[3])
        self._refresh(L, (0, 1), self.t - level * self.prm.dt)
        if level == 0 and not self.level1_set:
            self.lev[1] = L.copy()
        if level == 1:
            self.level1_set = True

    def _walls(self, t):
        """Wall data at time t: (T_walls, U_walls) for the exchange; the
        constant wall temperatures and steady wall velocity plus the
        time-dependent mode tau(t) W."""
        prm = self.prm
        T_walls, U_walls = (prm.T_in, prm.T_out), prm.wall_u
        if prm.wall_mode is not None:
            tid, W = prm.wall_mode
            c = _time_fn(tid, t)
            if W.get("T") is not None:
                T_walls = tuple(T_walls[w] + c * np.asarray(W["T"][w]) for w in range(2))
            if any(W.get(k) is not None for k in ("ur", "uth", "uph")):
                base = U_walls
                U_walls = {}
                for k, n in (("ur", (self.g.Nth, self.g.Nph)), ("uth", (self.g.Nth + 1, self.g.Nph)),
                             ("uph", (self.g.Nth, self.g.Nph + 1))):
                    a = np.zeros((2, 2) + n) if base is None or base.get(k) is None else np.asarray(base[k])
                    if W.get(k) is not None:
                        a = a + c * np.asarray(W[k])
                    U_walls[k] = a
        return T_walls, U_walls

    def _refresh(self, L, patches, t):
        d = L.as_dict()
        T_walls, U_walls = self._walls(t)
        xch.exchange_into(self.tables, d, d, patches, T_walls, U_walls, self._step4(),
                          (self.prm.Tbc_in, self.prm.Tbc_out))
        if self.prm.step7:
            xch.pressure_ring(self.tables, L.p1, patches)
            xch.pressure_ring(self.tables, L.p2, patches)

    def get_fields(self, level, aux=False):
        L = self.lev[level]
        g = self.g
        out = {"T": L.T[g.user_slices(C)].copy(), "ur": L.u2[0][g.user_slices(R)].copy(),
               "uth": L.u2[1][g.user_slices(TH)].copy(), "uph": L.u2[2][g.user_slices(PH)].copy(),
               "p": L.p2[g.user_slices(C)].copy()}
        if aux:
            out["ur1"] = L.u1[0][g.user_slices(R)].copy()
            out["uth1"] = L.u1[1][g.user_slices(TH)].copy()
            out["uph1"] = L.u1[2][g.user_slices(PH)].copy()
            out["p1"] = L.p1[g.user_slices(C)].copy()
        return out

    def set_forcing(self, tid, fT, fr, fth, fph):
        """One separable forcing mode tau_tid(t) F(x); arrays in user layout."""
        g = self.g
        def compact(loc, a):
            return view(self._to_padded(loc, a), g.region(loc)).copy()
        self.modes.append((tid, {"T": compact(C, fT), "ur": compact(R, fr),
                                 "uth": compact(TH, fth), "uph": compact(PH, fph)}))

    def forcing(self, t):
        g = self.g
        f = {"T": np.zeros(view(g.zeros(), g.region(C)).shape),
             "ur": np.zeros(view(g.zeros(), g.region(R)).shape),
             "uth": np.zeros(view(g.zeros(), g.region(TH)).shape),
             "uph": np.zeros(view(g.zeros(), g.region(PH)).shape)}
        for tid, F in self.modes:
            c = _time_fn(tid, t)
            for key in f:
                f[key] = f[key] + c * F[key]
        return f

    # ------------------------------------------------------------ the step
    def step(self, n_steps=1, n_schwarz=3):
        for _ in range(n_steps):
            self._one_step(n_schwarz)

    def _step4(self):
        return (self.prm.step4_eps, self.prm.step4_tol) if self.prm.step4 else None

    def _factors(self, A):
        prm, g = self.prm, self.g
        fac = {}
        for loc in (C, R, TH, PH):
            nu = prm.kappa if loc == C else prm.Pr
            gam = (xch.robin_ghost(*prm.Tbc_in, float(g.h_f(0)))[0],
                   xch.robin_ghost(*prm.Tbc_out, float(g.h_f(g.Nr)))[0])
            fac[loc] = {d: ops.factor(g, loc, d, A, prm.dt, nu, prm.chi, gam) for d in "rtp"}
        return fac

    def _one_step(self, K):
        prm, g = self.prm, self.g
        n, nm1 = self.lev
        dt = prm.dt
        # extrapolations (Sec. 3.1 notation w^{*,k+1/2} = 3w^k/2 - w^{k-1}/2)
        A = [1.5 * n.u2[m] - 0.5 * nm1.u2[m] for m in range(3)]
        it = Level(2.0 * n.T - nm1.T, [2.0 * n.u1[m] - nm1.u1[m] for m in range(3)],
                   [2.0 * n.u2[m] - nm1.u2[m] for m in range(3)],
                   2.0 * n.p1 - nm1.p1, 2.0 * n.p2 - nm1.p2)
        f = self.forcing(self.t + 0.5 * dt)
        fac = self._factors(A)
        T_walls, U_walls = self._walls(self.t + dt)     # the new level's wall data
        self.iters_done = 0
        for k in range(1, K + 1):
            if prm.schwarz_mode == "additive":
                d = it.as_dict()
                xch.exchange_into(self.tables, d, d, (0, 1), T_walls, U_walls, self._step4(),
                                  (prm.Tbc_in, prm.Tbc_out))
                norms = self._iterate(it, n, A, f, fac, (0, 1))
                if prm.step7:
                    xch.pressure_ring(self.tables, it.p1, (0, 1))
                    xch.pressure_ring(self.tables, it.p2, (0, 1))
            elif prm.schwarz_mode == "multiplicative":
                norms = np.zeros(len(FIELD_NAMES))
                for p in (0, 1):
                    d = it.as_dict()
                    xch.exchange_into(self.tables, d, d, (p,), T_walls, U_walls, self._step4(),
                                      (prm.Tbc_in, prm.Tbc_out))
                    norms += self._iterate(it, n, A, f, fac, (p,)) ** 2
                    if prm.step7:
                        xch.pressure_ring(self.tables, it.p1, (p,))
                        xch.pressure_ring(self.tables, it.p2, (p,))
                norms = np.sqrt(norms)
            else:
                raise ValueError(prm.schwarz_mode)
            self.last_norms = norms
            self.iters_done = k
            if prm.schwarz_tol > 0 and norms.max() < prm.schwarz_tol:
                break
        self._refresh(it, (0, 1), self.t + dt)
        self.lev = [it, n]
        self.t += dt
        self.steps_done += 1

    def _iterate(self, it, n, A, f, fac, patches):
        """One defect-correction pass over T, u_1, p_1, u_2, p_2 on ``patches``;
        returns the l2 norms of the increments in FIELD_NAMES order."""
        prm, g = self.prm, self.g
        dt, chi, nu = prm.dt, prm.chi, prm.Pr
        mask = np.zeros((2, 1, 1, 1))
        mask[list(patches)] = 1.0
        norms = []

        def norm(loc, c):
            return np.sqrt(np.sum(mask * g.weight(loc) * c * c))

        def advance(arr, arr_n, loc, rate):
            res = dt * rate - (view(arr, g.region(loc)) - view(arr_n, g.region(loc)))
            c = solve_factored(fac[loc], ops.ORDER[loc], res) * mask
            view(arr, g.region(loc))[...] += c
            return norm(loc, c)

        # temperature
        Xh = 0.5 * (it.T + n.T)
        norms.append(advance(it.T, n.T, C, ops.rate_T(g, Xh, A, f["T"], prm.kappa)))
        PrRa = prm.Pr * prm.Ra
        for s in (1, 2):
            U = it.u1 if s == 1 else it.u2
            Un = n.u1 if s == 1 else n.u2
            P = n.p1 if s == 1 else n.p2 + 0.5 * (it.p1 - n.p1)
            Tb = 0.5 * (it.T + n.T)
            for comp, loc, key in ((0, R, "ur"), (1, TH, "uth"), (2, PH, "uph")):
                Uh = [0.5 * (U[m] + Un[m]) for m in range(3)]
                D = ops.padded(g, ops.divergence(g, Uh))
                if comp == 0:
                    rate = ops.rate_ur(g, Uh, A, P, D, Tb, f[key], nu, chi, PrRa)
                elif comp == 1:
                    rate = ops.rate_ut(g, Uh, A, P, D, f[key], nu, chi)
                else:
                    rate = ops.rate_up(g, Uh, A, P, D, f[key], nu, chi)
                norms.append(advance(U[comp], Un[comp], loc, rate))
            Uh = [0.5 * (U[m] + Un[m]) for m in range(3)]
            div = ops.divergence(g, Uh)
            if s == 1:
                pnew = view(n.p1, g.region(C)) - div / chi
                pold = it.p1
            else:
                pnew = (view(n.p2, g.region(C)) + (view(it.p1, g.region(C)) - view(n.p1, g.region(C)))
                        - div / chi)
                pold = it.p2
            c = (pnew - view(pold, g.region(C))) * mask
            view(pold, g.region(C))[...] = np.where(mask > 0, pnew, view(pold, g.region(C)))
            if prm.step7:
                # the ring is overwritten by interpolation afterwards: its
                # increment is not an iteration increment
                c = c * self._ring_off
            norms.append(norm(C, c))
        # reorder to FIELD_NAMES: T, u1r, u1t, u1p, p1, u2r, u2t, u2p, p2
        return np.array(norms)
