"""Seeded, synthetic inputs for the Yin-Yang shell solver.

This module is shared by the oracle tests and the CUDA tests.  It holds the
*problem* (exact manufactured solutions of the continuous
Navier-Stokes-Boussinesq system, their forcing, seeded perturbations and shell
ensembles) and none of the discretisation: no difference stencil, no line
solve, no interpolation.  Exact solutions are written in global Cartesian
coordinates; their derivatives come from a small second-order forward-mode
automatic differentiation (value, gradient, Hessian), so the forcing of a
manufactured solution is derived without any spherical metric formula.

Continuous problem (Sec. 1, Eq. eq_ns / eq_heat_convec):
    du/dt + (u.grad)u + grad p - Pr lap u = Pr Ra T g + f_u,   div u = 0
    dT/dt + u.grad T - lap T = f_T
with g the unit vector opposite to gravity, read as +e_r, and Dirichlet walls.

Grid geometry (Sec. 2): each patch spans r in [R1, R2],
theta in [pi/4 - d, 3pi/4 + d], phi in [-3pi/4 - d, 3pi/4 + d] of its own
frame, with d = overlap_cells * h_theta, h_theta = (pi/2)/(N_theta - 2*overlap)
and h_phi = (3pi/2 + 2d)/N_phi.  The Yang frame is the Yin frame composed with
M(x, y, z) = (-x, z, y).

User field layout (both patches, patch index first, phi fastest):
    T, p : (2, Nr,   Nth,   Nph)   cell centres
    ur   : (2, Nr+1, Nth,   Nph)   r-faces (wall faces included)
    uth  : (2, Nr,   Nth+1, Nph)   theta-faces (patch-edge faces included)
    uph  : (2, Nr,   Nth,   Nph+1) phi-faces (patch-edge faces included)
Velocity components are in each patch's local spherical basis.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass
from typing import Optional

import numpy as np

# time-function ids of separable forcing modes: f(x, t) = sum_m tau_m(t) F_m(x)
TIME_FNS = {0: "1", 1: "cos t", 2: "sin t", 3: "cos^2 t", 4: "sin t cos t"}


def time_fn(tid: int, t: float) -> float:
    """Value of the time function with id ``tid`` at time ``t``."""
    if tid == 0:
        return 1.0
    if tid == 1:
        return math.cos(t)
    if tid == 2:
        return math.sin(t)
    if tid == 3:
        return math.cos(t) ** 2
    if tid == 4:
        return math.sin(t) * math.cos(t)
    raise ValueError(f"unknown time function {tid}")


# --------------------------------------------------------------------------
# grid points of the problem statement
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Spec:
    """Shell and grid parameters shared by every workload."""
    R1: float
    R2: float
    Nr: int
    Nth: int
    Nph: int
    overlap: int = 2
    # radii of the 2 Nr + 1 radial half points (faces at even, centres at odd
    # positions); None = uniform radial grid
    r_half: Optional[tuple] = None

    @property
    def hr(self):
        return (self.R2 - self.R1) / self.Nr

    @property
    def hth(self):
        return (math.pi / 2) / (self.Nth - 2 * self.overlap)

    @property
    def delta(self):
        return self.overlap * self.hth

    @property
    def hph(self):
        return (1.5 * math.pi + 2 * self.delta) / self.Nph

    @property
    def th0(self):
        return math.pi / 4 - self.delta

    @property
    def ph0(self):
        return -0.75 * math.pi - self.delta

    def shape(self, loc: str):
        Nr, Nt, Np = self.Nr, self.Nth, self.Nph
        return {"c": (2, Nr, Nt, Np), "r": (2, Nr + 1, Nt, Np),
                "t": (2, Nr, Nt + 1, Np), "p": (2, Nr, Nt, Np + 1)}[loc]

    def coords(self, loc: str):
        """Local (r, theta, phi) of every user-layout point of location type
        ``loc`` ('c' centre, 'r'/'t'/'p' face normal to r/theta/phi), as
        broadcastable arrays of shape (1, ni, 1, 1), (1, 1, nj, 1), (1, 1, 1, nk)."""
        Nr, Nt, Np = self.Nr, self.Nth, self.Nph
        ri = np.arange(Nr + 1 if loc == "r" else Nr, dtype=np.float64)
        tj = np.arange(Nt + 1 if loc == "t" else Nt, dtype=np.float64)
        pk = np.arange(Np + 1 if loc == "p" else Np, dtype=np.float64)
        if self.r_half is None:
            r = self.R1 + (ri + (0.0 if loc == "r" else 0.5)) * self.hr
        else:
            r = np.asarray(self.r_half, dtype=np.float64)[2 * ri.astype(int) + (0 if loc == "r" else 1)]
        th = self.th0 + (tj + (0.0 if loc == "t" else 0.5)) * self.hth
        ph = self.ph0 + (pk + (0.0 if loc == "p" else 0.5)) * self.hph
        return r[None, :, None, None], th[None, None, :, None], ph[None, None, None, :]


def stretched_radii(R1, R2, Nr, beta):
    """Radii of the 2 Nr + 1 half points of a smoothly stretched radial grid:
    r(xi) = R1 + (R2 - R1) (xi - beta sin(2 pi xi) / (2 pi)) at xi = m / (2 Nr),
    cells finer near both walls (spacing ratio (1 - beta) / (1 + beta) between
    the walls and mid-shell), 0 <= beta < 1."""
    xi = np.arange(2 * Nr + 1) / (2.0 * Nr)
    r = R1 + (R2 - R1) * (xi - beta * np.sin(2.0 * math.pi * xi) / (2.0 * math.pi))
    r[0], r[-1] = R1, R2
    return tuple(r.tolist())


def local_basis(th, ph):
    """Local spherical unit vectors (e_r, e_theta, e_phi) in local Cartesian
    components, each a tuple of three arrays."""
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    er = (st * cp, st * sp, ct + 0 * ph)
    et = (ct * cp, ct * sp, -st + 0 * ph)
    ep = (-sp + 0 * th, cp + 0 * th, 0 * th + 0 * ph)
    return er, et, ep


def global_points(spec: Spec, loc: str):
    """Global Cartesian coordinates (x, y, z), each of the user-layout shape
    of ``loc``; patch 0 is Yin, patch 1 is Yang = M applied to the Yin formula."""
    r, th, ph = spec.coords(loc)
    shp = spec.shape(loc)
    xl = np.broadcast_to((r * np.sin(th) * np.cos(ph))[0], shp[1:])
    yl = np.broadcast_to((r * np.sin(th) * np.sin(ph))[0], shp[1:])
    zl = np.broadcast_to((r * np.cos(th) + 0 * ph)[0], shp[1:])
    x = np.stack([xl, -xl])
    y = np.stack([yl, zl])
    z = np.stack([zl, yl])
    return x, y, z


def to_local_components(spec: Spec, loc: str, v):
    """Project a global Cartesian vector field v = (vx, vy, vz) sampled at the
    ``loc`` points onto each patch's local spherical basis; returns
    (v_r, v_theta, v_phi)."""
    r, th, ph = spec.coords(loc)
    er, et, ep = local_basis(th[0], ph[0])
    vx, vy, vz = v
    # local Cartesian components: Yin = global, Yang = M (global), M = M^-1
    lx = np.stack([vx[0], -vx[1]])
    ly = np.stack([vy[0], vz[1]])
    lz = np.stack([vz[0], vy[1]])
    out = []
    for e in (er, et, ep):
        out.append(lx * e[0] + ly * e[1] + lz * e[2])
    return out


# --------------------------------------------------------------------------
# second-order forward-mode AD in (x, y, z)
# --------------------------------------------------------------------------
class Jet:
    """f together with its gradient g[..., 3] and Hessian H[..., 3, 3]."""

    __slots__ = ("v", "g", "H")

    def __init__(self, v, g, H):
        self.v, self.g, self.H = v, g, H

    @staticmethod
    def variables(x, y, z):
        x, y, z = (np.asarray(a, dtype=np.float64) for a in (x, y, z))
        shp = x.shape
        out = []
        for m, a in enumerate((x, y, z)):
            g = np.zeros(shp + (3,))
            g[..., m] = 1.0
            out.append(Jet(a.copy(), g, np.zeros(shp + (3, 3))))
        return out

    @staticmethod
    def _lift(o, like):
        if isinstance(o, Jet):
            return o
        v = np.broadcast_to(np.asarray(o, dtype=np.float64), like.v.shape)
        return Jet(v, np.zeros(like.g.shape), np.zeros(like.H.shape))

    def __add__(self, o):
        o = Jet._lift(o, self)
        return Jet(self.v + o.v, self.g + o.g, self.H + o.H)

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, -self.g, -self.H)

    def __sub__(self, o):
        return self + (-Jet._lift(o, self))

    def __rsub__(self, o):
        return Jet._lift(o, self) - self

    def __mul__(self, o):
        if not isinstance(o, Jet):
            c = np.asarray(o, dtype=np.float64)
            return Jet(self.v * c, self.g * c[..., None] if c.ndim else self.g * c,
                       self.H * c[..., None, None] if c.ndim else self.H * c)
        v = self.v * o.v
        g = self.g * o.v[..., None] + o.g * self.v[..., None]
        H = (self.H * o.v[..., None, None] + o.H * self.v[..., None, None]
             + self.g[..., :, None] * o.g[..., None, :] + o.g[..., :, None] * self.g[..., None, :])
        return Jet(v, g, H)

    __rmul__ = __mul__

    def _chain(self, f0, f1, f2):
        g = self.g * f1[..., None]
        H = self.H * f1[..., None, None] + f2[..., None, None] * self.g[..., :, None] * self.g[..., None, :]
        return Jet(f0, g, H)

    def recip(self):
        v = self.v
        return self._chain(1.0 / v, -1.0 / v ** 2, 2.0 / v ** 3)

    def __truediv__(self, o):
        if not isinstance(o, Jet):
            return self * (1.0 / np.asarray(o, dtype=np.float64))
        return self * o.recip()

    def __rtruediv__(self, o):
        return Jet._lift(o, self) * self.recip()

    def sin(self):
        return self._chain(np.sin(self.v), np.cos(self.v), -np.sin(self.v))

    def cos(self):
        return self._chain(np.cos(self.v), -np.sin(self.v), -np.cos(self.v))

    def exp(self):
        e = np.exp(self.v)
        return self._chain(e, e, e)

    def sqrt(self):
        s = np.sqrt(self.v)
        return self._chain(s, 0.5 / s, -0.25 / (s * self.v))

    def lap(self):
        return self.H[..., 0, 0] + self.H[..., 1, 1] + self.H[..., 2, 2]


# --------------------------------------------------------------------------
# exact solutions (time factor separated: u = c_u(t) U(x), T = c_T(t) Th(x),
# p = c_p(t) P(x))
# --------------------------------------------------------------------------
class Exact:
    """A manufactured solution of the continuous problem."""

    name = "base"
    time_fn = 1  # cos t, unless overridden

    def __init__(self, R1, R2, Pr, Ra):
        self.R1, self.R2, self.Pr, self.Ra = R1, R2, Pr, Ra

    def s_of_r(self, r, F):
        """Wall-vanishing radial profile sin(pi (r - R1)/(R2 - R1))."""
        L = self.R2 - self.R1
        return F.sin((r - self.R1) * (math.pi / L))

    def ds_of_r(self, r, F):
        L = self.R2 - self.R1
        return F.cos((r - self.R1) * (math.pi / L)) * (math.pi / L)

    def fields(self, x, y, z, F):
        """Spatial parts (U[3], P, Th) of global Cartesian x, y, z, written with
        the functions of namespace F (numpy, sympy or the Jet namespace)."""
        raise NotImplementedError

    def tfac(self, t):
        return time_fn(self.time_fn, t)


class TrigShell(Exact):
    """Trigonometric solution with homogeneous walls:
    s(r) = sin(pi (r-R1)/(R2-R1)),  u = c0 grad(s^2) x grad(x^2 + y z)
    T = s(r) (xy + yz + zx) / r^2,  p = x y z / r^3, all times cos t.
    u is tangential and divergence-free."""

    name = "trig"
    c0 = 0.25

    def fields(self, x, y, z, F):
        r = F.sqrt(x * x + y * y + z * z)
        s, ds = self.s_of_r(r, F), self.ds_of_r(r, F)
        q = 2.0 * s * ds / r * self.c0
        # x_vec cross grad(x^2 + y z) = (y^2 - z^2, 2 x z - x y, x z - 2 x y)
        U = [q * (y * y - z * z), q * (2.0 * x * z - x * y), q * (x * z - 2.0 * x * y)]
        Th = s * (x * y + y * z + z * x) / (r * r)
        P = x * y * z / (r * r * r)
        return U, P, Th


class CurlShell(Exact):
    """Solution with a non-zero radial velocity and homogeneous walls:
    u = c0 curl(s(r)^2 A),  A = (sin(k y), sin(k z), sin(k x)),
    T = s(r) cos(x) sin(y + z),  p = sin(x) cos(y) + z^2 / 2, all times cos t.
    curl(q A) = q curl A + grad q x A with curl A = -k (cos kz, cos kx, cos ky)."""

    name = "curl"
    c0 = 1.0
    k = 1.3

    def fields(self, x, y, z, F):
        k = self.k
        r = F.sqrt(x * x + y * y + z * z)
        s, ds = self.s_of_r(r, F), self.ds_of_r(r, F)
        q = s * s
        dq_over_r = 2.0 * s * ds / r           # grad q = dq_over_r * (x, y, z)
        Ax, Ay, Az = F.sin(y * k), F.sin(z * k), F.sin(x * k)
        cA = [F.cos(z * k) * (-k), F.cos(x * k) * (-k), F.cos(y * k) * (-k)]
        cross = [y * Az - z * Ay, z * Ax - x * Az, x * Ay - y * Ax]
        U = [(q * cA[m] + dq_over_r * cross[m]) * self.c0 for m in range(3)]
        Th = s * F.cos(x) * F.sin(y + z)
        P = F.sin(x) * F.cos(y) + 0.5 * z * z
        return U, P, Th


class RadialHeat(Exact):
    """Closed-form heat solution T = sin(pi (r-R1)/L)/r exp(-(pi/L)^2 t) of
    dT/dt = lap T with T = 0 on both walls, u = 0, p = 0 (Ra = 0).
    lap(g(r)/r) = g''(r)/r, so it needs no forcing."""

    name = "radial_heat"

    def fields(self, x, y, z, F):
        r = F.sqrt(x * x + y * y + z * z)
        zero = r * 0.0
        return [zero, zero, zero], zero, self.s_of_r(r, F) / r

    def tfac(self, t):
        L = self.R2 - self.R1
        return math.exp(-((math.pi / L) ** 2) * t)


class RadialHeatRobin(Exact):
    """Closed-form heat solution with T = 0 at r = R1 and the homogeneous Robin
    condition a T + b dT/dn = 0 at r = R2 (n = e_r there; b = 1, a = 0 is
    Neumann): T = sin(k (r - R1)) / r exp(-k^2 t), lap(g(r)/r) = g''/r, with k
    the smallest positive root of
      a R2 sin(k L) + b (k R2 cos(k L) - sin(k L)) = 0,  L = R2 - R1
    (R2^2 times the condition: dT/dr = (k r cos - sin) / r^2 at r = R2).
    u = 0, p = 0, Ra = 0: no forcing."""

    name = "radial_heat_robin"
    a, b = 0.0, 1.0

    def __init__(self, R1, R2, Pr, Ra, a=0.0, b=1.0):
        super().__init__(R1, R2, Pr, Ra)
        self.a, self.b = a, b
        L = R2 - R1
        f = lambda k: a * R2 * math.sin(k * L) + b * (k * R2 * math.cos(k * L) - math.sin(k * L))
        # bracket the first sign change above k = 0+ and bisect
        lo, step = 1e-6, 1e-3
        while f(lo) * f(lo + step) > 0:
            lo += step
        hi = lo + step
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if f(lo) * f(mid) <= 0:
                hi = mid
            else:
                lo = mid
        self.k = 0.5 * (lo + hi)

    def fields(self, x, y, z, F):
        r = F.sqrt(x * x + y * y + z * z)
        zero = r * 0.0
        return [zero, zero, zero], zero, F.sin((r - self.R1) * self.k) / r

    def tfac(self, t):
        return math.exp(-(self.k ** 2) * t)


class SymmetricShell(Exact):
    """Data invariant under M(x, y, z) = (-x, z, y): a scalar f(MX) = f(X) and
    a vector v(MX) = M v(X).  Used for Yin/Yang congruence.
    f = s(r) (x^2 + y z),  u = c0 grad f x grad h with h = s(r)^2 (x^2 + 2 y z)."""

    name = "symmetric"
    c0 = 0.5

    def fields(self, x, y, z, F):
        r = F.sqrt(x * x + y * y + z * z)
        s, ds = self.s_of_r(r, F), self.ds_of_r(r, F)
        # f = s * g1, g1 = x^2 + y z ; h = s^2 * g2, g2 = x^2 + 2 y z
        g1 = x * x + y * z
        g2 = x * x + 2.0 * y * z
        dg1 = [2.0 * x, z, y]
        dg2 = [2.0 * x, 2.0 * z, 2.0 * y]
        X = [x, y, z]
        gf = [ds / r * X[m] * g1 + s * dg1[m] for m in range(3)]
        gh = [2.0 * s * ds / r * X[m] * g2 + s * s * dg2[m] for m in range(3)]
        U = [(gf[1] * gh[2] - gf[2] * gh[1]) * self.c0,
             (gf[2] * gh[0] - gf[0] * gh[2]) * self.c0,
             (gf[0] * gh[1] - gf[1] * gh[0]) * self.c0]
        Th = s * g1
        P = g1 * r
        return U, P, Th


class LandauJet(Exact):
    """Landau's round jet (the steady solution used in Sec. 5.1), axisymmetric
    about the global z-axis, with nu = Pr and jet parameter A > 1: stream
    function psi = 2 nu r sin^2(theta) / (A - cos theta), so
      u_r = (2 nu / r) ((A^2 - 1) / (A - cos theta)^2 - 1),
      u_theta = -(2 nu / r) sin(theta) / (A - cos theta),
      p = 4 nu^2 (A cos theta - 1) / (r^2 (A - cos theta)^2),  T = 0.
    Steady (time factor 1); needs the wall velocity of the formula (wall_velocity)."""

    name = "landau"
    time_fn = 0
    A = 2.0

    def fields(self, x, y, z, F):
        nu, A = self.Pr, self.A
        r = F.sqrt(x * x + y * y + z * z)
        c = z / r
        w = A - c
        ur = (2.0 * nu) / r * ((A * A - 1.0) / (w * w) - 1.0)
        # u_theta e_theta = -(2 nu / (r (A - c))) (z x / r^2, z y / r^2, -(x^2 + y^2) / r^2)
        g = (-2.0 * nu) / (r * w) / (r * r)
        U = [ur * x / r + g * (z * x), ur * y / r + g * (z * y), ur * z / r - g * (x * x + y * y)]
        P = (4.0 * nu * nu) * (A * c - 1.0) / (r * r * w * w)
        Th = x * 0.0
        return U, P, Th


class PaperShell(Exact):
    """The manufactured solution of Sec. 5.1, given in Cartesian form:
      u = cos t (2 x^2 y z, -x y^2 z, -x y z^2),  p = cos t x y z,
      T = 2 cos t x^2 y z,
    divergence-free (4xyz - 2xyz - 2xyz = 0), with time-dependent,
    non-zero velocity and temperature on both walls (the paper runs it with
    R1 = 1, R2 = 2, Ra = Pr = 1): it needs the wall data of wall_velocity and
    wall_temperature, which follow cos t."""

    name = "paper"

    def fields(self, x, y, z, F):
        U = [2.0 * x * x * y * z, -x * y * y * z, -x * y * z * z]
        return U, x * y * z, 2.0 * x * x * y * z


EXACT = {c.name: c for c in (TrigShell, CurlShell, RadialHeat, RadialHeatRobin, SymmetricShell, LandauJet,
                             PaperShell)}


def wall_temperature(ex: Exact, spec: Spec, t: float = 0.0):
    """Temperature of ``ex`` on the walls r = R1 and r = R2 at the cell-centre
    angles of each patch: array [2 walls][2 patches][Nth][Nph]."""
    c = ex.tfac(t)
    _, th, ph = spec.coords("c")
    th2, ph2 = th[0, 0], ph[0, 0]
    walls = []
    for R in (spec.R1, spec.R2):
        xl = R * np.sin(th2) * np.cos(ph2)
        yl = R * np.sin(th2) * np.sin(ph2)
        zl = R * np.cos(th2) + 0.0 * ph2
        x, y, z = np.stack([xl, -xl]), np.stack([yl, zl]), np.stack([zl, yl])
        _, _, Th = ex.fields(x, y, z, np)
        walls.append(np.broadcast_to(Th, x.shape) * c)
    return np.stack(walls)


def wall_velocity(ex: Exact, spec: Spec, t: float = 0.0):
    """Velocity of ``ex`` on the walls r = R1 and r = R2 in each patch's local
    basis, at every face point of the wall planes: dict 'ur' [2 walls][2
    patches][Nth][Nph], 'uth' [..][Nth+1][Nph], 'uph' [..][Nth][Nph+1]."""
    c = ex.tfac(t)
    out = {}
    for key, loc, comp in (("ur", "c", 0), ("uth", "t", 1), ("uph", "p", 2)):
        _, th, ph = spec.coords(loc)
        th2, ph2 = th[0, 0], ph[0, 0]
        er, et, ep = local_basis(th2, ph2)
        walls = []
        for R in (spec.R1, spec.R2):
            xl = R * np.sin(th2) * np.cos(ph2)
            yl = R * np.sin(th2) * np.sin(ph2)
            zl = R * np.cos(th2) + 0.0 * ph2
            x, y, z = np.stack([xl, -xl]), np.stack([yl, zl]), np.stack([zl, yl])
            U, _, _ = ex.fields(x, y, z, np)
            U = [np.broadcast_to(u, x.shape) for u in U]
            lx, ly, lz = np.stack([U[0][0], -U[0][1]]), np.stack([U[1][0], U[2][1]]), np.stack([U[2][0], U[1][1]])
            e = (er, et, ep)[comp]
            walls.append((lx * e[0] + ly * e[1] + lz * e[2]) * c)
        out[key] = np.stack(walls)
    return out


class JetNS:
    """Function namespace acting on Jets (for fields(..., F=JetNS))."""
    sin = staticmethod(lambda a: a.sin())
    cos = staticmethod(lambda a: a.cos())
    sqrt = staticmethod(lambda a: a.sqrt())
    exp = staticmethod(lambda a: a.exp())


def _jets_at(ex: Exact, spec: Spec, loc: str):
    x, y, z = global_points(spec, loc)
    X, Y, Z = Jet.variables(x, y, z)
    return ex.fields(X, Y, Z, JetNS)


def sample_fields(ex: Exact, spec: Spec, t: float):
    """Exact T, u (local components at their own MAC points) and p at time t,
    in the user layout: dict with keys T, ur, uth, uph, p."""
    c = ex.tfac(t)
    out = {}
    x, y, z = global_points(spec, "c")
    U, P, Th = ex.fields(x, y, z, np)
    out["T"] = np.broadcast_to(Th * c, spec.shape("c")).copy()
    out["p"] = np.broadcast_to(P * c, spec.shape("c")).copy()
    for loc, key, comp in (("r", "ur", 0), ("t", "uth", 1), ("p", "uph", 2)):
        x, y, z = global_points(spec, loc)
        U, _, _ = ex.fields(x, y, z, np)
        U = [np.broadcast_to(u, x.shape) for u in U]
        out[key] = to_local_components(spec, loc, U)[comp] * c
    return out


_FORCING_FNS = {}


def _forcing_fns(ex: Exact):
    """Symbolic forcing of a cos-t solution, compiled to numpy:
      f_u = -sin t U + cos^2 t (U.grad)U + cos t (grad P - Pr lap U - Pr Ra Th e_r)
      f_T = -sin t Th + cos^2 t U.grad Th + cos t (-lap Th)
    Returns a function (x, y, z) -> 12 arrays: (f_sin, f_cos2, f_cos) x (u_x, u_y, u_z, T)."""
    key = (type(ex).__name__, ex.R1, ex.R2, ex.Pr, ex.Ra)
    if key in _FORCING_FNS:
        return _FORCING_FNS[key]
    import sympy as sp
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)
    U, P, Th = ex.fields(x, y, z, sp)
    r = sp.sqrt(x * x + y * y + z * z)
    er = (x / r, y / r, z / r)
    lap = lambda f: sum(sp.diff(f, v, 2) for v in X)
    Pr, Ra = ex.Pr, ex.Ra
    f_sin = [-U[m] for m in range(3)] + [-Th]
    f_cos2 = [sum(U[n] * sp.diff(U[m], X[n]) for n in range(3)) for m in range(3)]
    f_cos2.append(sum(U[m] * sp.diff(Th, X[m]) for m in range(3)))
    f_cos = [sp.diff(P, X[m]) - Pr * lap(U[m]) - Pr * Ra * Th * er[m] for m in range(3)] + [-lap(Th)]
    fn = sp.lambdify((x, y, z), f_sin + f_cos2 + f_cos, modules="numpy", cse=True)
    _FORCING_FNS[key] = fn
    return fn


def forcing_modes(ex: Exact, spec: Spec, chunk: int = 1 << 18):
    """Separable forcing of a cos-t manufactured solution, as a list of
    (time_fn_id, fields) with fields = dict(T, ur, uth, uph) in user layout.

    With u = cos t U, p = cos t P, T = cos t Th:
      f_u = -sin t U + cos^2 t (U.grad)U + cos t (grad P - Pr lap U - Pr Ra Th e_r)
      f_T = -sin t Th + cos^2 t U.grad Th + cos t (-lap Th).
    Derivatives are taken symbolically in Cartesian coordinates."""
    if ex.time_fn != 1 or isinstance(ex, RadialHeat):
        raise ValueError("forcing_modes needs a cos-t solution")
    fn = _forcing_fns(ex)
    tids = (2, 3, 1)
    modes = {tid: {} for tid in tids}
    for loc, key, comp in (("c", "T", None), ("r", "ur", 0), ("t", "uth", 1), ("p", "uph", 2)):
        x, y, z = global_points(spec, loc)
        xf, yf, zf = x.ravel(), y.ravel(), z.ravel()
        vals = [np.empty(xf.size) for _ in range(12)]

        def work(a):
            b = min(a + chunk, xf.size)
            out = fn(xf[a:b], yf[a:b], zf[a:b])
            for m in range(12):
                vals[m][a:b] = out[m]
        # numpy releases the GIL inside ufuncs: chunks evaluate in parallel
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as pool:
            list(pool.map(work, range(0, xf.size, chunk)))
        vals = [v.reshape(x.shape) for v in vals]
        for g, tid in enumerate(tids):
            blk = vals[4 * g:4 * g + 4]
            if comp is None:
                modes[tid][key] = blk[3]
            else:
                modes[tid][key] = to_local_components(spec, loc, blk[:3])[comp]
    return [(tid, modes[tid]) for tid in (1, 2, 3)]


def exact_rates(ex: Exact, spec: Spec, loc: str, t: float, Pr: float, Ra: float, chi: float,
                a_ex: Exact | None = None):
    """Continuous operators at the ``loc`` points, for pinning discrete stencils.

    Returns a dict of local-basis values (all at time t):
      'vlap'  : vector Laplacian of u written with the continuity substitution
                used by the momentum rows (Sec. 3.3.1-3.3.3): lap_vec u
                + (2/r) div u e_r + (2 cot(theta)/r) div u e_theta
      'adv'   : (a.grad) u  (a = a_ex's velocity, default u itself)
      'gradp' : grad p
      'graddiv': grad(div u)
      'buoy'  : Pr Ra T e_r
      'lapT', 'advT' : lap T and a.grad T (scalar, only for loc 'c')
      'div'   : div u (scalar)."""
    c = ex.tfac(t)
    U, P, Th = _jets_at(ex, spec, loc)
    if a_ex is None:
        A = [Ui * c for Ui in U]
    else:
        Ua, _, _ = _jets_at(a_ex, spec, loc)
        ca = a_ex.tfac(t)
        A = [Ui * ca for Ui in Ua]
    x, y, z = global_points(spec, loc)
    rr = np.sqrt(x * x + y * y + z * z)
    er = (x / rr, y / rr, z / rr)
    # cos(theta)/sin(theta) of the local frame
    _, th, _ = spec.coords(loc)
    cot = np.broadcast_to((np.cos(th) / np.sin(th))[0], x.shape[1:])
    div = sum(U[m].g[..., m] for m in range(3)) * c
    out = {"div": div}
    vlap_cart = [U[m].lap() * c for m in range(3)]
    vl = to_local_components(spec, loc, vlap_cart)
    vl[0] = vl[0] + 2.0 / rr * div
    vl[1] = vl[1] + 2.0 * np.stack([cot, cot]) / rr * div
    out["vlap"] = vl
    out["adv"] = to_local_components(
        spec, loc, [sum(A[n].v * U[m].g[..., n] for n in range(3)) * c for m in range(3)])
    out["gradp"] = to_local_components(spec, loc, [P.g[..., m] * c for m in range(3)])
    out["graddiv"] = to_local_components(
        spec, loc, [sum(U[n].H[..., n, m] for n in range(3)) * c for m in range(3)])
    out["buoy"] = to_local_components(spec, loc, [Pr * Ra * Th.v * c * er[m] for m in range(3)])
    out["lapT"] = Th.lap() * c
    out["advT"] = sum(A[m].v * Th.g[..., m] for m in range(3)) * c
    return out


# --------------------------------------------------------------------------
# seeded workloads
# --------------------------------------------------------------------------
def conductive_profile(spec: Spec, T_in: float = 1.0, T_out: float = 0.0):
    """Conductive temperature T_c(r) = A/r + B with T_c(R1) = T_in,
    T_c(R2) = T_out, sampled at cell centres (user layout)."""
    r, _, _ = spec.coords("c")
    A = (T_in - T_out) / (1.0 / spec.R1 - 1.0 / spec.R2)
    B = T_in - A / spec.R1
    return np.broadcast_to(A / r + B, spec.shape("c")).copy()


def convection_perturbation(spec: Spec, seed: int = 3, amp: float = 1e-3, kmax: int = 6):
    """Seeded perturbation sum c_klm sin(k pi (r-R1)/L) cos(m phi) sin(l theta)
    with k, l, m <= kmax and c ~ U(-1, 1), normalised to max |pert| = amp.
    theta, phi are the global (Yin-frame) angles; Yang samples through M."""
    rng = np.random.default_rng(seed)
    coef = rng.uniform(-1.0, 1.0, size=(kmax, kmax, kmax + 1))
    r, _, _ = spec.coords("c")
    x, y, z = global_points(spec, "c")
    rr = np.sqrt(x * x + y * y + z * z)
    gth = np.arccos(np.clip(z / rr, -1.0, 1.0))
    gph = np.arctan2(y, x)
    L = spec.R2 - spec.R1
    # the triple sum contracted point by point: sum_k rad_k sum_l sth_l
    # (sum_m c_klm cph_m), in chunks of points (bounded memory)
    rr, gth, gph = (np.broadcast_to(a, spec.shape("c")).ravel() for a in (rr, gth, gph))
    pert = np.empty(rr.size)
    cmat = coef.reshape(kmax * kmax, kmax + 1).T
    def multiples(x, n, sine):
        """Rows sin(j x), j = 1..n (sine) or cos(j x), j = 0..n, by the
        recurrence f_{j+1} = 2 cos(x) f_j - f_{j-1}."""
        c1 = np.cos(x)
        out = np.empty((n if sine else n + 1, x.size))
        if sine:
            out[0] = np.sin(x)
            prev = np.zeros_like(x)
        else:
            out[0] = 1.0
            out[1] = c1
            prev = out[0]
        for j in range(1, out.shape[0]):
            if not sine and j == 1:
                continue
            out[j] = 2.0 * c1 * out[j - 1] - prev
            prev = out[j - 1]
        return out

    for a in range(0, rr.size, 1 << 20):
        sl = slice(a, a + (1 << 20))
        rad = multiples((rr[sl] - spec.R1) * (math.pi / L), kmax, True)      # (k, p)
        sth = multiples(gth[sl], kmax, True)                                 # (l, p)
        cph = multiples(gph[sl], kmax, False)                                # (m, p)
        A = (cmat.T @ cph).reshape(kmax, kmax, -1)                           # (k, l, p)
        pert[sl] = np.sum(rad * np.einsum("klp,lp->kp", A, sth), axis=0)
    pert = pert.reshape(spec.shape("c"))
    return pert * (amp / np.abs(pert).max())


def shell_ensemble(seed: int = 4, n: int = 64, nr_max: int = 64, nth_max: int = 96):
    """Seeded ensemble of uneven shells: Nr ~ U{16..nr_max}, Nth ~ U{16..nth_max}
    (multiples of 4 are not required), Nph = 3 Nth, R1/R2 ~ U[0.35, 0.6] with
    R2 = 1, Ra log-uniform in [1e3, 1e6], Pr in {0.7, 1, 7}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        Nr = int(rng.integers(16, nr_max + 1))
        Nth = int(rng.integers(16, nth_max + 1))
        ratio = float(rng.uniform(0.35, 0.6))
        Ra = float(10 ** rng.uniform(3.0, 6.0))
        Pr = float(rng.choice([0.7, 1.0, 7.0]))
        out.append(dict(R1=ratio, R2=1.0, Nr=Nr, Nth=Nth, Nph=3 * Nth, Ra=Ra, Pr=Pr))
    return out


def convection_initial(spec: Spec, Pr: float, Ra: float, seed: int = 3, amp: float = 1e-3,
                       T_in: float = 1.0, T_out: float = 0.0, kmax: int = 6):
    """Thermal-convection start (user layout): T = conductive profile + seeded
    perturbation, u = 0, and p in discrete hydrostatic balance with T along
    each radial column, p_{i} - p_{i-1} = h_r Pr Ra (T_{i-1} + T_i)/2, p_0 = 0
    (buoyancy Pr Ra T e_r balanced by the pressure gradient)."""
    T = conductive_profile(spec, T_in, T_out) + convection_perturbation(spec, seed, amp, kmax)
    p = np.zeros_like(T)
    for i in range(1, spec.Nr):
        p[:, i] = p[:, i - 1] + spec.hr * Pr * Ra * 0.5 * (T[:, i - 1] + T[:, i])
    return {"T": T, "ur": np.zeros(spec.shape("r")), "uth": np.zeros(spec.shape("t")),
            "uph": np.zeros(spec.shape("p")), "p": p}
