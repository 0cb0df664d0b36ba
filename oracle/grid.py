"""Yin-Yang grid, MAC placement and metric (oracle; test infrastructure).

Sec. 2: two identical latitude-longitude patches.  Yin uses
x = r sin(th) cos(ph), y = r sin(th) sin(ph), z = r cos(th); Yang uses
x = -r sin(th) cos(ph), y = r cos(th), z = r sin(th) sin(ph), i.e. the Yin map
followed by M(x, y, z) = (-x, z, y).  M is an involution, so it also maps Yang
local Cartesian coordinates back to Yin ones.

Patch extents: the ranges printed in Sec. 2 are garbled (theta cannot exceed
pi); the reading used is theta in [pi/4 - d, 3pi/4 + d],
phi in [-3pi/4 - d, 3pi/4 + d] with one overlap angle d = overlap * h_theta,
h_theta = (pi/2) / (N_theta - 2 overlap), h_phi = (3pi/2 + 2d) / N_phi.

MAC placement (Sec. 4): T and p at cell centres, u_r on r-faces, u_theta on
theta-faces, u_phi on phi-faces, uniform spacing in theta and phi.

Radial grid (Sec. 4 allows a non-uniform grid; its tests use uniform ones):
uniform by default, else given by the radii of all 2 Nr + 1 half points
r_half[m] (faces at even m, centres at odd m; r_half[0] = R1,
r_half[2 Nr] = R2).  The reading taken for "centred differences on a
non-uniform grid" is the stretched-coordinate one: a half-cell difference
divides by the distance between its two points, h_c(i) = r_f(i+1) - r_f(i) at
centre i and h_f(i) = r_c(i) - r_c(i-1) at face i; a whole-cell centred
difference divides by 2 h of its point; averages of radial neighbours stay
arithmetic means.  Ghost half points are the mirror images of the interior
ones about the walls, so that h_f(0) = 2 (r_c(0) - R1).  On a uniform grid
every h is h_r.

Storage: every field of one patch is an array indexed by logical
(i, j, k) in [-1, Nr] x [-1, Nth] x [-1, Nph], stored with offset +1, so a
field array has shape (2, Nr+2, Nth+2, Nph+2) (patch first).  A face index i
names the face at r = R1 + i h_r; a centre index i names r = R1 + (i+1/2) h_r.
"""
from __future__ import annotations

import math

import numpy as np

# location types
C, R, TH, PH = "c", "r", "t", "p"

M = np.array([[-1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, 1.0, 0.0]])


class Grid:
    def __init__(self, R1, R2, Nr, Nth, Nph, overlap=2, r_half=None):
        if not (R1 > 0 and R2 > R1):
            raise ValueError("need 0 < R1 < R2")
        if Nth <= 2 * overlap:
            raise ValueError("N_theta too small for the overlap")
        self.R1, self.R2 = float(R1), float(R2)
        self.Nr, self.Nth, self.Nph = int(Nr), int(Nth), int(Nph)
        self.overlap = int(overlap)
        self.hr = (self.R2 - self.R1) / self.Nr     # the uniform grid's radial spacing
        self.uniform_r = r_half is None
        if r_half is not None:
            rh = np.array(r_half, dtype=np.float64)
            if rh.shape != (2 * self.Nr + 1,) or not np.all(np.diff(rh) > 0):
                raise ValueError("r_half: 2 Nr + 1 strictly increasing radii")
            tol = 1e-12 * (self.R2 - self.R1)
            if abs(rh[0] - self.R1) > tol or abs(rh[-1] - self.R2) > tol:
                raise ValueError("r_half must start at R1 and end at R2")
            rh[0], rh[-1] = self.R1, self.R2
            # 4 ghost half points beyond each wall, mirrored about it
            lo = 2.0 * self.R1 - rh[4:0:-1]
            hi = 2.0 * self.R2 - rh[-2:-6:-1]
            self._rh = np.concatenate([lo, rh, hi])    # half point m at index m + 4
        self.hth = (math.pi / 2) / (self.Nth - 2 * self.overlap)
        self.delta = self.overlap * self.hth
        self.hph = (1.5 * math.pi + 2 * self.delta) / self.Nph
        self.th0 = math.pi / 4 - self.delta
        self.ph0 = -0.75 * math.pi - self.delta
        if self.th0 <= 0:
            raise ValueError("patch reaches the pole: N_theta too small")
        # theta_1 of the modified phi operator (Sec. 3.2): smallest theta of the patch
        self.theta1 = self.th0
        self.shape = (2, self.Nr + 2, self.Nth + 2, self.Nph + 2)

    # 1-D coordinates, indexed by logical index (array of logical indices in)
    def r_c(self, i):
        if self.uniform_r:
            return self.R1 + (np.asarray(i, dtype=np.float64) + 0.5) * self.hr
        return self._rh[2 * np.asarray(i) + 1 + 4]

    def r_f(self, i):
        if self.uniform_r:
            return self.R1 + np.asarray(i, dtype=np.float64) * self.hr
        return self._rh[2 * np.asarray(i) + 4]

    # radial spacings: h_c at centre i (cell width), h_f at face i (centre distance)
    def h_c(self, i):
        if self.uniform_r:
            return np.full(np.shape(i), self.hr)
        return self.r_f(np.asarray(i) + 1) - self.r_f(i)

    def h_f(self, i):
        if self.uniform_r:
            return np.full(np.shape(i), self.hr)
        return self.r_c(i) - self.r_c(np.asarray(i) - 1)

    def th_c(self, j):
        return self.th0 + (np.asarray(j, dtype=np.float64) + 0.5) * self.hth

    def th_f(self, j):
        return self.th0 + np.asarray(j, dtype=np.float64) * self.hth

    def ph_c(self, k):
        return self.ph0 + (np.asarray(k, dtype=np.float64) + 0.5) * self.hph

    def ph_f(self, k):
        return self.ph0 + np.asarray(k, dtype=np.float64) * self.hph

    # regions of unknowns, logical half-open ranges (i0, i1, j0, j1, k0, k1)
    def region(self, loc):
        Nr, Nt, Np = self.Nr, self.Nth, self.Nph
        return {C: (0, Nr, 0, Nt, 0, Np),
                R: (1, Nr, 0, Nt, 0, Np),      # wall faces carry Dirichlet data
                TH: (0, Nr, 1, Nt, 0, Np),     # edge faces come from the exchange
                PH: (0, Nr, 0, Nt, 1, Np)}[loc]

    def zeros(self):
        return np.zeros(self.shape)

    def coords(self, loc, reg=None):
        """Broadcastable (r, theta) of the points of region ``reg`` (default:
        the unknowns of ``loc``) with shapes (1, ni, 1, 1) and (1, 1, nj, 1)."""
        i0, i1, j0, j1, _, _ = self.region(loc) if reg is None else reg
        ii, jj = np.arange(i0, i1), np.arange(j0, j1)
        r = self.r_f(ii) if loc == R else self.r_c(ii)
        th = self.th_f(jj) if loc == TH else self.th_c(jj)
        return r[None, :, None, None], th[None, None, :, None]

    def user_slices(self, loc):
        """Slices of a padded array holding the user-layout points of ``loc``
        (interior plus boundary faces)."""
        Nr, Nt, Np = self.Nr, self.Nth, self.Nph
        ni = Nr + 1 if loc == R else Nr
        nj = Nt + 1 if loc == TH else Nt
        nk = Np + 1 if loc == PH else Np
        return (slice(None), slice(1, 1 + ni), slice(1, 1 + nj), slice(1, 1 + nk))

    def weight(self, loc):
        """Midpoint-rule weight r^2 sin(theta) h h_th h_ph at the unknowns of
        ``loc``, h the radial spacing of the point (h_f at r-faces, h_c else)."""
        r, th = self.coords(loc)
        i0, i1 = self.region(loc)[:2]
        ii = np.arange(i0, i1)
        h = (self.h_f(ii) if loc == R else self.h_c(ii))[None, :, None, None]
        return r * r * np.sin(th) * h * self.hth * self.hph


def view(a, reg, di=0, dj=0, dk=0):
    """The block of padded array ``a`` covering logical region ``reg`` shifted by (di, dj, dk)."""
    i0, i1, j0, j1, k0, k1 = reg
    return a[:, i0 + 1 + di:i1 + 1 + di, j0 + 1 + dj:j1 + 1 + dj, k0 + 1 + dk:k1 + 1 + dk]


def sph_to_unit(th, ph):
    """Unit vector of spherical angles, local Cartesian components (last axis)."""
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th) + 0 * ph], axis=-1)


def unit_to_sph(x):
    """Spherical angles (theta, phi) of unit vectors x[..., 3]."""
    th = np.arccos(np.clip(x[..., 2], -1.0, 1.0))
    ph = np.arctan2(x[..., 1], x[..., 0])
    return th, ph


def e_theta(th, ph):
    return np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th) + 0 * ph], axis=-1)


def e_phi(th, ph):
    return np.stack([-np.sin(ph) + 0 * th, np.cos(ph) + 0 * th, 0 * th + 0 * ph], axis=-1)
