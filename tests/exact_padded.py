"""Exact fields sampled on the oracle's padded arrays (ghosts included),
for operator-level pins.  Uses the oracle grid for point positions and the
workload module's exact solutions; shared by CPU tests only."""
import numpy as np

from paper_1905_02300_gb300 import workloads as W


def padded_exact(g, ex, t, which=("T", "p", "ur", "ut", "up"), a_ex=None):
    """Dict of padded arrays (2, Nr+2, Nth+2, Nph+2) of the exact solution
    ``ex`` at time t: keys T, p, ur, ut, up (local spherical components)."""
    ii = np.arange(-1, g.Nr + 1)
    jj = np.arange(-1, g.Nth + 1)
    kk = np.arange(-1, g.Nph + 1)
    out = {}
    c = ex.tfac(t)
    for loc in ("c", "r", "t", "p"):
        r = g.r_f(ii) if loc == "r" else g.r_c(ii)
        th = g.th_f(jj) if loc == "t" else g.th_c(jj)
        ph = g.ph_f(kk) if loc == "p" else g.ph_c(kk)
        R, TH, PH = np.meshgrid(r, th, ph, indexing="ij")
        xl = R * np.sin(TH) * np.cos(PH)
        yl = R * np.sin(TH) * np.sin(PH)
        zl = R * np.cos(TH)
        x, y, z = np.stack([xl, -xl]), np.stack([yl, zl]), np.stack([zl, yl])
        X, Y, Z = W.Jet.variables(x, y, z)
        U, P, Th = ex.fields(X, Y, Z, W.JetNS)
        if loc == "c":
            out["T"] = Th.v * c
            out["p"] = P.v * c
            continue
        st, ct, sp, cp = np.sin(TH), np.cos(TH), np.sin(PH), np.cos(PH)
        e = {"r": (st * cp, st * sp, ct), "t": (ct * cp, ct * sp, -st), "p": (-sp, cp, 0 * sp)}[loc]
        vx, vy, vz = U[0].v, U[1].v, U[2].v
        lx, ly, lz = np.stack([vx[0], -vx[1]]), np.stack([vy[0], vz[1]]), np.stack([vz[0], vy[1]])
        out["u" + loc] = (lx * e[0] + ly * e[1] + lz * e[2]) * c
    return out
