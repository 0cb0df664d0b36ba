"""Host-side check of the padded field layout and of the access pattern of the
FP32 residual kernels that compute 4 phi-points per thread (CPU, no GPU).

The layout (include/ys.h, csrc/ys_internal.cuh lidx): per patch a box of
logical (i, j, k) in [-1, Nr] x [-1, Nth] x [-1, Nph], rows along phi of pitch
P = ceil((Nph + 2) / 8) * 8 starting 8 elements into the row, patch stride
PS = ceil(((Nr + 2) (Nth + 2) P + 16) / 32) * 32.  A thread of the vector
residuals takes the group k = 4 g .. 4 g + 3 of one (patch, i, j) row, loads
16-byte vectors at the group's own offset and at the offsets of its stencil
rows (q +- SI, q +- P, q - SI + P, q + SI - P) and one scalar at each end
(q - 1, q + 4, ...), and masks the lanes outside the unknowns' region.  Every
address, masked lanes included, must lie inside the field (2 PS elements) and
every vector load must be 16-byte aligned; the groups must cover each row's
unknowns exactly once, for the two-dimensional launches and for the batched
launches' flat group ranges alike.
"""
import numpy as np
import pytest

NV = 4


def layout(Nr, Nt, Np):
    NJ = Nt + 2
    P = ((Np + 2) + 7) // 8 * 8
    SI = NJ * P
    PS = ((Nr + 2) * SI + 16 + 31) // 32 * 32
    return dict(NJ=NJ, P=P, SI=SI, PS=PS, total=2 * PS)


def lidx(L, p, i, j, k):
    return p * L["PS"] + ((i + 1) * L["NJ"] + (j + 1)) * L["P"] + k + 8


def region(loc, Nr, Nt, Np):
    return (1 if loc == "r" else 0, Nr, 1 if loc == "t" else 0, Nt, 1 if loc == "p" else 0, Np)


# vector-load and scalar offsets of each residual body (T at centres, u_r, u_theta, u_phi)
def offsets(loc, L):
    SI, P = L["SI"], L["P"]
    vec = {"c": [0, SI, -SI, P, -P], "r": [0, SI, -SI, P, -P, -SI + P], "t": [0, SI, -SI, P, -P, SI - P],
           "p": [0, SI, -SI, P, -P]}[loc]
    sca = {"c": [NV, -1], "r": [NV, -1, -SI + NV], "t": [NV, -1, -P + NV], "p": [NV, -1, -1 + SI, -1 + P]}[loc]
    return vec, sca


def groups_2d(loc, Nr, Nt, Np, tpb_max=256):
    """(row, k) of every thread of the single-shell launch (resid_launch)."""
    i0, i1, j0, j1, _, _ = region(loc, Nr, Nt, Np)
    gpr = (Np + NV - 1) // NV
    tpb = min(tpb_max, (gpr + 31) // 32 * 32)
    gx = (gpr + tpb - 1) // tpb
    rows = 2 * (i1 - i0) * (j1 - j0)
    for row in range(rows):
        for t in range(gx * tpb):
            yield row, NV * t


def groups_flat(loc, Nr, Nt, Np, tpb=128):
    """(row, k) of every thread of the batched launch (flat group range)."""
    i0, i1, j0, j1, _, _ = region(loc, Nr, Nt, Np)
    gpr = (Np + NV - 1) // NV
    rows = 2 * (i1 - i0) * (j1 - j0)
    nblk = (rows * gpr + tpb - 1) // tpb
    for g in range(nblk * tpb):
        row, grp = divmod(g, gpr)
        if row < rows:
            yield row, NV * grp


def check(Nr, Nt, Np, gen):
    L = layout(Nr, Nt, Np)
    for loc in ("c", "r", "t", "p"):
        i0, i1, j0, j1, k0, k1 = region(loc, Nr, Nt, Np)
        nj, ni = j1 - j0, i1 - i0
        vec, sca = offsets(loc, L)
        covered = {}
        for row, k in gen(loc, Nr, Nt, Np):
            j = j0 + row % nj
            i = i0 + (row // nj) % ni
            p = row // (ni * nj)
            lanes = [l for l in range(NV) if k0 <= k + l < k1]
            if not lanes:
                continue
            q = lidx(L, p, i, j, k)
            for o in vec:
                assert (q + o) % NV == 0, (loc, p, i, j, k, o)
                assert 0 <= q + o and q + o + NV <= L["total"], (loc, p, i, j, k, o)
            for o in sca:
                assert 0 <= q + o < L["total"], (loc, p, i, j, k, o)
            for l in lanes:
                key = (p, i, j, k + l)
                assert key not in covered
                covered[key] = True
        expect = 2 * ni * nj * (k1 - k0)
        assert len(covered) == expect, (loc, len(covered), expect)


@pytest.mark.parametrize("dims", [(9, 21, 151), (12, 12, 36), (16, 16, 48), (8, 10, 30), (13, 17, 41)])
def test_vector_residual_groups_in_bounds_aligned_and_covering(dims):
    check(*dims, groups_2d)
    check(*dims, groups_flat)


def test_full_size_rows_stay_inside_the_patch_box():
    """The extreme rows of large grids: the furthest reads of the last group of
    the last row stay inside the field (the box's tail slack)."""
    for Nr, Nt, Np in ((128, 128, 384), (112, 112, 336), (256, 256, 768), (64, 96, 287)):
        L = layout(Nr, Nt, Np)
        gpr = (Np + NV - 1) // NV
        for loc in ("c", "r", "t", "p"):
            i0, i1, j0, j1, _, _ = region(loc, Nr, Nt, Np)
            vec, sca = offsets(loc, L)
            for p in (0, 1):
                for i in (i0, i1 - 1):
                    for j in (j0, j1 - 1):
                        for k in (0, NV * (gpr - 1)):
                            q = lidx(L, p, i, j, k)
                            assert all(0 <= q + o and q + o + NV <= L["total"] for o in vec)
                            assert all(0 <= q + o < L["total"] for o in sca)
