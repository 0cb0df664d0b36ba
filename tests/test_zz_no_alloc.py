"""The allocation-free entry point ys_factor_solve_static against ys_step.

Callers that cannot allocate device memory (code under another allocator's
budget, callbacks that must not enter the driver's allocator) use
ys_factor_solve_static, whose scratch is a static device array.  With one
Schwarz iteration, ys_step advances T by exactly one factored solve:
T^1 = T^0 + P_T^-1 r_T, with T^0 = 2 T^n - T^{n-1}.  The test computes r_T
for the same state (FP64 oracle), calls the new entry point twice in a row
through the C ABI on caller-owned device buffers, and checks each output
against T^1 - T^0 from ys_step, within the parity tolerance used elsewhere
(1e-11 relative max-norm).  It runs alone or after the other tests.

The velocity unknowns (u_r, u_theta, u_phi, each with its own-direction
extras and grad-div rows) and a temperature factor with Robin and Neumann
walls are checked against the oracle's factored line solves: the same
seeded right-hand side and advecting velocity, each 1-D factor of the
oracle solved by its Thomas algorithm in the unknown's order.
"""
import ctypes

import numpy as np
import pytest

from oracle import exchange as xch
from oracle import operators as ops
from oracle.grid import C, PH, R, TH, view
from oracle.linesolve import solve_factored
from oracle.scheme import Level, Oracle, Params
from paper_1905_02300_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KW = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=1e-3, Nr=16, Nth=16, Nph=48)
CHI = 1.0                     # default of ys_params.chi


def _oracle_rhs_T(f0, fm, modes):
    """r_T = dt Rate_T((T^0 + T^n)/2) - (T^0 - T^n) of the first iteration,
    with the advecting velocity a, both in the user layouts."""
    o = Oracle(Params(**KW))
    o.set_fields(0, f0["T"], f0["ur"], f0["uth"], f0["uph"], f0["p"])
    o.set_fields(1, fm["T"], fm["ur"], fm["uth"], fm["uph"], fm["p"])
    for tid, F in modes:
        o.set_forcing(tid, F["T"], F["ur"], F["uth"], F["uph"])
    g = o.g
    n, nm1 = o.lev
    A = [1.5 * n.u2[m] - 0.5 * nm1.u2[m] for m in range(3)]
    it = Level(2.0 * n.T - nm1.T, [2.0 * n.u1[m] - nm1.u1[m] for m in range(3)],
               [2.0 * n.u2[m] - nm1.u2[m] for m in range(3)], 2.0 * n.p1 - nm1.p1, 2.0 * n.p2 - nm1.p2)
    d = it.as_dict()
    xch.exchange_into(o.tables, d, d, (0, 1))
    f = o.forcing(o.t + 0.5 * KW["dt"])
    rate = ops.rate_T(g, 0.5 * (it.T + n.T), A, f["T"])
    rhs = KW["dt"] * rate - (view(it.T, g.region(C)) - view(n.T, g.region(C)))
    a_user = [A[0][g.user_slices(R)], A[1][g.user_slices(TH)], A[2][g.user_slices(PH)]]
    return np.ascontiguousarray(rhs), [np.ascontiguousarray(a) for a in a_user]


def test_static_scratch_solve_matches_ys_step(gpu_lib):
    import torch
    ys = gpu_lib
    spec = W.Spec(KW["R1"], KW["R2"], KW["Nr"], KW["Nth"], KW["Nph"])
    ex = W.TrigShell(KW["R1"], KW["R2"], KW["Pr"], KW["Ra"])
    f0, fm = W.sample_fields(ex, spec, 0.0), W.sample_fields(ex, spec, -KW["dt"])
    modes = W.forcing_modes(ex, spec)

    # the existing entry point: one step with one Schwarz iteration
    s = ys.Solver(**KW)
    s.set_fields_dict(0, f0)
    s.set_fields_dict(1, fm)
    for m, (tid, F) in enumerate(modes):
        s.set_forcing(m, tid, F["T"], F["ur"], F["uth"], F["uph"])
    s.step(1, 1)
    expect = s.get_fields(0)["T"] - (2.0 * f0["T"] - fm["T"])

    rhs, A = _oracle_rhs_T(f0, fm, modes)
    dev = torch.device("cuda", torch.cuda.current_device())
    dA = [torch.from_numpy(a).to(dev) for a in A]
    drhs = torch.from_numpy(rhs).to(dev)
    prm = ys.default_params(**KW)
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for call in range(2):
        dx = torch.full_like(drhs, float("nan"))
        rc = ys.lib.ys_factor_solve_static(ctypes.byref(prm), 0, dA[0].data_ptr(), dA[1].data_ptr(),
                                           dA[2].data_ptr(), drhs.data_ptr(), dx.data_ptr(),
                                           ctypes.c_void_p(stream))
        assert rc == ys.YS_OK, ys.lib.ys_strerror(rc)
        torch.cuda.synchronize()
        x = dx.cpu().numpy()
        err = np.abs(x - expect).max() / np.abs(expect).max()
        assert err <= 1e-11, (call, err)
        outs.append(x)
    assert np.array_equal(outs[0], outs[1])


def _call_static(ys, prm, loc, dA, drhs, stream):
    import torch
    dx = torch.full_like(drhs, float("nan"))
    rc = ys.lib.ys_factor_solve_static(ctypes.byref(prm), loc, dA[0].data_ptr(), dA[1].data_ptr(), dA[2].data_ptr(),
                                       drhs.data_ptr(), dx.data_ptr(), ctypes.c_void_p(stream))
    assert rc == ys.YS_OK, ys.lib.ys_strerror(rc)
    torch.cuda.synchronize()
    return dx.cpu().numpy()


# (unknown, parameters that differ from KW): the three velocity components at
# a viscosity and chi other than 1, and T with a Robin inner and a Neumann
# outer wall (the wall rows of its radial factor follow the ghost factors)
CASES = [(1, dict(Pr=0.7, chi=1.5)), (2, dict(Pr=0.7, chi=1.5)), (3, dict(Pr=0.7, chi=1.5)),
         (0, dict(Tbc_inner_a=1.0, Tbc_inner_b=0.5, Tbc_outer_a=0.0, Tbc_outer_b=1.0))]


@pytest.mark.parametrize("loc,extra", CASES, ids=["u_r", "u_theta", "u_phi", "T_robin_neumann"])
def test_static_scratch_solve_matches_the_oracle_factors(gpu_lib, loc, extra):
    import torch
    ys = gpu_lib
    kw = dict(KW, chi=CHI)
    kw.update({k: v for k, v in extra.items() if not k.startswith("Tbc")})
    spec = W.Spec(kw["R1"], kw["R2"], kw["Nr"], kw["Nth"], kw["Nph"])
    ex = W.CurlShell(kw["R1"], kw["R2"], kw["Pr"], kw["Ra"])
    f0, fm = W.sample_fields(ex, spec, 0.0), W.sample_fields(ex, spec, -kw["dt"])
    o = Oracle(Params(**{k: kw[k] for k in ("R1", "R2", "Pr", "Ra", "dt", "Nr", "Nth", "Nph", "chi")}))
    g = o.g
    # advecting velocity 1.5 u^n - 0.5 u^{n-1} in the user layouts, and padded
    # with zeros outside them (the entry point reads the user layouts only)
    keys, locs = ("ur", "uth", "uph"), (R, TH, PH)
    A_user = [np.ascontiguousarray(1.5 * f0[k] - 0.5 * fm[k]) for k in keys]
    A_pad = []
    for a, lc in zip(A_user, locs):
        z = g.zeros()
        z[g.user_slices(lc)] = a
        A_pad.append(z)
    ul = (C, R, TH, PH)[loc]
    rng = np.random.default_rng(11 + loc)
    rhs_user = np.ascontiguousarray(rng.uniform(-1.0, 1.0, size=g.zeros()[g.user_slices(ul)].shape))
    rhs_pad = g.zeros()
    rhs_pad[g.user_slices(ul)] = rhs_user
    gam = (-1.0, -1.0)
    if loc == 0:
        gam = (xch.robin_ghost(extra["Tbc_inner_a"], extra["Tbc_inner_b"], float(g.h_f(0)))[0],
               xch.robin_ghost(extra["Tbc_outer_a"], extra["Tbc_outer_b"], float(g.h_f(g.Nr)))[0])
    nu = 1.0 if loc == 0 else kw["Pr"]
    fac = {d: ops.factor(g, ul, d, A_pad, kw["dt"], nu, kw["chi"], gam) for d in "rtp"}
    x_pad = g.zeros()
    view(x_pad, g.region(ul))[...] = solve_factored(fac, ops.ORDER[ul], view(rhs_pad, g.region(ul)))
    expect = x_pad[g.user_slices(ul)]

    dev = torch.device("cuda", torch.cuda.current_device())
    dA = [torch.from_numpy(a).to(dev) for a in A_user]
    drhs = torch.from_numpy(rhs_user).to(dev)
    prm = ys.default_params(**kw, **{k: v for k, v in extra.items() if k.startswith("Tbc")})
    stream = torch.cuda.current_stream().cuda_stream
    outs = [_call_static(ys, prm, loc, dA, drhs, stream) for _ in range(2)]
    for call, x in enumerate(outs):
        err = np.abs(x - expect).max() / np.abs(expect).max()
        assert err <= 1e-11, (loc, call, err)
    assert np.array_equal(outs[0], outs[1])


def test_static_scratch_rejects_oversized_grid(gpu_lib):
    ys = gpu_lib
    prm = ys.default_params(**dict(KW, Nr=48, Nth=48, Nph=144))
    dummy = ctypes.c_void_p(1)
    rc = ys.lib.ys_factor_solve_static(ctypes.byref(prm), 0, dummy, dummy, dummy, dummy, dummy, None)
    assert rc == ys.YS_EINVAL
