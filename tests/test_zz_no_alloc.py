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
"""
import ctypes

import numpy as np
import pytest

from oracle import exchange as xch
from oracle import operators as ops
from oracle.grid import C, PH, R, TH, view
from oracle.scheme import Level, Oracle, Params
from paper_1905_02300_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KW = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=1e-3, Nr=16, Nth=16, Nph=48)


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


def test_static_scratch_rejects_oversized_grid(gpu_lib):
    ys = gpu_lib
    prm = ys.default_params(**dict(KW, Nr=48, Nth=48, Nph=144))
    dummy = ctypes.c_void_p(1)
    rc = ys.lib.ys_factor_solve_static(ctypes.byref(prm), 0, dummy, dummy, dummy, dummy, dummy, None)
    assert rc == ys.YS_EINVAL
