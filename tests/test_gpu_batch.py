"""Batched ensembles and serving (continuous batching) on the GPU.

A shell's fields must not depend on what else is in the batch: the per-shell
arithmetic and block decomposition of the batched kernels are the same alone
and in any mix, so those checks are bitwise.  Against the single-shell path
(other kernels) the mixed form is checked at its 1e-5 relative tolerance;
in FP64 the two paths are bitwise equal (measured, and asserted)."""
import time

import numpy as np
import pytest

from paper_1905_02300_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHELLS = [dict(R1=0.45, Nr=16, Nth=20, Ra=2e3, Pr=1.0), dict(R1=0.55, Nr=20, Nth=16, Ra=1e4, Pr=0.7),
          dict(R1=0.35, Nr=12, Nth=24, Ra=5e3, Pr=7.0)]


def make(ys, sp, precision=None):
    Nr, Nth = sp["Nr"], sp["Nth"]
    rh = W.stretched_radii(sp["R1"], 1.0, Nr, sp["stretch"]) if "stretch" in sp else None
    spec = W.Spec(sp["R1"], 1.0, Nr, Nth, 3 * Nth)
    hr = spec.hr if rh is None else float(np.min(np.diff(np.asarray(rh)[::2])))
    hmin = min(hr, sp["R1"] * spec.hth, sp["R1"] * np.sin(spec.th0) * spec.hph)
    kw = dict(R1=sp["R1"], R2=1.0, Pr=sp["Pr"], Ra=sp["Ra"], Nr=Nr, Nth=Nth, Nph=3 * Nth, dt=0.5 * hmin * hmin,
              T_inner=1.0, T_outer=0.0, precision=ys.YS_MIXED if precision is None else precision, r_half=rh)
    s = ys.Solver(**kw)
    spec = W.Spec(kw["R1"], 1.0, Nr, Nth, 3 * Nth, r_half=rh)
    s.set_fields_dict(0, W.convection_initial(spec, sp["Pr"], sp["Ra"], T_in=1.0))
    return s, kw


def fields(s):
    return s.get_fields(0, aux=True)


def same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


def close(a, b, tol=1e-5):
    for k in a:
        scale = max(np.abs(b[c]).max() for c in (("ur", "uth", "uph") if k in ("ur", "uth", "uph") else
                                                  ("ur1", "uth1", "uph1") if k in ("ur1", "uth1", "uph1") else (k,)))
        if np.abs(a[k] - b[k]).max() > tol * max(scale, 1e-300):
            return False
    return True


def alone(ys, sp, n):
    """fields after n steps of the shell alone in a batch"""
    b = ys.Batch(1)
    s, _ = make(ys, sp)
    slot = b.add(s)
    b.step(n)
    b.sync()
    f = fields(b.remove(slot))
    b.close()
    return f


def test_batch_is_mix_independent_and_matches_single_shell_path(gpu_lib):
    ys = gpu_lib
    ref, single = [], []
    for sp in SHELLS:
        ref.append(alone(ys, sp, 5))
        s, _ = make(ys, sp)
        s.step(5, 3)
        single.append(fields(s))
    b = ys.Batch(8)
    members = [make(ys, sp)[0] for sp in SHELLS]
    slots = [b.add(m) for m in members]
    b.step(5)
    b.sync()
    for slot, r, sg in zip(slots, ref, single):
        s = b.remove(slot)
        assert s.stats()["steps"] == 5
        f = fields(s)
        assert same(f, r)
        assert close(f, sg)
    assert b.launches_per_step() > 0
    b.close()


def test_stretched_radial_grid_shell_in_a_batch(gpu_lib):
    """A shell on a stretched radial grid batches with uniform ones: its
    fields are the same alone and in the mix (bitwise) and within 1e-5 of the
    single-shell path (its coefficient tables travel with it)."""
    ys = gpu_lib
    mix = [dict(R1=0.45, Nr=16, Nth=20, Ra=2e3, Pr=1.0, stretch=0.5), SHELLS[1]]
    ref = alone(ys, mix[0], 5)
    s, _ = make(ys, mix[0])
    s.step(5, 3)
    single = fields(s)
    b = ys.Batch(4)
    slots = [b.add(make(ys, sp)[0]) for sp in mix]
    b.step(5)
    b.sync()
    f = fields(b.remove(slots[0]))
    assert same(f, ref)
    assert close(f, single)
    b.close()


def test_fp64_single_shell_path_matches_the_batched_kernels(gpu_lib):
    """The FP64 single-shell step reads the half-level sums psi + psi^n, the
    bootstrapped momentum pressure P2 and the phi factors' lane-segment
    products from fields formed once per iteration or step; the batched
    kernels form every one of them where they use it, with the same
    additions and products.  The same shells (one on a stretched radial
    grid) advanced 4 steps by both paths are bitwise equal in every field."""
    ys = gpu_lib
    for sp in (SHELLS[0], dict(SHELLS[1], stretch=0.5)):
        s1, _ = make(ys, sp, precision=ys.YS_FP64)
        s1.step(4, 3)
        ref = fields(s1)
        s1.close()
        b = ys.Batch(1, precision=ys.YS_FP64, n_schwarz=3)
        s2, _ = make(ys, sp, precision=ys.YS_FP64)
        slot = b.add(s2)
        b.step(4)
        b.sync()
        got = fields(b.remove(slot))
        b.close()
        e = {k: float(np.abs(got[k] - ref[k]).max() / max(np.abs(ref[k]).max(), 1e-300)) for k in ref}
        assert same(got, ref), (sp, e)


def test_shells_join_and_leave_between_steps(gpu_lib):
    ys = gpu_lib
    a_ref = alone(ys, SHELLS[0], 6)
    b_ref = alone(ys, SHELLS[1], 3)
    bt = ys.Batch(4)
    a, _ = make(ys, SHELLS[0])
    sa = bt.add(a)
    bt.step(3)
    b, _ = make(ys, SHELLS[1])
    sb = bt.add(b)
    bt.step(3)
    bt.sync()
    assert same(fields(bt.remove(sa)), a_ref)
    assert same(fields(bt.remove(sb)), b_ref)  # b ran 3 steps
    bt.close()


def test_autotune_keeps_results(gpu_lib):
    ys = gpu_lib
    ref = alone(ys, SHELLS[2], 8)
    bt = ys.Batch(2)
    s, _ = make(ys, SHELLS[2])
    slot = bt.add(s)
    chosen = bt.autotune(trial_steps=1)      # 4 candidates x (1 + 1) steps = 8 steps
    assert chosen in (32, 64, 128, 256)
    bt.sync()
    assert same(fields(bt.remove(slot)), ref)
    bt.close()


def test_server_continuous_batching(gpu_lib):
    ys = gpu_lib
    reqs = [(SHELLS[0], 4), (SHELLS[1], 7), (SHELLS[2], 3), (SHELLS[0], 5), (SHELLS[2], 6)]
    expect = []
    for sp, n in reqs:
        f = alone(ys, sp, n)
        expect.append({k: f[k] for k in ("T", "ur", "uth", "uph", "p")})
    # budget for about two shells at a time: the rest wait for memory
    srv = ys.Server(hbm_budget_bytes=60 << 20, max_slots=8)
    tickets = []
    for sp, n in reqs:
        _, kw = make(ys, sp)
        spec = W.Spec(kw["R1"], 1.0, kw["Nr"], kw["Nth"], kw["Nph"])
        tickets.append(srv.submit(W.convection_initial(spec, sp["Pr"], sp["Ra"], T_in=1.0), n, **kw))
        time.sleep(0.01)
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < 120:
        for t in tickets:
            if t in done:
                continue
            st, f, lat, rc = srv.poll(t)
            if st >= 2:
                done[t] = (st, f, lat, rc)
        time.sleep(0.002)
    assert len(done) == len(tickets)
    for t, e in zip(tickets, expect):
        st, f, lat, rc = done[t]
        assert st == ys.Server.DONE and rc == 0 and lat > 0
        for k in e:
            assert np.array_equal(f[k], e[k]), k
    # the server's own record: the budget never let more than ~2 run together
    peak = srv.stats()["peak_running"]
    assert 1 <= peak <= 3, peak
    srv.close()


def test_server_failed_request_does_not_poison_others(gpu_lib):
    ys = gpu_lib
    srv = ys.Server(hbm_budget_bytes=1 << 30, max_slots=4)
    _, kw = make(ys, SHELLS[1])
    good = alone(ys, SHELLS[1], 4)
    spec = W.Spec(kw["R1"], 1.0, kw["Nr"], kw["Nth"], kw["Nph"])
    init = W.convection_initial(spec, SHELLS[1]["Pr"], SHELLS[1]["Ra"], T_in=1.0)
    bad = {k: v.copy() for k, v in init.items()}
    bad["T"][0, 3, 4, 5] = np.nan
    tb = srv.submit(bad, 4, **kw)
    tg = srv.submit(init, 4, **kw)
    t0 = time.time()
    res = {}
    while len(res) < 2 and time.time() - t0 < 60:
        for t in (tb, tg):
            if t not in res:
                st, f, lat, rc = srv.poll(t)
                if st >= 2:
                    res[t] = (st, f, rc)
        time.sleep(0.002)
    assert res[tb][0] == ys.Server.FAILED and res[tb][2] == ys.YS_EDIVERGED
    st, f, rc = res[tg]
    assert st == ys.Server.DONE
    assert all(np.array_equal(f[k], good[k]) for k in f)
    srv.close()


def test_served_footprint_is_the_context_allocation(gpu_lib):
    """The figure the serving queue admits by (ys_shell_device_bytes, host
    only) is the device memory a created context holds, for the shells of
    these tests in both precisions and on a stretched radial grid."""
    import ctypes
    ys = gpu_lib
    for sp in SHELLS + [dict(SHELLS[0], stretch=0.5)]:
        for prec in (ys.YS_FP64, ys.YS_MIXED):
            s, kw = make(ys, sp, prec)
            p = ys.default_params(**kw)
            assert s.device_bytes() == ys.lib.ys_shell_device_bytes(ctypes.byref(p)), (sp, prec)
            s.close()


# uneven FP64 shells held to the oracle: phi lines longer than one scan chunk
# of 384, a stretched radial grid, a hot inner wall, a larger ragged shell
ORACLE_SHELLS = [dict(R1=0.45, Nr=8, Nth=12, Nph=400, Pr=1.0, Ra=50.0),
                 dict(R1=0.5, Nr=12, Nth=16, Nph=48, Pr=0.7, Ra=200.0, stretch=0.5),
                 dict(R1=0.4, Nr=10, Nth=14, Nph=42, Pr=7.0, Ra=1e3, T_in=1.0),
                 dict(R1=0.55, Nr=17, Nth=20, Nph=61, Pr=1.0, Ra=1e4)]
DT_ORACLE = 1e-4


def _oracle_case(sp, levels=2):
    """(solver parameters, level fields, oracle after set-up): the curl
    solution at t = 0 and t = -dt without forcing (batched shells take no
    forcing modes), plus the conductive profile when the inner wall is hot."""
    from oracle.scheme import Oracle, Params
    rh = W.stretched_radii(sp["R1"], 1.0, sp["Nr"], sp["stretch"]) if "stretch" in sp else None
    spec = W.Spec(sp["R1"], 1.0, sp["Nr"], sp["Nth"], sp["Nph"], r_half=rh)
    ex = W.CurlShell(sp["R1"], 1.0, sp["Pr"], sp["Ra"])
    T_in = sp.get("T_in", 0.0)
    lv = [W.sample_fields(ex, spec, -m * DT_ORACLE) for m in range(levels)]
    if T_in:
        Tc = W.conductive_profile(spec, T_in, 0.0)
        for f in lv:
            f["T"] = f["T"] + Tc
    kw = dict(R1=sp["R1"], R2=1.0, Pr=sp["Pr"], Ra=sp["Ra"], Nr=sp["Nr"], Nth=sp["Nth"], Nph=sp["Nph"],
              dt=DT_ORACLE, T_inner=T_in, T_outer=0.0, r_half=rh)
    o = Oracle(Params(R1=sp["R1"], R2=1.0, Pr=sp["Pr"], Ra=sp["Ra"], dt=DT_ORACLE, Nr=sp["Nr"], Nth=sp["Nth"],
                      Nph=sp["Nph"], T_in=T_in, T_out=0.0, r_half=rh))
    for m, f in enumerate(lv):
        o.set_fields(m, f["T"], f["ur"], f["uth"], f["uph"], f["p"])
    return kw, lv, o


def _parity(got, ref):
    return {k: float(np.abs(got[k] - ref[k]).max() / max(np.abs(ref[k]).max(), 1e-300)) for k in ref}


def test_fp64_batch_of_uneven_shells_matches_the_oracle(gpu_lib):
    """An FP64 batch of four uneven shells (one launch per kernel class over
    all of them, the batched kernels of the ensemble path) against the
    oracle, shell by shell, at the FP64 parity bound 1e-11 after 4 steps of 3
    Schwarz iterations."""
    ys = gpu_lib
    b = ys.Batch(4, precision=ys.YS_FP64, n_schwarz=3)
    cases, slots = [], []
    for sp in ORACLE_SHELLS:
        kw, lv, o = _oracle_case(sp)
        s = ys.Solver(**kw, precision=ys.YS_FP64)
        for m, f in enumerate(lv):
            s.set_fields_dict(m, f)
        slots.append(b.add(s))
        o.step(4, 3)
        cases.append(o)
    b.step(4)
    b.sync()
    for sp, slot, o in zip(ORACLE_SHELLS, slots, cases):
        s = b.remove(slot)
        assert s.stats()["steps"] == 4
        e = _parity(s.get_fields(0, aux=True), o.get_fields(0, aux=True))
        assert max(e.values()) <= 1e-11, (sp, e)
    b.close()


def test_served_fp64_request_matches_the_oracle(gpu_lib):
    """One request served in FP64 (continuous-batching server, fields packed
    through ys_submit / ys_poll, one time level given) against the oracle."""
    ys = gpu_lib
    sp = ORACLE_SHELLS[2]
    kw, lv, o = _oracle_case(sp, levels=1)
    o.step(5, 3)
    srv = ys.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    t = srv.submit(lv[0], 5, precision=ys.YS_FP64, **kw)
    t0 = time.time()
    while time.time() - t0 < 60:
        st, f, lat, rc = srv.poll(t)
        if st >= 2:
            break
        time.sleep(0.002)
    srv.close()
    assert st == ys.Server.DONE and rc == 0, (st, rc)
    ref = o.get_fields(0)
    e = _parity(f, ref)
    assert max(e.values()) <= 1e-11, e


def test_batch_member_that_blows_up_is_flagged_alone(gpu_lib):
    """In an FP64 batch with 3 Schwarz iterations a member whose iteration
    diverges (the blow-up state of the single-shell watch test) is reported by
    ys_batch_norms as YS_EDIVERGED, while its batch mate reports OK and ends
    bitwise where it ends alone."""
    import ctypes
    from tests.test_gpu_parity import blow_up_state
    ys = gpu_lib
    kw, lv0, lv1, aux = blow_up_state()

    def good():
        kwg, lv, _ = _oracle_case(ORACLE_SHELLS[2])
        s = ys.Solver(**kwg, precision=ys.YS_FP64)
        for m, f in enumerate(lv):
            s.set_fields_dict(m, f)
        return s

    b1 = ys.Batch(1, precision=ys.YS_FP64, n_schwarz=3)
    slot = b1.add(good())
    b1.step(2)
    b1.sync()
    ref = fields(b1.remove(slot))
    b1.close()

    b = ys.Batch(2, precision=ys.YS_FP64, n_schwarz=3)
    bad = ys.Solver(**kw)
    bad.set_fields_dict(0, lv0, aux)
    bad.set_fields_dict(1, lv1, aux)
    sb = b.add(bad)
    sg = b.add(good())
    b.step(1)
    b.sync()
    nrm = np.empty(ys.NFIELDS)
    ptr = nrm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert ys.lib.ys_batch_norms(b.h, sb, ptr) == ys.YS_EDIVERGED
    assert np.isfinite(nrm).all(), nrm
    assert ys.lib.ys_batch_norms(b.h, sg, ptr) == ys.YS_OK
    b.remove(sb)
    b.step(1)
    b.sync()
    assert same(fields(b.remove(sg)), ref)
    b.close()


def _wait(srv, t, states, limit=60.0):
    t0 = time.time()
    while time.time() - t0 < limit:
        r = srv.poll(t)
        if r[0] in states:
            return r
        time.sleep(0.002)
    raise AssertionError(f"request {t} not in {states} after {limit} s")


def _served(ys, sp):
    _, kw = make(ys, sp)
    spec = W.Spec(kw["R1"], 1.0, kw["Nr"], kw["Nth"], kw["Nph"])
    return W.convection_initial(spec, sp["Pr"], sp["Ra"], T_in=1.0), kw


def test_server_deadline_fails_the_late_request_alone(gpu_lib):
    """A request that cannot finish before its deadline fails with
    YS_ETIMEOUT at a step boundary past it; the request served beside it
    completes, bitwise as alone."""
    ys = gpu_lib
    expect = alone(ys, SHELLS[1], 4)
    srv = ys.Server(hbm_budget_bytes=1 << 30, max_slots=4)
    f_long, kw_long = _served(ys, SHELLS[2])
    f_ok, kw_ok = _served(ys, SHELLS[1])
    t_long = srv.submit(f_long, 10 ** 6, deadline_s=0.5, **kw_long)
    t_ok = srv.submit(f_ok, 4, **kw_ok)
    st, f, lat, rc = _wait(srv, t_ok, (ys.Server.DONE, ys.Server.FAILED))
    assert st == ys.Server.DONE and rc == ys.YS_OK
    assert all(np.array_equal(f[k], expect[k]) for k in f)
    st, _, lat, rc = _wait(srv, t_long, (ys.Server.DONE, ys.Server.FAILED))
    assert st == ys.Server.FAILED and rc == ys.YS_ETIMEOUT and 0.5 <= lat < 30.0, (st, rc, lat)
    srv.close()


def test_server_cancels_queued_and_running_requests_alone(gpu_lib):
    """With one slot: a queued request cancelled fails at once with
    YS_ECANCELED, the running one at its next step boundary; the request
    queued behind them is then admitted and completes bitwise as alone;
    cancelling a finished request is refused."""
    ys = gpu_lib
    expect = alone(ys, SHELLS[1], 4)
    srv = ys.Server(hbm_budget_bytes=1 << 30, max_slots=1)
    f_long, kw_long = _served(ys, SHELLS[2])
    f_ok, kw_ok = _served(ys, SHELLS[1])
    t1 = srv.submit(f_long, 10 ** 6, **kw_long)
    _wait(srv, t1, (ys.Server.RUNNING,))
    t2 = srv.submit(f_long, 10 ** 6, **kw_long)
    assert srv.poll(t2)[0] == ys.Server.QUEUED
    srv.cancel(t2)
    st, _, _, rc = srv.poll(t2)
    assert st == ys.Server.FAILED and rc == ys.YS_ECANCELED
    t3 = srv.submit(f_ok, 4, **kw_ok)
    srv.cancel(t1)
    st, _, _, rc = _wait(srv, t1, (ys.Server.DONE, ys.Server.FAILED))
    assert st == ys.Server.FAILED and rc == ys.YS_ECANCELED
    st, f, _, rc = _wait(srv, t3, (ys.Server.DONE, ys.Server.FAILED))
    assert st == ys.Server.DONE and rc == ys.YS_OK
    assert all(np.array_equal(f[k], expect[k]) for k in f)
    with pytest.raises(ys.YSError) as e:
        srv.cancel(t3)
    assert e.value.code == ys.YS_EINVAL
    srv.close()


def test_server_queue_limit_refuses_with_busy(gpu_lib):
    """A full queue refuses a new request with YS_EBUSY at submit; once a
    queued request leaves (cancelled) the next submit is accepted."""
    ys = gpu_lib
    srv = ys.Server(hbm_budget_bytes=1 << 30, max_slots=1, max_queue=2)
    f_long, kw_long = _served(ys, SHELLS[2])
    t1 = srv.submit(f_long, 10 ** 6, **kw_long)
    _wait(srv, t1, (ys.Server.RUNNING,))
    q = [srv.submit(f_long, 10 ** 6, **kw_long) for _ in range(2)]
    with pytest.raises(ys.YSError) as e:
        srv.submit(f_long, 10 ** 6, **kw_long)
    assert e.value.code == ys.YS_EBUSY
    srv.cancel(q[0])
    q.append(srv.submit(f_long, 10 ** 6, **kw_long))
    for t in [t1] + q[1:]:
        srv.cancel(t)
    for t in [t1] + q[1:]:
        assert _wait(srv, t, (ys.Server.FAILED,))[3] == ys.YS_ECANCELED
    srv.close()
