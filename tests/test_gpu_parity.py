"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance: relative max-norm per field, err = max|gpu - oracle| / max|oracle|,
<= 1e-11 after 10 steps in FP64 (the stated parity target for the plain
method), tighter for single steps.  Both sides get the same seeded synthetic
inputs from paper_1905_02300_gb300.workloads.
"""
import math

import numpy as np
import pytest

from oracle.scheme import Oracle, Params
from paper_1905_02300_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("T", "ur", "uth", "uph", "p", "ur1", "uth1", "uph1", "p1")


def make_pair(ys, kind="trig", R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, Nr=16, Nth=16, Nph=48, dt=1e-3,
              mode="additive", tol=0.0, step7=True, T_in=0.0, T_out=0.0, with_gpu=True, with_oracle=True,
              r_half=None, precision=None):
    spec = W.Spec(R1, R2, Nr, Nth, Nph, r_half=r_half)
    ex = W.EXACT[kind](R1, R2, Pr, Ra)
    f0, fm = W.sample_fields(ex, spec, 0.0), W.sample_fields(ex, spec, -dt)
    if T_in or T_out:
        Tc = W.conductive_profile(spec, T_in, T_out)
        f0["T"] = f0["T"] + Tc
        fm["T"] = fm["T"] + Tc
    modes = [] if kind == "radial_heat" else W.forcing_modes(ex, spec)
    o = s = None
    if with_oracle:
        o = Oracle(Params(R1=R1, R2=R2, Pr=Pr, Ra=Ra, dt=dt, Nr=Nr, Nth=Nth, Nph=Nph, schwarz_mode=mode,
                          schwarz_tol=tol, step7=step7, T_in=T_in, T_out=T_out, r_half=r_half))
        o.set_fields(0, f0["T"], f0["ur"], f0["uth"], f0["uph"], f0["p"])
        o.set_fields(1, fm["T"], fm["ur"], fm["uth"], fm["uph"], fm["p"])
        for tid, F in modes:
            o.set_forcing(tid, F["T"], F["ur"], F["uth"], F["uph"])
    if with_gpu:
        kw = {} if precision is None else {"precision": precision}
        s = ys.Solver(R1=R1, R2=R2, Pr=Pr, Ra=Ra, dt=dt, Nr=Nr, Nth=Nth, Nph=Nph,
                      schwarz_mode=ys.YS_MULTIPLICATIVE if mode == "multiplicative" else ys.YS_ADDITIVE,
                      schwarz_tol=tol, step7=1 if step7 else 0, T_inner=T_in, T_outer=T_out, r_half=r_half, **kw)
        s.set_fields_dict(0, f0)
        s.set_fields_dict(1, fm)
        for m, (tid, F) in enumerate(modes):
            s.set_forcing(m, tid, F["T"], F["ur"], F["uth"], F["uph"])
    return o, s, spec, ex


def rel_errs(s, o, level=0):
    g = s.get_fields(level, aux=True)
    r = o.get_fields(level, aux=True)
    return {k: np.abs(g[k] - r[k]).max() / max(np.abs(r[k]).max(), 1e-300) for k in FIELDS}


def assert_parity(s, o, tol, level=0):
    e = rel_errs(s, o, level)
    bad = {k: v for k, v in e.items() if not v <= tol}
    assert not bad, (bad, e)
    return e


def test_set_get_roundtrip_and_boundary_refresh(gpu_lib):
    o, s, spec, ex = make_pair(gpu_lib)
    for level in (0, 1):
        assert_parity(s, o, 1e-14, level)


def test_one_step_one_iteration(gpu_lib):
    o, s, _, _ = make_pair(gpu_lib)
    o.step(1, 1)
    s.step(1, 1)
    assert_parity(s, o, 1e-13)
    gn, it = s.norms()
    assert it == 1
    assert np.allclose(gn, o.last_norms, rtol=1e-9, atol=1e-300)


def test_c1_fp64_parity_after_10_steps(gpu_lib):
    """16x16x48 per patch, R1=0.5, R2=1, Pr=1, Ra=1e3, trigonometric
    manufactured solution with homogeneous walls, dt=1e-3, 10 steps, 3 Schwarz
    iterations: every field within 1e-11 relative max-norm of the oracle."""
    o, s, _, _ = make_pair(gpu_lib)
    o.step(10, 3)
    s.step(10, 3)
    e = assert_parity(s, o, 1e-11)
    assert s.stats()["steps"] == 10 and abs(s.stats()["t"] - o.t) < 1e-15
    # both time levels
    assert_parity(s, o, 1e-11, level=1)
    print(e)


def test_ragged_multi_tile_curl_solution(gpu_lib):
    """Odd sizes spanning several 128-thread tiles along phi with a ragged tail,
    non-zero radial velocity."""
    o, s, _, _ = make_pair(gpu_lib, kind="curl", Nr=9, Nth=21, Nph=151, dt=2e-3, Ra=50.0)
    o.step(3, 2)
    s.step(3, 2)
    assert_parity(s, o, 1e-12)


def test_multiplicative_schwarz(gpu_lib):
    o, s, _, _ = make_pair(gpu_lib, kind="curl", mode="multiplicative", Ra=10.0)
    o.step(3, 2)
    s.step(3, 2)
    assert_parity(s, o, 1e-12)


def test_step7_off(gpu_lib):
    o, s, _, _ = make_pair(gpu_lib, step7=False)
    o.step(2, 3)
    s.step(2, 3)
    assert_parity(s, o, 1e-12)


def test_inhomogeneous_wall_temperature(gpu_lib):
    o, s, _, _ = make_pair(gpu_lib, kind="curl", Ra=100.0, T_in=1.0, T_out=0.0)
    o.step(3, 3)
    s.step(3, 3)
    assert_parity(s, o, 1e-12)


def test_tolerance_driven_iterations(gpu_lib):
    o, s, _, _ = make_pair(gpu_lib, kind="curl", Ra=10.0, tol=1e-8)
    o.step(2, 50)
    s.step(2, 50)
    gn, it = s.norms()
    assert it == o.iters_done and it < 50
    assert_parity(s, o, 1e-11)


def test_radial_heat_closed_form_on_gpu(gpu_lib):
    errs = []
    for N, dt in ((16, 2e-3), (32, 5e-4)):
        _, s, spec, ex = make_pair(gpu_lib, kind="radial_heat", Ra=0.0, Nr=N, Nth=N, Nph=3 * N, dt=dt,
                                   tol=1e-12, with_oracle=False)
        s.step(int(round(0.016 / dt)), 80)
        got = s.get_fields(0)["T"]
        exact = W.sample_fields(ex, spec, s.stats()["t"])["T"]
        errs.append(np.abs(got - exact).max())
    assert math.log2(errs[0] / errs[1]) > 1.7, errs


def test_restart_is_bitwise(gpu_lib):
    """Checkpoint/resume: 6 steps straight == 3 steps, save both levels (with
    the system-1 fields), restore into a fresh context, 3 more steps."""
    _, a, _, _ = make_pair(gpu_lib, kind="curl", Ra=10.0, with_oracle=False)
    _, b, _, _ = make_pair(gpu_lib, kind="curl", Ra=10.0, with_oracle=False)
    a.step(6, 3)
    b.step(3, 3)
    lv = [b.get_fields(l, aux=True) for l in (0, 1)]
    t = b.stats()["t"]
    _, c, _, _ = make_pair(gpu_lib, kind="curl", Ra=10.0, with_oracle=False)
    for l in (1, 0):
        f = lv[l]
        c.set_fields(l, f["T"], f["ur"], f["uth"], f["uph"], f["p"], aux=(f["ur1"], f["uth1"], f["uph1"], f["p1"]))
    c.set_time(t)
    c.step(3, 3)
    ga, gc = a.get_fields(0, aux=True), c.get_fields(0, aux=True)
    for k in FIELDS:
        assert np.array_equal(ga[k], gc[k]), k


# ---------------------------------------------------------------- full size
FULL = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, Nr=128, Nth=128, Nph=384, dt=5e-4)


def test_full_size_yin_yang_congruence_bitwise(gpu_lib):
    """128x128x384 per patch (the benchmarked size and launch configuration):
    M-invariant data stays bitwise identical on both patches."""
    ys = gpu_lib
    spec = W.Spec(FULL["R1"], FULL["R2"], 128, 128, 384)
    ex = W.SymmetricShell(FULL["R1"], FULL["R2"], 1.0, 1e3)
    f0 = W.sample_fields(ex, spec, 0.0)
    for k in f0:
        f0[k][1] = f0[k][0]
    s = ys.Solver(**FULL)
    s.set_fields_dict(0, f0)
    s.step(2, 3)
    g = s.get_fields(0, aux=True)
    for k in FIELDS:
        assert np.array_equal(g[k][0], g[k][1]), k
    assert np.isfinite(g["uth"]).all() and np.abs(g["uth"]).max() > 1e-3


def test_full_size_space_convergence(gpu_lib):
    """Second order in space on 32x32x96, 64x64x192 and 128x128x384 per patch
    (manufactured solution, small dt, Schwarz to tolerance)."""
    errs = []
    for N in (32, 64, 128):
        _, s, spec, ex = make_pair(gpu_lib, kind="curl", Nr=N, Nth=N, Nph=3 * N, dt=2.5e-4, Ra=10.0,
                                   tol=1e-9, with_oracle=False)
        s.step(4, 40)
        g = s.get_fields(0)
        exact = W.sample_fields(ex, spec, s.stats()["t"])
        e = {}
        for k, loc in (("T", "c"), ("ur", "r"), ("uth", "t"), ("uph", "p")):
            r, th, _ = spec.coords(loc)
            w = np.broadcast_to(r * r * np.sin(th), g[k].shape)
            d = g[k] - exact[k]
            e[k] = math.sqrt(np.sum(w * d * d) / np.sum(w))
        errs.append(e)
    for k in errs[0]:
        for a, b in ((0, 1), (1, 2)):
            assert math.log2(errs[a][k] / errs[b][k]) > 1.7, (k, errs)


@pytest.mark.parametrize("ab", [(0.0, 1.0), (1.0, 0.5)])
def test_neumann_and_robin_temperature_walls(gpu_lib, ab):
    """Temperature wall condition a T + b dT/dn = 0 at R2 (Neumann, Robin):
    FP64 parity with the oracle after 10 steps of the closed-form heat
    solution, and the mixed form within 1e-5."""
    ys = gpu_lib
    a, b = ab
    N, dt = 12, 1e-3
    spec = W.Spec(0.5, 1.0, N, N, 3 * N)
    ex = W.RadialHeatRobin(0.5, 1.0, 1.0, 0.0, a=a, b=b)
    f0, fm = W.sample_fields(ex, spec, 0.0), W.sample_fields(ex, spec, -dt)
    o = Oracle(Params(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, Tbc_out=(a, b)))
    o.set_fields(0, f0["T"], f0["ur"], f0["uth"], f0["uph"], f0["p"])
    o.set_fields(1, fm["T"], fm["ur"], fm["uth"], fm["uph"], fm["p"])
    o.step(10, 3)
    for prec, tol in ((ys.YS_FP64, 1e-11), (ys.YS_MIXED, 1e-5)):
        s = ys.Solver(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, precision=prec,
                      Tbc_outer_a=a, Tbc_outer_b=b)
        s.set_fields_dict(0, f0)
        s.set_fields_dict(1, fm)
        s.step(10, 3)
        g = s.get_fields(0)["T"]
        r = o.get_fields(0)["T"]
        err = np.abs(g - r).max() / np.abs(r).max()
        assert err <= tol, (prec, err)


def test_stretched_radial_grid_parity(gpu_lib):
    """Sec. 4 non-uniform radial grid (cells 3x finer at the walls than
    mid-shell): FP64 within 1e-11 of the oracle after 10 steps, both time
    levels and the Schwarz increment norms; the mixed form within 1e-5, also
    with inhomogeneous wall temperatures (deviation variables built on the
    stretched grid)."""
    ys = gpu_lib
    rh = W.stretched_radii(0.5, 1.0, 16, 0.5)
    o, s, _, _ = make_pair(ys, r_half=rh)
    o.step(10, 3)
    s.step(10, 3)
    assert_parity(s, o, 1e-11)
    assert_parity(s, o, 1e-11, level=1)
    gn, _ = s.norms()
    assert np.allclose(gn, o.last_norms, rtol=1e-9, atol=1e-300)
    # mixed form: the measure of tests/test_gpu_mixed.py (a velocity component
    # against the velocity vector's largest value: the exact u_r is zero here)
    vel = {"ur": ("ur", "uth", "uph"), "uth": ("ur", "uth", "uph"), "uph": ("ur", "uth", "uph"),
           "ur1": ("ur1", "uth1", "uph1"), "uth1": ("ur1", "uth1", "uph1"), "uph1": ("ur1", "uth1", "uph1")}
    for T_in in (0.0, 1.0):
        o, s, _, _ = make_pair(ys, r_half=rh, T_in=T_in, precision=ys.YS_MIXED)
        o.step(10, 3)
        s.step(10, 3)
        g, r = s.get_fields(0, aux=True), o.get_fields(0, aux=True)
        e = {k: np.abs(g[k] - r[k]).max() / max(np.abs(r[c]).max() for c in vel.get(k, (k,))) for k in FIELDS}
        assert max(e.values()) <= 1e-5, (T_in, e)


def test_stretched_radial_grid_ragged_and_robin(gpu_lib):
    """Stretched radial grid on odd sizes with a ragged phi tail, and with a
    Robin temperature wall (its ghost uses the wall's own centre distance)."""
    ys = gpu_lib
    rh = W.stretched_radii(0.5, 1.0, 9, 0.4)
    o, s, _, _ = make_pair(ys, kind="curl", Nr=9, Nth=21, Nph=151, dt=2e-3, Ra=50.0, r_half=rh)
    o.step(3, 2)
    s.step(3, 2)
    assert_parity(s, o, 1e-12)
    N, dt = 12, 1e-3
    rh = W.stretched_radii(0.5, 1.0, N, 0.5)
    spec = W.Spec(0.5, 1.0, N, N, 3 * N, r_half=rh)
    ex = W.RadialHeatRobin(0.5, 1.0, 1.0, 0.0, a=1.0, b=0.5)
    f0, fm = W.sample_fields(ex, spec, 0.0), W.sample_fields(ex, spec, -dt)
    o = Oracle(Params(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, Tbc_out=(1.0, 0.5), r_half=rh))
    o.set_fields(0, f0["T"], f0["ur"], f0["uth"], f0["uph"], f0["p"])
    o.set_fields(1, fm["T"], fm["ur"], fm["uth"], fm["uph"], fm["p"])
    o.step(10, 3)
    s = ys.Solver(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=dt, Nr=N, Nth=N, Nph=3 * N, Tbc_outer_a=1.0,
                  Tbc_outer_b=0.5, r_half=rh)
    s.set_fields_dict(0, f0)
    s.set_fields_dict(1, fm)
    s.step(10, 3)
    g, r = s.get_fields(0)["T"], o.get_fields(0)["T"]
    assert np.abs(g - r).max() <= 1e-11 * np.abs(r).max()



def test_device_pointer_fields_agree_with_host_buffers(gpu_lib):
    """ys_set_fields_dev (fields already on the device, e.g. torch tensors)
    fills the same state as the host-buffer path: the fields after two
    steps are equal bit for bit."""
    import torch
    ys = gpu_lib
    o, s1, spec, ex = make_pair(ys, with_oracle=False)
    _, s2, _, _ = make_pair(ys, with_oracle=False)
    f0 = W.sample_fields(ex, spec, 0.0)
    keys = ("T", "ur", "uth", "uph", "p")
    dev = {k: torch.from_numpy(np.ascontiguousarray(f0[k], dtype=np.float64)).to("cuda:0") for k in keys}
    torch.cuda.synchronize()
    rc = ys.lib.ys_set_fields_dev(s2.h, 0, *[dev[k].data_ptr() for k in keys], None)
    assert rc == ys.YS_OK
    s1.set_fields(0, *[f0[k] for k in keys])
    s1.step(2, 2)
    s2.step(2, 2)
    g1, g2 = s1.get_fields(0), s2.get_fields(0)
    for k in keys:
        assert np.array_equal(g1[k], g2[k]), k


def test_caller_stream_gives_the_same_fields(gpu_lib):
    """Running a context on a caller-provided stream (ys_set_stream, e.g. a
    torch stream) changes where the work is queued, not what it computes:
    the fields after three steps are equal bit for bit, and the context's own
    stream can be taken back."""
    import torch
    ys = gpu_lib
    _, s1, _, _ = make_pair(ys, with_oracle=False)
    _, s2, _, _ = make_pair(ys, with_oracle=False)
    stream = torch.cuda.Stream()
    s2.set_stream(stream.cuda_stream)
    s1.step(3, 2)
    s2.step(3, 2)
    g1, g2 = s1.get_fields(0), s2.get_fields(0)
    s2.set_stream(0)
    s2.step(1, 2)
    s1.step(1, 2)
    h1, h2 = s1.get_fields(0), s2.get_fields(0)
    for k in ("T", "ur", "uth", "uph", "p"):
        assert np.array_equal(g1[k], g2[k]), k
        assert np.array_equal(h1[k], h2[k]), k


def test_pinned_and_pageable_host_buffers_agree(gpu_lib):
    """set/get through page-locked host buffers (read and written by the
    (un)pack kernels over the CPU-GPU link) and through pageable ones (staged
    copies) give the same state and the same fields, bit for bit."""
    import torch
    ys = gpu_lib
    o, s1, spec, ex = make_pair(ys, with_oracle=False)
    _, s2, _, _ = make_pair(ys, with_oracle=False)
    f0 = W.sample_fields(ex, spec, 0.0)
    pinned = {}
    for k, a in f0.items():
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        pinned[k] = t.numpy()
    s2.set_fields(0, *[pinned[k] for k in ("T", "ur", "uth", "uph", "p")])
    s1.set_fields(0, *[f0[k] for k in ("T", "ur", "uth", "uph", "p")])
    s1.step(2, 2)
    s2.step(2, 2)
    out = {k: torch.empty(a.shape, dtype=torch.float64, pin_memory=True).numpy() for k, a in f0.items()}
    rc = ys.lib.ys_get_fields(s2.h, 0, *[ys._ptr(out[k]) for k in ("T", "ur", "uth", "uph", "p")], None)
    assert rc == ys.YS_OK
    g1 = s1.get_fields(0)
    for k in ("T", "ur", "uth", "uph", "p"):
        assert np.array_equal(g1[k], out[k]), k


@pytest.mark.parametrize("Nph", [300, 400, 576])
def test_long_phi_lines_take_the_wide_and_multi_chunk_scans(gpu_lib, Nph):
    """phi lines of 300, 400 and 576 positions on a thin 8 x 12 shell: the
    warp-scan line solves give each lane 12 consecutive positions, as on the
    128 x 128 x 384 shell; 300 fits one chunk of 384 with a ragged end, 400
    and 576 take a full chunk of 384 and then a ragged one (16 and 192
    positions), the path of lines longer than 384.  FP64 against the oracle
    at the 1e-11 parity bound after 3 steps of 3 iterations.

    The mixed form: T and velocity within 1e-5 of the oracle.  Its pressures
    are bounded by the storage itself: a velocity stored in FP32 carries a
    relative rounding of 6e-8, whose discrete divergence, ~6e-8 |u| / (chi h),
    enters the pressure update at every step, and the phi cells here are 40
    times narrower than the theta cells.  The test measures that floor on
    the same grid: the FP64 path started from the initial fields rounded to
    FP32 once.  The mixed pressures must stay within 10 times its distance to
    the oracle (and the stated 1e-5 where the floor allows)."""
    from tests.test_gpu_mixed import rel_errs as mixed_errs
    ys = gpu_lib
    kw = dict(kind="curl", Nr=8, Nth=12, Nph=Nph, dt=1e-4, Ra=50.0)
    o, s, _, _ = make_pair(ys, **kw)
    _, sm, _, _ = make_pair(ys, **kw, with_oracle=False, precision=ys.YS_MIXED)
    o.step(3, 3)
    s.step(3, 3)
    sm.step(3, 3)
    ref = o.get_fields(0, aux=True)
    e = assert_parity(s, o, 1e-11)
    em = mixed_errs(sm.get_fields(0, aux=True), ref)
    # the FP32 storage floor of the pressure on this grid
    spec = W.Spec(0.5, 1.0, 8, 12, Nph)
    ex = W.CurlShell(0.5, 1.0, 1.0, 50.0)
    s32 = gpu_lib.Solver(R1=0.5, R2=1.0, Pr=1.0, Ra=50.0, dt=1e-4, Nr=8, Nth=12, Nph=Nph)
    for lvl, t in ((0, 0.0), (1, -1e-4)):
        f = W.sample_fields(ex, spec, t)
        s32.set_fields_dict(lvl, {k: v.astype(np.float32).astype(np.float64) for k, v in f.items()})
    for m, (tid, F) in enumerate(W.forcing_modes(ex, spec)):
        s32.set_forcing(m, tid, F["T"], F["ur"], F["uth"], F["uph"])
    s32.step(3, 3)
    floor = mixed_errs(s32.get_fields(0, aux=True), ref)
    print(Nph, e, em, floor)
    assert max(v for k, v in em.items() if k not in ("p", "p1")) <= 1e-5, em
    for k in ("p", "p1"):
        assert em[k] <= max(1e-5, 10.0 * floor[k]), (k, em[k], floor[k])


def blow_up_state(c=1e6):
    """Inconsistent time levels, a failure made on the host: the second-order
    velocity of level n-1 is twice that of level n, which is c times the curl
    solution, while the first-order system, T and p are at rest.  The
    extrapolated iterate is then c u, and the advecting velocity
    1.5 u^n - 0.5 u^{n-1} = c u / 2 is so large that the line operators lose
    diagonal dominance: the defect correction diverges within the step."""
    spec = W.Spec(0.5, 1.0, 16, 16, 48)
    f = W.sample_fields(W.CurlShell(0.5, 1.0, 1.0, 10.0), spec, 0.0)
    z = {k: np.zeros_like(v) for k, v in f.items()}
    aux = (z["ur"], z["uth"], z["uph"], z["p"])
    lv0 = dict(z, ur=c * f["ur"], uth=c * f["uth"], uph=c * f["uph"])
    lv1 = dict(z, ur=2 * c * f["ur"], uth=2 * c * f["uth"], uph=2 * c * f["uph"])
    return dict(R1=0.5, R2=1.0, Pr=1.0, Ra=10.0, dt=1e-3, Nr=16, Nth=16, Nph=48), lv0, lv1, aux


def test_schwarz_blow_up_is_reported_while_the_norms_are_finite(gpu_lib):
    """The divergence watch: on the blow-up state the oracle's largest
    increment norm grows more than 1e3-fold from the second iteration to the
    third, all finite.  ys_step with 2 iterations (nothing to compare: the
    watch starts at the third) returns OK, with 3 it returns YS_EDIVERGED
    although every norm it read back is finite (the NaN test alone would not
    trip)."""
    ys = gpu_lib
    kw, lv0, lv1, aux = blow_up_state()
    o = Oracle(Params(**kw))
    o.set_fields(0, lv0["T"], lv0["ur"], lv0["uth"], lv0["uph"], lv0["p"], aux=aux)
    o.set_fields(1, lv1["T"], lv1["ur"], lv1["uth"], lv1["uph"], lv1["p"], aux=aux)
    rec = []
    iterate = o._iterate

    def watched(*a, **k):
        r = iterate(*a, **k)
        rec.append(float(np.max(r)))
        return r

    o._iterate = watched
    o.step(1, 3)
    assert np.isfinite(rec).all() and rec[2] > 1e3 * rec[1], rec
    for K, expect in ((2, ys.YS_OK), (3, ys.YS_EDIVERGED)):
        s = ys.Solver(**kw)
        s.set_fields_dict(0, lv0, aux)
        s.set_fields_dict(1, lv1, aux)
        rc = ys.lib.ys_step(s.h, 1, K)
        assert rc == expect, (K, rc)
        nrm, it = s.norms()
        assert it == K and np.isfinite(nrm).all(), nrm
        s.close()
