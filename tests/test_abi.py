"""The C-ABI library loads and exports every function include/ys.h declares (a
plain C program can include the header and link it); argument validation, the
host-only entries and the serving queue's admission checks work without a GPU
(no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ys_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02300_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared("ys.h")
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_validation_without_gpu():
    from paper_1905_02300_gb300 import ys
    bad = [dict(R1=0.0, R2=1.0), dict(R1=1.0, R2=0.5), dict(dt=0.0), dict(Nr=4), dict(Nph=10, Nth=16),
           dict(chi=0.0), dict(Nth=13, Nph=13, Nr=8)]   # last: too coarse for the exchange
    for b in bad:
        kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=1e-3, Nr=16, Nth=16, Nph=48)
        kw.update(b)
        with pytest.raises(ys.YSError) as e:
            ys.Solver(**kw)
        assert e.value.code == ys.YS_EINVAL, (b, e.value)


def test_strerror_and_defaults():
    from paper_1905_02300_gb300 import ys
    assert ys.lib.ys_strerror(ys.YS_EDIVERGED) == b"diverged (NaN/Inf or Schwarz blow-up)"
    assert ys.lib.ys_strerror(ys.YS_ETIMEOUT) == b"deadline passed"
    assert ys.lib.ys_strerror(ys.YS_ECANCELED) == b"cancelled"
    p = ys.default_params()
    assert p.chi == 1.0 and p.overlap == 2 and p.step7 == 1 and p.precision == ys.YS_FP64


def test_invalid_radial_half_points_rejected_without_gpu():
    """Non-uniform radial grids: radii that do not increase, or do not start at
    R1 / end at R2, are rejected before any device work (YS_EINVAL); a wrong
    count is caught by the binding."""
    import numpy as np
    from paper_1905_02300_gb300 import ys, workloads as W
    kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=1e-3, Nr=16, Nth=16, Nph=48)
    good = np.array(W.stretched_radii(0.5, 1.0, 16, 0.5))
    bad = [good[::-1].copy(), good + 0.01, np.concatenate([good[:5], good[5:6], good[5:-1]])]
    for b in bad:
        with pytest.raises(ys.YSError) as e:
            ys.Solver(**kw, r_half=b)
        assert e.value.code == ys.YS_EINVAL
    with pytest.raises(ValueError):
        ys.Solver(**kw, r_half=good[:-1])
    with pytest.raises(ValueError):    # every path to the library, not only the Solver
        ys.default_params(**kw, r_half=np.concatenate([good, good[-1:] + 0.1]))



def _layout_bytes(Nr, Nt, Np, mixed, rec_counts, line_count, x_count):
    """Bytes of one shell's device allocation from the field layout of
    include/ys.h: 75 bulk fields (3 levels x 7 unknowns, 3 advecting
    velocities, 4 forcing combinations, 2 work fields, 36 line-factor fields,
    9 per-step sums of the advecting velocity) of the precision's size, in
    FP64 5 more (the two-level sums of the velocity and of T and the
    bootstrapped momentum pressure that the residuals and pressure updates
    read), 6 FP64 pressures, in FP64 the phi factors' lane-segment products,
    the 14 metric tables of max(Nr, Nth) + 6 entries (FP64 and
    FP32 pairs), the row tables (FP64 and FP32, each padded to 32 entries),
    the exchange entries (72 bytes each: 6 ints, 6 doubles), 4 deviation profiles of Nr + 2
    values, the norms and the staging buffer of the largest face-centred
    field; each part rounded up to 256 bytes."""
    r256 = lambda b: (b + 255) // 256 * 256
    P = ((Np + 2) + 7) // 8 * 8
    total = 2 * (((Nr + 2) * (Nt + 2) * P + 16 + 31) // 32 * 32)
    R = 4 if mixed else 8
    met = 14 * (max(Nr, Nt) + 6)
    rows = sum((n + 31) // 32 * 32 for n in rec_counts) + (line_count + 31) // 32 * 32
    stage = 2 * max((Nr + 1) * Nt * Np, Nr * (Nt + 1) * Np, Nr * Nt * (Np + 1))
    bulk = 75 if mixed else 80
    # FP64: 8 arrays of lane-segment products of the phi factors, 32 per
    # chunk of 32 ec positions of each of 2 Nr Nt lines
    ec = 4 if Np <= 128 else 8 if Np <= 256 else 12
    chunks = -(-Np // (32 * ec))
    segs = 0 if mixed else r256(8 * 2 * Nr * Nt * 32 * chunks * 8)
    return (r256(bulk * total * R) + r256(6 * total * 8) + segs + r256(met * 8) + r256(2 * met * 4) + r256(rows * 8)
            + r256(rows * 4) + r256(x_count * 72) + r256(4 * (Nr + 2) * 8) + 256 + stage * 8)


@pytest.mark.parametrize("dims", [(8, 12, 36), (16, 16, 48), (13, 17, 51), (128, 128, 384)])
@pytest.mark.parametrize("mixed", [False, True])
def test_shell_device_bytes_match_the_layout(dims, mixed):
    """ys_shell_device_bytes (what ys_create_ex allocates and the serving queue
    admits by) counts every part of the documented layout; a stretched radial
    grid takes the same memory; invalid parameters give 0."""
    import numpy as np
    from paper_1905_02300_gb300 import ys, workloads as W
    Nr, Nt, Np = dims
    kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=1e-3, Nr=Nr, Nth=Nt, Nph=Np,
              precision=ys.YS_MIXED if mixed else ys.YS_FP64)
    p = ys.default_params(**kw)
    n, rec = ctypes.c_size_t(0), ctypes.c_int(0)
    recs = []
    for t in range(5):
        assert ys.lib.ys_residual_coefficients(ctypes.byref(p), t, None, 0, ctypes.byref(n), ctypes.byref(rec)) == 0
        recs.append(n.value)
    assert ys.lib.ys_line_coefficients(ctypes.byref(p), None, 0, ctypes.byref(n)) == 0
    line = n.value
    xc = 0
    for k in range(5):
        assert ys.lib.ys_exchange_table(ctypes.byref(p), k, None, 0, ctypes.byref(n)) == 0
        xc += n.value // 12
    got = ys.lib.ys_shell_device_bytes(ctypes.byref(p))
    assert got == _layout_bytes(Nr, Nt, Np, mixed, recs, line, xc)
    ps = ys.default_params(**kw, r_half=np.array(W.stretched_radii(0.5, 1.0, Nr, 0.5)))
    assert ys.lib.ys_shell_device_bytes(ctypes.byref(ps)) == got
    bad = ys.default_params(**dict(kw, Nr=4))
    assert ys.lib.ys_shell_device_bytes(ctypes.byref(bad)) == 0
    assert ys.lib.ys_shell_device_bytes(None) == 0


def test_server_rejects_unfit_and_invalid_requests_at_submit():
    """The serving queue refuses, before any device work, a request whose
    shell can never fit its memory budget and one with invalid parameters
    (YS_EINVAL), and one with a non-uniform radial grid."""
    import numpy as np
    from paper_1905_02300_gb300 import ys, workloads as W
    kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=1e-3, Nr=16, Nth=16, Nph=48)
    p = ys.default_params(**kw)
    need = ys.lib.ys_shell_device_bytes(ctypes.byref(p))
    h = ctypes.c_void_p()
    assert ys.lib.ys_server_create(need // 2, 4, ctypes.byref(h)) == ys.YS_OK
    try:
        init = np.zeros(2 * 16 * 16 * 48 * 5 + 2 * (16 * 48 + 16 * 48 + 16 * 16))   # packed [T|ur|uth|uph|p]
        t = ctypes.c_uint64()
        ptr = init.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        assert ys.lib.ys_submit(h, ctypes.byref(p), ptr, 3, 2, ctypes.byref(t)) == ys.YS_EINVAL
        bad = ys.default_params(**dict(kw, Nr=4))
        assert ys.lib.ys_submit(h, ctypes.byref(bad), ptr, 3, 2, ctypes.byref(t)) == ys.YS_EINVAL
        st = ys.default_params(**kw, r_half=np.array(W.stretched_radii(0.5, 1.0, 16, 0.5)))
        assert ys.lib.ys_submit(h, ctypes.byref(st), ptr, 3, 2, ctypes.byref(t)) == ys.YS_EINVAL
        running, queued = ctypes.c_int(-1), ctypes.c_int(-1)
        assert ys.lib.ys_server_stats(h, None, None, ctypes.byref(running), ctypes.byref(queued), None) == ys.YS_OK
        assert running.value == 0 and queued.value == 0
    finally:
        assert ys.lib.ys_server_destroy(h) == ys.YS_OK


def test_server_deadline_cancel_and_queue_limit_arguments_without_gpu():
    """Host-side checks of the serving controls, before any device work: a
    negative or NaN deadline is refused at submit, cancelling an unknown
    ticket is refused, and the queue limit must lie in 1..4096 (YS_EINVAL)."""
    import math
    import numpy as np
    from paper_1905_02300_gb300 import ys
    kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=1e-3, Nr=16, Nth=16, Nph=48)
    p = ys.default_params(**kw)
    h = ctypes.c_void_p()
    assert ys.lib.ys_server_create(1 << 30, 4, ctypes.byref(h)) == ys.YS_OK
    try:
        init = np.zeros(2 * 16 * 16 * 48 * 5 + 2 * (16 * 48 + 16 * 48 + 16 * 16))
        ptr = init.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        t = ctypes.c_uint64()
        for d in (-1.0, math.nan):
            assert ys.lib.ys_submit_ex(h, ctypes.byref(p), ptr, 3, 2, d, ctypes.byref(t)) == ys.YS_EINVAL
        assert ys.lib.ys_cancel(h, ctypes.c_uint64(12345)) == ys.YS_EINVAL
        for q in (0, -3, 4097):
            assert ys.lib.ys_server_set_queue_limit(h, q) == ys.YS_EINVAL
        assert ys.lib.ys_server_set_queue_limit(h, 2) == ys.YS_OK
    finally:
        assert ys.lib.ys_server_destroy(h) == ys.YS_OK


def test_server_binding_checks_the_packed_field_length():
    """The binding refuses fields whose packed length is not the shell's (the
    library would read past the caller's buffer); with the right length, a
    shell larger than the budget is refused by the library."""
    import numpy as np
    from paper_1905_02300_gb300 import ys
    Nr, Nt, Np = 8, 12, 36
    kw = dict(R1=0.5, R2=1.0, Pr=1.0, Ra=0.0, dt=1e-3, Nr=Nr, Nth=Nt, Nph=Np)
    f = {"T": np.zeros((2, Nr, Nt, Np)), "ur": np.zeros((2, Nr + 1, Nt, Np)), "uth": np.zeros((2, Nr, Nt + 1, Np)),
         "uph": np.zeros((2, Nr, Nt, Np + 1)), "p": np.zeros((2, Nr, Nt, Np))}
    for budget, fields in ((1 << 30, dict(f, p=np.zeros((2, Nr, Nt, Np - 1)))), (1 << 10, f)):
        srv = ys.Server(hbm_budget_bytes=budget, max_slots=2)
        try:
            with pytest.raises(ys.YSError) as e:
                srv.submit(fields, 2, **kw)
            assert e.value.code == ys.YS_EINVAL
        finally:
            srv.close()


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "ys.h"

int main(void) {
  ys_params p;
  size_t n = 0, bytes;
  ys_default_params(&p);
  p.R1 = 0.5; p.R2 = 1.0; p.Pr = 1.0; p.Ra = 1e3; p.dt = 1e-3;
  p.Nr = 8; p.Nth = 12; p.Nph = 36;
  bytes = ys_shell_device_bytes(&p);
  if (bytes == 0) return 2;
  if (ys_exchange_table(&p, 4, NULL, 0, &n) != YS_OK || n == 0 || n % 12 != 0) return 3;
  p.dt = 0.0;
  if (ys_shell_device_bytes(&p) != 0) return 4;
  if (strlen(ys_strerror(YS_EINVAL)) == 0) return 5;
  printf("%zu %zu\n", bytes, n / 12);
  return 0;
}
"""


def test_header_is_plain_c_and_the_library_links_from_c(tmp_path):
    """A C99 program includes include/ys.h, links libys.so and calls host-only
    entries through the C ABI (no Python, no GPU): the header is plain C and
    the exported names are unmangled."""
    import shutil
    import subprocess
    from paper_1905_02300_gb300 import build
    from paper_1905_02300_gb300 import ys
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), lib,
                        "-Wl,-rpath," + libdir, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    bytes_, npts = map(int, r.stdout.split())
    p = ys.default_params(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, dt=1e-3, Nr=8, Nth=12, Nph=36)
    assert bytes_ == ys.lib.ys_shell_device_bytes(ctypes.byref(p))
    assert npts == 2 * 36 + 2 * 12 - 4     # the pressure ring of a 12 x 36 patch
