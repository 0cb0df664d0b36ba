"""Python binding of the C ABI in include/ys.h (ctypes; marshalling only).

Every computation runs in the CUDA library libys.so; this module only moves
numpy buffers across the boundary.  Importing it loads the library and raises
if it is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libys.so")

YS_OK, YS_EINVAL, YS_ENOMEM, YS_ECUDA, YS_EDIVERGED, YS_ETIMEOUT, YS_EAGAIN, YS_EBUSY, YS_ECANCELED = range(9)
YS_FP64, YS_MIXED = 0, 1
YS_ADDITIVE, YS_MULTIPLICATIVE = 0, 1
NFIELDS = 9
FIELD_NAMES = ("T", "u1r", "u1t", "u1p", "p1", "u2r", "u2t", "u2p", "p2")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1905_02300_gb300.build.build()")
lib = C.CDLL(LIB_PATH)


class Params(C.Structure):
    _fields_ = [("R1", C.c_double), ("R2", C.c_double), ("Pr", C.c_double), ("Ra", C.c_double),
                ("dt", C.c_double), ("Nr", C.c_int), ("Nth", C.c_int), ("Nph", C.c_int),
                ("chi", C.c_double), ("overlap", C.c_int), ("precision", C.c_int),
                ("schwarz_mode", C.c_int), ("schwarz_tol", C.c_double), ("T_inner", C.c_double),
                ("T_outer", C.c_double), ("step7", C.c_int), ("step4", C.c_int), ("step4_eps", C.c_double),
                ("step4_tol", C.c_double), ("Tbc_inner_a", C.c_double), ("Tbc_inner_b", C.c_double),
                ("Tbc_outer_a", C.c_double), ("Tbc_outer_b", C.c_double), ("r_half", C.POINTER(C.c_double))]


_dp = C.POINTER(C.c_double)
_sig = {
    "ys_default_params": (None, [C.POINTER(Params)]),
    "ys_create": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                            C.c_double, C.POINTER(C.c_void_p)]),
    "ys_create_ex": (C.c_int, [C.POINTER(Params), C.POINTER(C.c_void_p)]),
    "ys_set_fields": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, _dp]),
    "ys_set_fields_ex": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]),
    "ys_set_fields_dev": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "ys_set_forcing": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp, _dp, _dp, _dp]),
    "ys_set_wall_velocity": (C.c_int, [C.c_void_p, _dp, _dp, _dp]),
    "ys_set_time": (C.c_int, [C.c_void_p, C.c_double]),
    "ys_set_wall_data": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp]),
    "ys_step": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "ys_get_fields": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]),
    "ys_get_stats": (C.c_int, [C.c_void_p, _dp, _dp, C.POINTER(C.c_long)]),
    "ys_get_norms": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int)]),
    "ys_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ys_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "ys_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_char_p), _dp, C.POINTER(C.c_long), C.c_int]),
    "ys_launch_count": (C.c_long, [C.c_void_p]),
    "ys_measure_fp64_rate": (C.c_int, [_dp]),
    "ys_device_bytes": (C.c_size_t, [C.c_void_p]),
    "ys_shell_device_bytes": (C.c_size_t, [C.POINTER(Params)]),
    "ys_destroy": (C.c_int, [C.c_void_p]),
    "ys_factor_solve_static": (C.c_int, [C.POINTER(Params), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]),
    "ys_line_coefficients": (C.c_int, [C.POINTER(Params), C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "ys_residual_coefficients": (C.c_int, [C.POINTER(Params), C.c_int, C.c_void_p, C.c_size_t,
                                           C.POINTER(C.c_size_t), C.POINTER(C.c_int)]),
    "ys_exchange_table": (C.c_int, [C.POINTER(Params), C.c_int, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "ys_strerror": (C.c_char_p, [C.c_int]),
    "ys_batch_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "ys_batch_add": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    "ys_batch_remove": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "ys_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "ys_batch_sync": (C.c_int, [C.c_void_p]),
    "ys_batch_norms": (C.c_int, [C.c_void_p, C.c_int, _dp]),
    "ys_batch_set_line_threads": (C.c_int, [C.c_void_p, C.c_int]),
    "ys_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "ys_batch_launches_per_step": (C.c_long, [C.c_void_p]),
    "ys_batch_destroy": (C.c_int, [C.c_void_p]),
    "ys_batch_stream": (C.c_void_p, [C.c_void_p]),
    "ys_batch_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "ys_batch_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_char_p), _dp, C.POINTER(C.c_long), C.c_int]),
    "ys_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]),
    "ys_submit": (C.c_int, [C.c_void_p, C.POINTER(Params), _dp, C.c_int, C.c_int, C.POINTER(C.c_uint64)]),
    "ys_submit_ex": (C.c_int, [C.c_void_p, C.POINTER(Params), _dp, C.c_int, C.c_int, C.c_double,
                               C.POINTER(C.c_uint64)]),
    "ys_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "ys_server_set_queue_limit": (C.c_int, [C.c_void_p, C.c_int]),
    "ys_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_int), _dp, _dp]),
    "ys_server_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_long), _dp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int)]),
    "ys_server_destroy": (C.c_int, [C.c_void_p]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def measure_fp64_rate():
    """Dense FP64 FMA rate of the current device, TFLOP/s (ys_measure_fp64_rate)."""
    v = C.c_double()
    _check(lib.ys_measure_fp64_rate(C.byref(v)), "ys_measure_fp64_rate")
    return v.value


class YSError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {lib.ys_strerror(code).decode()} ({code})")
        self.code = code


def _check(code, what):
    if code != YS_OK:
        raise YSError(code, what)


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def default_params(**kw) -> Params:
    """ys_params with the library defaults and the given fields.  r_half (a
    sequence of 2 Nr + 1 radii) is kept alive on the returned struct
    (attribute _r_half) for as long as the struct is."""
    p = Params()
    lib.ys_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        if k == "r_half":
            if v is None:
                p.r_half = None
                continue
            arr = np.ascontiguousarray(v, dtype=np.float64)
            p._r_half = arr
            p.r_half = arr.ctypes.data_as(_dp)
            continue
        setattr(p, k, v)
    rh = getattr(p, "_r_half", None)
    if rh is not None and rh.shape != (2 * p.Nr + 1,):
        raise ValueError("r_half: 2 Nr + 1 radii expected")   # the library reads exactly that many
    return p


class Solver:
    """One shell on the GPU (owns a ys_ctx)."""

    def __init__(self, **params):
        self.params = default_params(**params)
        h = C.c_void_p()
        _check(lib.ys_create_ex(C.byref(self.params), C.byref(h)), "ys_create_ex")
        self.h = h
        p = self.params
        Nr, Nt, Np = p.Nr, p.Nth, p.Nph
        self.shapes = {"T": (2, Nr, Nt, Np), "p": (2, Nr, Nt, Np), "ur": (2, Nr + 1, Nt, Np),
                       "uth": (2, Nr, Nt + 1, Np), "uph": (2, Nr, Nt, Np + 1)}

    def close(self):
        if getattr(self, "h", None):
            lib.ys_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arr(self, key, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != self.shapes[key]:
            raise ValueError(f"{key}: shape {a.shape} != {self.shapes[key]}")
        return a

    def set_fields(self, level, T, ur, uth, uph, p, aux=None):
        arrs = [self._arr("T", T), self._arr("ur", ur), self._arr("uth", uth), self._arr("uph", uph),
                self._arr("p", p)]
        auxp = None
        if aux is not None:
            auxp = np.ascontiguousarray(np.concatenate([self._arr("ur", aux[0]).ravel(), self._arr("uth", aux[1]).ravel(),
                                                        self._arr("uph", aux[2]).ravel(), self._arr("p", aux[3]).ravel()]))
        _check(lib.ys_set_fields_ex(self.h, level, *[_ptr(a) for a in arrs], _ptr(auxp)), "ys_set_fields_ex")

    def set_fields_dict(self, level, f, aux=None):
        self.set_fields(level, f["T"], f["ur"], f["uth"], f["uph"], f["p"], aux)

    def set_forcing(self, mode, time_fn, fT, fr, fth, fph):
        arrs = [self._arr("T", fT), self._arr("ur", fr), self._arr("uth", fth), self._arr("uph", fph)]
        _check(lib.ys_set_forcing(self.h, mode, time_fn, *[_ptr(a) for a in arrs]), "ys_set_forcing")

    def set_wall_velocity(self, walls):
        """Dirichlet wall velocity: dict 'ur' [2][2][Nth][Nph], 'uth'
        [2][2][Nth+1][Nph], 'uph' [2][2][Nth][Nph+1] (wall, patch, j, k);
        a missing key means no-slip for that component."""
        Nt, Np = self.params.Nth, self.params.Nph
        shapes = {"ur": (2, 2, Nt, Np), "uth": (2, 2, Nt + 1, Np), "uph": (2, 2, Nt, Np + 1)}
        arrs = []
        for k in ("ur", "uth", "uph"):
            a = walls.get(k)
            if a is not None:
                a = np.ascontiguousarray(a, dtype=np.float64)
                if a.shape != shapes[k]:
                    raise ValueError(f"{k}: shape {a.shape}, expected {shapes[k]}")
            arrs.append(a)
        _check(lib.ys_set_wall_velocity(self.h, *[_ptr(a) for a in arrs]), "ys_set_wall_velocity")

    def set_wall_data(self, time_fn, walls):
        """Time-dependent wall data tau(t) W: dict with any of 'T'
        [2][2][Nth][Nph] and 'ur', 'uth', 'uph' as in set_wall_velocity."""
        Nt, Np = self.params.Nth, self.params.Nph
        shapes = {"T": (2, 2, Nt, Np), "ur": (2, 2, Nt, Np), "uth": (2, 2, Nt + 1, Np), "uph": (2, 2, Nt, Np + 1)}
        arrs = []
        for k in ("T", "ur", "uth", "uph"):
            a = walls.get(k)
            if a is not None:
                a = np.ascontiguousarray(a, dtype=np.float64)
                if a.shape != shapes[k]:
                    raise ValueError(f"{k}: shape {a.shape}, expected {shapes[k]}")
            arrs.append(a)
        _check(lib.ys_set_wall_data(self.h, time_fn, *[_ptr(a) for a in arrs]), "ys_set_wall_data")

    def set_time(self, t):
        _check(lib.ys_set_time(self.h, t), "ys_set_time")

    def step(self, n_steps=1, n_schwarz=3):
        _check(lib.ys_step(self.h, n_steps, n_schwarz), "ys_step")

    def get_fields(self, level=0, aux=False):
        out = {k: np.empty(self.shapes[k]) for k in ("T", "ur", "uth", "uph", "p")}
        auxa = None
        if aux:
            n = sum(int(np.prod(self.shapes[k])) for k in ("ur", "uth", "uph", "p"))
            auxa = np.empty(n)
        _check(lib.ys_get_fields(self.h, level, _ptr(out["T"]), _ptr(out["ur"]), _ptr(out["uth"]),
                                 _ptr(out["uph"]), _ptr(out["p"]), _ptr(auxa)), "ys_get_fields")
        if aux:
            o = 0
            for k, key in (("ur", "ur1"), ("uth", "uth1"), ("uph", "uph1"), ("p", "p1")):
                n = int(np.prod(self.shapes[k]))
                out[key] = auxa[o:o + n].reshape(self.shapes[k])
                o += n
        return out

    def stats(self):
        nrm, t, steps = C.c_double(), C.c_double(), C.c_long()
        _check(lib.ys_get_stats(self.h, C.byref(nrm), C.byref(t), C.byref(steps)), "ys_get_stats")
        return {"norm": nrm.value, "t": t.value, "steps": steps.value}

    def norms(self):
        a = np.empty(NFIELDS)
        it = C.c_int()
        _check(lib.ys_get_norms(self.h, _ptr(a), C.byref(it)), "ys_get_norms")
        return a, it.value

    def set_stream(self, stream_handle):
        _check(lib.ys_set_stream(self.h, C.c_void_p(stream_handle)), "ys_set_stream")

    def profile(self, on=True):
        _check(lib.ys_profile_enable(self.h, 1 if on else 0), "ys_profile_enable")

    def profile_read(self):
        cap = 64
        names = (C.c_char_p * cap)()
        ms = (C.c_double * cap)()
        cnt = (C.c_long * cap)()
        n = lib.ys_profile_read(self.h, names, ms, cnt, cap)
        if n < 0:
            raise YSError(-n, "ys_profile_read")
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(n)}

    def launch_count(self):
        return lib.ys_launch_count(self.h)

    def device_bytes(self):
        return lib.ys_device_bytes(self.h)


class Batch:
    """Ensemble of shells advanced together (one launch per kernel class,
    one CUDA graph per step).  Solvers added to a batch are stepped only by it
    until removed."""

    def __init__(self, capacity, precision=YS_MIXED, n_schwarz=3):
        h = C.c_void_p()
        _check(lib.ys_batch_create(capacity, precision, n_schwarz, C.byref(h)), "ys_batch_create")
        self.h = h
        self.members = {}

    def add(self, solver):
        slot = C.c_int()
        _check(lib.ys_batch_add(self.h, solver.h, C.byref(slot)), "ys_batch_add")
        self.members[slot.value] = solver
        return slot.value

    def remove(self, slot):
        out = C.c_void_p()
        _check(lib.ys_batch_remove(self.h, slot, C.byref(out)), "ys_batch_remove")
        return self.members.pop(slot)

    def step(self, n=1):
        _check(lib.ys_batch_step(self.h, n), "ys_batch_step")

    def sync(self):
        _check(lib.ys_batch_sync(self.h), "ys_batch_sync")

    def norms(self, slot):
        a = np.empty(NFIELDS)
        _check(lib.ys_batch_norms(self.h, slot, _ptr(a)), "ys_batch_norms")
        return a

    def set_line_threads(self, t):
        _check(lib.ys_batch_set_line_threads(self.h, t), "ys_batch_set_line_threads")

    def autotune(self, trial_steps=2):
        ch = C.c_int()
        _check(lib.ys_batch_autotune(self.h, trial_steps, C.byref(ch)), "ys_batch_autotune")
        return ch.value

    def launches_per_step(self):
        return lib.ys_batch_launches_per_step(self.h)

    def stream_handle(self):
        return lib.ys_batch_stream(self.h)

    def profile(self, on=True):
        _check(lib.ys_batch_profile_enable(self.h, 1 if on else 0), "ys_batch_profile_enable")

    def profile_read(self):
        """{kernel class: (total ms, launches)} of the profiled steps."""
        cap = 32
        names = (C.c_char_p * cap)()
        ms = np.zeros(cap)
        cnt = (C.c_long * cap)()
        n = lib.ys_batch_profile_read(self.h, names, _ptr(ms), cnt, cap)
        if n < 0:
            raise YSError(-n, "ys_batch_profile_read")
        return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(n)}

    def close(self):
        if getattr(self, "h", None):
            for slot in list(self.members):
                self.remove(slot)
            lib.ys_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_fields(f):
    """[T | ur | uth | uph | p] packed as the serving API expects."""
    return np.concatenate([np.ascontiguousarray(f[k], dtype=np.float64).ravel()
                           for k in ("T", "ur", "uth", "uph", "p")])


def unpack_fields(buf, Nr, Nth, Nph):
    shapes = {"T": (2, Nr, Nth, Nph), "ur": (2, Nr + 1, Nth, Nph), "uth": (2, Nr, Nth + 1, Nph),
              "uph": (2, Nr, Nth, Nph + 1), "p": (2, Nr, Nth, Nph)}
    out, o = {}, 0
    for k in ("T", "ur", "uth", "uph", "p"):
        n = int(np.prod(shapes[k]))
        out[k] = buf[o:o + n].reshape(shapes[k])
        o += n
    return out


class Server:
    """Request loop with continuous batching (ys_server_*)."""

    QUEUED, RUNNING, DONE, FAILED = 0, 1, 2, 3

    def __init__(self, hbm_budget_bytes, max_slots, max_queue=None):
        h = C.c_void_p()
        _check(lib.ys_server_create(hbm_budget_bytes, max_slots, C.byref(h)), "ys_server_create")
        self.h = h
        self.shapes = {}
        if max_queue is not None:
            _check(lib.ys_server_set_queue_limit(self.h, max_queue), "ys_server_set_queue_limit")

    def cancel(self, ticket):
        _check(lib.ys_cancel(self.h, C.c_uint64(ticket)), "ys_cancel")

    def submit(self, fields, n_steps, n_schwarz=3, deadline_s=0.0, **params):
        p = default_params(**params)
        buf = pack_fields(fields)
        Nr, Nt, Np = p.Nr, p.Nth, p.Nph
        need = 2 * Nr * Nt * Np * 2 + 2 * (Nr + 1) * Nt * Np + 2 * Nr * (Nt + 1) * Np + 2 * Nr * Nt * (Np + 1)
        if buf.size != need:
            raise YSError(YS_EINVAL, "ys_submit: fields of %d values, the shell needs %d" % (buf.size, need))
        t = C.c_uint64()
        _check(lib.ys_submit_ex(self.h, C.byref(p), _ptr(buf), n_steps, n_schwarz, deadline_s, C.byref(t)),
               "ys_submit_ex")
        self.shapes[t.value] = (p.Nr, p.Nth, p.Nph)
        return t.value

    def poll(self, ticket, fields=True):
        """(state, fields or None, latency_s or None, error code); with
        fields=False the result is not copied out."""
        Nr, Nt, Np = self.shapes[ticket]
        n = 2 * Nr * Nt * Np * 2 + 2 * (Nr + 1) * Nt * Np + 2 * Nr * (Nt + 1) * Np + 2 * Nr * Nt * (Np + 1)
        buf = np.empty(n) if fields else None
        st, lat = C.c_int(), C.c_double()
        rc = lib.ys_poll(self.h, C.c_uint64(ticket), C.byref(st), _ptr(buf), C.byref(lat))
        if rc == YS_EAGAIN:
            return st.value, None, None, rc
        if rc != YS_OK:
            return st.value, None, lat.value, rc
        return st.value, unpack_fields(buf, Nr, Nt, Np) if fields else None, lat.value, rc

    def stats(self):
        steps, cu, run, q, pk = C.c_long(), C.c_double(), C.c_int(), C.c_int(), C.c_int()
        _check(lib.ys_server_stats(self.h, C.byref(steps), C.byref(cu), C.byref(run), C.byref(q), C.byref(pk)),
               "ys_server_stats")
        return {"steps": steps.value, "cell_updates": cu.value, "running": run.value, "queued": q.value,
                "peak_running": pk.value}

    def close(self):
        if getattr(self, "h", None):
            lib.ys_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
