"""Thin ctypes binding of libgpsoc (include/gpsoc.h).  Argument marshalling only:
every numerical step runs in the library's CUDA kernels.  Importing works
without a GPU; creating a problem needs the built library and a CUDA device and
raises GpsocError otherwise (there is no CPU fallback)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpsoc.so")

GPSOC_FP64, GPSOC_MIXED, GPSOC_HYBRID = 0, 1, 2
GPSOC_STOP_DPHI, GPSOC_STOP_RES, GPSOC_STOP_ENERGY = 1, 2, 3
TRAP_HARMONIC, TRAP_HARMONIC_QUARTIC, TRAP_USER = 0, 1, 2
_STATUS = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTCONV", "ENONFINITE", "ETIMEOUT", "ESTATE", "EBUDGET",
           "ESTAGNATED", "ECANCELED"]


def status_name(code: int) -> str:
    return _STATUS[code] if 0 <= code < len(_STATUS) else f"status {code}"


class GpsocError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{status_name(code)}: {msg}")
        self.code = code


# GPSOC_PRECOND_*: combined P_C, kinetic P_Delta alone, potential P_V alone, none
PRECONDS = ("combined", "kinetic", "potential", "none")


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3)]


class Trap(C.Structure):
    _fields_ = [("kind", C.c_int), ("g", C.c_double * 3), ("quad", C.c_double), ("quart", C.c_double),
                ("user_V", C.POINTER(C.c_double))]


class Params(C.Structure):
    _fields_ = [("Omega", C.c_double), ("gamma", C.c_double), ("beta0", C.c_double), ("beta1", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("stop", C.c_int), ("tol", C.c_double), ("res_tol", C.c_double),
                ("max_iter", C.c_int), ("theta_trial", C.c_double), ("sigma", C.c_double),
                ("max_halvings", C.c_int), ("cm_levels", C.c_int), ("check_every", C.c_int),
                ("fp32_switch", C.c_double), ("fp32_min_points", C.c_int), ("precond", C.c_int),
                ("fp32_res_switch", C.c_double), ("fp32_carry", C.c_int), ("hybrid_refresh", C.c_int),
                ("hybrid_lead_res", C.c_double), ("line_search", C.c_int)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("total_iters", C.c_int), ("levels", C.c_int),
                ("beta_resets", C.c_int), ("halvings", C.c_int), ("fp32_iters", C.c_int), ("fp64_iters", C.c_int),
                ("energy", C.c_double), ("mu", C.c_double), ("mass", C.c_double * 3), ("res_inf", C.c_double),
                ("dE_last", C.c_double), ("level_iters", C.c_int * 8), ("level_fp32_iters", C.c_int * 8),
                ("level_res_fp32", C.c_double * 8)]

    def as_dict(self):
        return {"status": status_name(self.status), "iters": self.iters, "total_iters": self.total_iters,
                "levels": self.levels, "beta_resets": self.beta_resets, "halvings": self.halvings,
                "fp32_iters": self.fp32_iters, "fp64_iters": self.fp64_iters, "energy": self.energy,
                "mu": self.mu, "mass": list(self.mass), "res_inf": self.res_inf, "dE_last": self.dE_last,
                "level_iters": list(self.level_iters[:max(self.levels, 1)]),
                "level_fp32_iters": list(self.level_fp32_iters[:max(self.levels, 1)]),
                "level_res_fp32": list(self.level_res_fp32[:max(self.levels, 1)])}


class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("slots_per_bucket", C.c_int), ("precision", C.c_int),
                ("iters_per_step", C.c_int)]


_lib = None

_PROTOS = {
    "gpsoc_create": (C.c_int, [C.POINTER(Grid), C.POINTER(Trap), C.POINTER(Params), C.c_int, C.c_void_p,
                               C.POINTER(C.c_void_p)]),
    "gpsoc_destroy": (None, [C.c_void_p]),
    "gpsoc_solve_size": (C.c_size_t, [C.c_void_p, C.c_int]),
    "gpsoc_set_initial": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "gpsoc_set_initial_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "gpsoc_set_initial_kind": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int]),
    "gpsoc_solve": (C.c_int, [C.c_void_p, C.POINTER(Opts), C.POINTER(Result)]),
    "gpsoc_iterate": (C.c_int, [C.c_void_p, C.POINTER(Opts), C.c_int, C.c_int, C.POINTER(Result)]),
    "gpsoc_get_psi": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gpsoc_get_psi_device": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gpsoc_get_observables": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gpsoc_apply_h": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "gpsoc_apply_precond": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "gpsoc_step_model": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "gpsoc_prolong": (C.c_int, [C.c_void_p, C.c_int]),
    "gpsoc_fft_axis": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "gpsoc_profile": (C.c_int, [C.c_void_p, C.POINTER(Opts), C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "gpsoc_profile_name": (C.c_char_p, [C.c_void_p, C.c_int]),
    "gpsoc_kernel_launches": (C.c_uint64, [C.c_void_p]),
    "gpsoc_tile_shape": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int)]),
    "gpsoc_tile_candidates": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                        C.POINTER(C.c_int)]),
    "gpsoc_tuning_set": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "gpsoc_autotune": (C.c_int, [C.c_void_p, C.POINTER(Opts), C.c_int, C.c_void_p, C.c_void_p]),
    "gpsoc_probe_peaks": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "gpsoc_apply_h_noalloc": (C.c_int, [C.POINTER(Grid), C.POINTER(Trap), C.POINTER(Params), C.c_int, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p]),
    "gpsoc_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(C.c_void_p)]),
    "gpsoc_server_destroy": (None, [C.c_void_p]),
    "gpsoc_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Grid), C.POINTER(Trap), C.POINTER(Params), C.c_void_p,
                                      C.POINTER(Opts), C.POINTER(C.c_uint64)]),
    "gpsoc_server_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "gpsoc_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.POINTER(Result), C.c_void_p]),
    "gpsoc_server_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "gpsoc_server_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "gpsoc_last_error": (C.c_char_p, []),
    "gpsoc_version": (C.c_char_p, []),
}


def library():
    """Load libgpsoc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GpsocError(3, f"{LIB_PATH} is missing: run paper_2602_17950_gb300.build.build() first")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(code):
    if code != 0:
        raise GpsocError(code, library().gpsoc_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def probe_peaks():
    """(FP64, FP32) FMA throughput of the current device in TFLOP/s."""
    a, b = C.c_double(0), C.c_double(0)
    _check(library().gpsoc_probe_peaks(C.byref(a), C.byref(b)))
    return a.value, b.value


def apply_h_noalloc(n, L, params, trap, d_psi: int, d_hpsi: int, stream="torch") -> np.ndarray:
    """H(Phi) of the device states at d_psi into d_hpsi without any device
    allocation (gpsoc_apply_h_noalloc); returns the 9 observables per solve.
    For callers that cannot allocate device memory at this point."""
    dim = len(n)
    g = Grid(dim, (C.c_int * 3)(*(list(n) + [1] * (3 - dim))), (C.c_double * 3)(*(list(L) + [1.0] * (3 - dim))))
    trap = dict(trap or {})
    gv = list(trap.get("g", (1.0, 1.0, 1.0))) + [1.0] * 3
    t = Trap(int(trap.get("kind", 0)), (C.c_double * 3)(*gv[:3]), float(trap.get("quad", 0.0)),
             float(trap.get("quart", 0.0)), None)
    params = [tuple(p) for p in params]
    parr = (Params * len(params))(*[Params(*map(float, p)) for p in params])
    obs = np.zeros((len(params), 9))
    st = _current_stream() if stream == "torch" else stream
    code = library().gpsoc_apply_h_noalloc(C.byref(g), C.byref(t), parr, len(params), C.c_void_p(d_psi),
                                           C.c_void_p(d_hpsi), _ptr(obs), st)
    if code != 0:   # this entry point reports through its status only
        raise GpsocError(code, "gpsoc_apply_h_noalloc failed")
    return obs


class Problem:
    """A batch of ground-state problems sharing grid and trap (gpsoc_create).

    n, L: grid sizes and box half-widths per axis (2 or 3 entries).
    params: list of (Omega, gamma, beta0, beta1) per solve.
    trap: dict(kind=0|1|2, g=(gx, gy[, gz]), quad=, quart=, user_V=array)."""

    def __init__(self, n, L, params, trap=None, stream="torch"):
        lib = library()
        self.dim = len(n)
        g = Grid(self.dim, (C.c_int * 3)(*(list(n) + [1] * (3 - self.dim))),
                 (C.c_double * 3)(*(list(L) + [1.0] * (3 - self.dim))))
        trap = dict(trap or {})
        gv = list(trap.get("g", (1.0, 1.0, 1.0))) + [1.0] * 3
        self._userV = None
        uv = None
        if trap.get("user_V") is not None:
            self._userV = np.ascontiguousarray(trap["user_V"], dtype=np.float64)
            uv = self._userV.ctypes.data_as(C.POINTER(C.c_double))
        t = Trap(int(trap.get("kind", 0)), (C.c_double * 3)(*gv[:3]), float(trap.get("quad", 0.0)),
                 float(trap.get("quart", 0.0)), uv)
        params = [tuple(p) for p in params]
        self.batch = len(params)
        parr = (Params * self.batch)(*[Params(*map(float, p)) for p in params])
        st = _current_stream() if stream == "torch" else stream
        h = C.c_void_p()
        _check(lib.gpsoc_create(C.byref(g), C.byref(t), parr, self.batch, st, C.byref(h)))
        self._h = h
        self.n = tuple(n)
        self.L = tuple(L)
        self.level = 0

    # -------------------------------------------------------------- helpers
    def shape(self, level=None):
        level = self.level if level is None else level
        return (self.batch, 3) + tuple(k >> level for k in self.n[::-1])

    def close(self):
        if getattr(self, "_h", None):
            library().gpsoc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def opts(precision=GPSOC_FP64, stop=GPSOC_STOP_ENERGY, tol=1e-12, res_tol=0.0, max_iter=100000,
             theta_trial=0.0, sigma=0.0, max_halvings=0, cm_levels=1, check_every=0, fp32_switch=0.0,
             fp32_min_points=0, precond="combined", fp32_res_switch=0.0, fp32_carry=0, hybrid_refresh=0,
             hybrid_lead_res=0.0, line_search=0):
        pk = PRECONDS.index(precond) if isinstance(precond, str) else int(precond)
        return Opts(precision, stop, tol, res_tol, max_iter, theta_trial, sigma, max_halvings, cm_levels,
                    check_every, fp32_switch, fp32_min_points, pk, fp32_res_switch, int(fp32_carry),
                    int(hybrid_refresh), float(hybrid_lead_res),
                    1 if line_search in (1, "exact") else 0)

    # -------------------------------------------------------------- state
    def set_initial(self, psi: np.ndarray, level=0):
        psi = np.ascontiguousarray(psi, dtype=np.complex128).reshape(self.shape(level))
        _check(library().gpsoc_set_initial(self._h, _ptr(psi), level))
        self.level = level

    def set_initial_device(self, dptr: int, is_fp32=False, level=0):
        _check(library().gpsoc_set_initial_device(self._h, C.c_void_p(dptr), int(is_fp32), level))
        self.level = level

    def set_initial_kind(self, kinds, level=0):
        k = (C.c_int * 3)(*kinds)
        _check(library().gpsoc_set_initial_kind(self._h, k, level))
        self.level = level

    def psi(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape(), dtype=np.complex128)
        assert out.dtype == np.complex128 and out.flags.c_contiguous and out.size == np.prod(self.shape())
        _check(library().gpsoc_get_psi(self._h, _ptr(out)))
        return out

    def psi_to_device(self, dptr: int):
        _check(library().gpsoc_get_psi_device(self._h, C.c_void_p(dptr)))

    def observables(self):
        E = np.empty(self.batch)
        mu = np.empty(self.batch)
        m = np.empty((self.batch, 3))
        _check(library().gpsoc_get_observables(self._h, _ptr(E), _ptr(mu), _ptr(m)))
        return E, mu, m

    # -------------------------------------------------------------- solver
    def solve(self, raise_on_error=True, **kw):
        o = self.opts(**kw)
        res = (Result * self.batch)()
        code = library().gpsoc_solve(self._h, C.byref(o), res)
        if code in (0, 4, 5, 9):      # per-solve outcomes are reported in the results
            self.level = 0
        elif raise_on_error:
            _check(code)
        return [r.as_dict() for r in res]

    def iterate(self, iters, restart=True, **kw):
        o = self.opts(**kw)
        res = (Result * self.batch)()
        _check(library().gpsoc_iterate(self._h, C.byref(o), int(iters), int(restart), res))
        return [r.as_dict() for r in res]

    # -------------------------------------------------------------- operators
    def apply_h(self, precision=GPSOC_FP64):
        """H_l(Phi) and 9 observables per solve; precision=GPSOC_MIXED runs the FP32 kernels."""
        hp = np.empty(self.shape(), dtype=np.complex128)
        obs = np.empty((self.batch, 9))
        _check(library().gpsoc_apply_h(self._h, int(precision), _ptr(hp), _ptr(obs)))
        return hp, obs

    def apply_precond(self, r: np.ndarray, precision=GPSOC_FP64):
        r = np.ascontiguousarray(r, dtype=np.complex128).reshape(self.shape())
        out = np.empty_like(r)
        _check(library().gpsoc_apply_precond(self._h, int(precision), _ptr(r), _ptr(out)))
        return out

    def step_model(self, P: np.ndarray, thetas, precision=GPSOC_FP64):
        P = np.ascontiguousarray(P, dtype=np.complex128).reshape(self.shape())
        th = np.ascontiguousarray(thetas, dtype=np.float64)
        out = np.empty((self.batch, 2 + th.size))
        _check(library().gpsoc_step_model(self._h, int(precision), _ptr(P), _ptr(th), th.size, _ptr(out)))
        return out

    def prolong(self):
        _check(library().gpsoc_prolong(self._h, self.level))
        self.level -= 1

    def profile(self, iters=10, **kw):
        """Per-kernel average durations (ms) of one PCG iteration, CUDA events on the problem's stream."""
        o = self.opts(**kw)
        ms = np.zeros(128)
        nk = C.c_int(0)
        _check(library().gpsoc_profile(self._h, C.byref(o), int(iters), _ptr(ms), 128, C.byref(nk)))
        names = [library().gpsoc_profile_name(self._h, k).decode() for k in range(nk.value)]
        return list(zip(names, ms[:nk.value].tolist()))

    def kernel_launches(self) -> int:
        return int(library().gpsoc_kernel_launches(self._h))

    def tile_candidates(self, axis, level=0, precision=GPSOC_FP64):
        """Valid (lines per tile, FFT elements per thread) pairs of the passes along `axis`."""
        cnt = C.c_int(0)
        _check(library().gpsoc_tile_candidates(self._h, int(level), int(axis), int(precision), None, None, 0,
                                               C.byref(cnt)))
        la = np.zeros(max(cnt.value, 1), dtype=np.int32)
        ea = np.zeros(max(cnt.value, 1), dtype=np.int32)
        _check(library().gpsoc_tile_candidates(self._h, int(level), int(axis), int(precision), _ptr(la), _ptr(ea),
                                               cnt.value, C.byref(cnt)))
        return list(zip(la[:cnt.value].tolist(), ea[:cnt.value].tolist()))

    def tuning_set(self, axis, lines, ept, level=0, precision=GPSOC_FP64):
        """Use this tile (lines = 0: the built-in rule) for every problem of this grid, batch, precision."""
        _check(library().gpsoc_tuning_set(self._h, int(level), int(axis), int(precision), int(lines), int(ept)))

    def autotune(self, iters=6, **kw):
        """Time every candidate tile of each axis on the current level; returns [(lines, ept)] per axis."""
        o = self.opts(**kw)
        la = np.zeros(3, dtype=np.int32)
        ea = np.zeros(3, dtype=np.int32)
        _check(library().gpsoc_autotune(self._h, C.byref(o), int(iters), _ptr(la), _ptr(ea)))
        return [(int(la[a]), int(ea[a])) for a in range(self.dim)]

    def tile_shape(self, axis, level=0, precision=GPSOC_FP64):
        """(lines per tile, FFT elements per thread, threads) of the passes along `axis`."""
        a, b, c = C.c_int(0), C.c_int(0), C.c_int(0)
        _check(library().gpsoc_tile_shape(self._h, int(level), int(axis), int(precision), C.byref(a), C.byref(b),
                                          C.byref(c)))
        return a.value, b.value, c.value

    def fft_axis(self, data_dptr: int, count: int, axis: int, inverse=False):
        _check(library().gpsoc_fft_axis(self._h, C.c_void_p(data_dptr), count, axis, int(inverse)))


def _grid_trap(n, L, trap):
    dim = len(n)
    g = Grid(dim, (C.c_int * 3)(*(list(n) + [1] * (3 - dim))), (C.c_double * 3)(*(list(L) + [1.0] * (3 - dim))))
    trap = dict(trap or {})
    gv = list(trap.get("g", (1.0, 1.0, 1.0))) + [1.0] * 3
    t = Trap(int(trap.get("kind", 0)), (C.c_double * 3)(*gv[:3]), float(trap.get("quad", 0.0)),
             float(trap.get("quart", 0.0)), None)
    return g, t


class Server:
    """Continuous-batching request server (gpsoc_server_*)."""

    def __init__(self, hbm_budget_bytes=120e9, slots_per_bucket=32, precision=GPSOC_FP64, iters_per_step=32):
        o = ServerOpts(float(hbm_budget_bytes), int(slots_per_bucket), int(precision), int(iters_per_step))
        h = C.c_void_p()
        _check(library().gpsoc_server_create(C.byref(o), C.byref(h)))
        self._h = h
        self._shapes = {}

    def close(self):
        if getattr(self, "_h", None):
            library().gpsoc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, n, L, params, psi0, trap=None, **opts):
        g, t = _grid_trap(n, L, trap)
        par = Params(*map(float, params))
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128).reshape((3,) + tuple(n[::-1]))
        o = Problem.opts(**opts)
        tk = C.c_uint64(0)
        _check(library().gpsoc_server_submit(self._h, C.byref(g), C.byref(t), C.byref(par), _ptr(psi0), C.byref(o),
                                             C.byref(tk)))
        self._shapes[tk.value] = (3,) + tuple(n[::-1])
        return tk.value

    def step(self) -> int:
        busy = C.c_int(0)
        _check(library().gpsoc_server_step(self._h, C.byref(busy)))
        return busy.value

    def poll(self, ticket, want_psi=True, timeout_ms=0):
        """(result dict, psi) once finished, else None.  timeout_ms > 0 drives the server
        until the request finishes or the time runs out; < 0 waits without limit."""
        res = Result()
        shape = self._shapes.get(ticket)    # unknown tickets are rejected by the library
        psi = np.empty(shape, dtype=np.complex128) if want_psi and shape is not None else None
        code = library().gpsoc_server_poll(self._h, C.c_uint64(ticket), int(timeout_ms), C.byref(res),
                                           _ptr(psi) if psi is not None else None)
        if code == 6:                    # ETIMEOUT: still queued or running
            return None
        _check(code)
        self._shapes.pop(ticket, None)
        if res.status == 10:             # ECANCELED: no wave function
            psi = None
        return res.as_dict(), psi

    def cancel(self, ticket):
        _check(library().gpsoc_server_cancel(self._h, C.c_uint64(ticket)))

    def stats(self):
        b = C.c_double(0)
        nb = C.c_int(0)
        q = C.c_int(0)
        _check(library().gpsoc_server_stats(self._h, C.byref(b), C.byref(nb), C.byref(q)))
        return {"bytes_in_use": b.value, "buckets": nb.value, "queued": q.value}
