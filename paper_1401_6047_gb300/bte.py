"""Python binding of the C ABI in ``include/bte.h`` (ctypes, argument
marshalling only).

Every step of the solver runs in the CUDA library ``_lib/libbte.so``; this
module converts Python values to the ABI's structs and host arrays and turns
non-zero status codes into exceptions.  There is no CPU fallback: if the
library cannot be loaded, or the GPU is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
FP64, FP32_MIXED = 0, 1
_NAMES = {0: "BTE_OK", -1: "BTE_EINVAL", -2: "BTE_ENOMEM", -3: "BTE_ECUDA",
          -4: "BTE_EUNSTABLE", -5: "BTE_ETIMEOUT", -6: "BTE_ESTATE"}


class BteError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class bte_params(ctypes.Structure):
    _fields_ = [
        ("E_dc", ctypes.c_double), ("E_omega", ctypes.c_double), ("omega", ctypes.c_double),
        ("B", ctypes.c_double), ("mu", ctypes.c_double), ("alpha", ctypes.c_double),
        ("phiy_min", ctypes.c_double), ("phiy_max", ctypes.c_double), ("dt", ctypes.c_double),
        ("periods", ctypes.c_double), ("t_max", ctypes.c_double), ("avg_window", ctypes.c_double),
        ("n_max", ctypes.c_int32), ("m_points", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("B_omega", ctypes.c_double), ("B_phase", ctypes.c_double),
    ]


class bte_obs(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("step", ctypes.c_int64), ("v_dr", ctypes.c_double),
        ("norm", ctypes.c_double), ("v_dc_avg", ctypes.c_double), ("absorption", ctypes.c_double),
        ("norm_max_abs_err", ctypes.c_double), ("dt_eff", ctypes.c_double),
        ("steps_total", ctypes.c_int64), ("steps_per_period", ctypes.c_int64),
        ("window_steps", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class bte_tuning(ctypes.Structure):
    _fields_ = [("tile_m", ctypes.c_int32), ("chunk_n", ctypes.c_int32),
                ("graph_steps", ctypes.c_int32), ("vec", ctypes.c_int32),
                ("resident", ctypes.c_int32), ("walk", ctypes.c_int32),
                ("wide_cols", ctypes.c_int32)]


class bte_batch_opts(ctypes.Structure):
    _fields_ = [("tile_m", ctypes.c_int32), ("chunk_n", ctypes.c_int32), ("vec", ctypes.c_int32),
                ("graph_steps", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("resident", ctypes.c_int32), ("max_batch_bytes", ctypes.c_int64),
                ("stream", ctypes.c_void_p), ("resident_smem", ctypes.c_int32),
                ("walk", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Loads libbte.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        if not _build.up_to_date():
            _build.build()
        L = ctypes.CDLL(_build.LIB)
        vp = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(bte_params)
        T = ctypes.POINTER(bte_tuning)
        i64 = ctypes.c_int64
        sig = {
            "bte_workspace_size": ([P, T, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
            "bte_create": ([P, vp, ctypes.POINTER(vp)], ctypes.c_int),
            "bte_create_ex": ([P, vp, T, vp, ctypes.c_size_t, ctypes.POINTER(vp)], ctypes.c_int),
            "bte_step": ([vp, i64], ctypes.c_int),
            "bte_run": ([vp], ctypes.c_int),
            "bte_reset": ([vp], ctypes.c_int),
            "bte_observables": ([vp, ctypes.POINTER(bte_obs)], ctypes.c_int),
            "bte_trace": ([vp, i64, i64, dp, dp], ctypes.c_int),
            "bte_get_state": ([vp, ctypes.c_int, dp, dp], ctypes.c_int),
            "bte_set_state": ([vp, ctypes.c_int, dp, dp], ctypes.c_int),
            "bte_set_step": ([vp, i64, dp, dp], ctypes.c_int),
            "bte_pdf": ([vp, ctypes.c_int, ctypes.c_int32, dp], ctypes.c_int),
            "bte_destroy": ([vp], None),
            "bte_last_error": ([], ctypes.c_char_p),
            "bte_bessel_ratio": ([ctypes.c_double, ctypes.c_int32, dp], ctypes.c_int),
            "bte_time_grid": ([P, dp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                               ctypes.POINTER(i64)], ctypes.c_int),
            "bte_version": ([], ctypes.c_char_p),
            "bte_observe_noalloc": ([P, vp, vp, vp, vp], ctypes.c_int),
            "bte_wait_probe": ([vp, i64], ctypes.c_int),
            "bte_launch_shape": ([P, T] + [ctypes.POINTER(ctypes.c_int32)] * 5, ctypes.c_int),
            "bte_batch_run": ([P, ctypes.c_int32, ctypes.POINTER(bte_obs),
                               ctypes.POINTER(bte_batch_opts)], ctypes.c_int),
            "bte_batch_plan": ([P, ctypes.c_int32, ctypes.POINTER(bte_batch_opts),
                                ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
            "bte_batch_tune": ([P, ctypes.c_int32, ctypes.POINTER(bte_batch_opts), ctypes.c_int32,
                                ctypes.c_int32, ctypes.POINTER(bte_batch_opts), dp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != OK:
        raise BteError(rc, lib().bte_last_error().decode())


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def to_params(p) -> bte_params:
    """Any object (or dict) with the solver parameter names -> bte_params."""
    g = (lambda k, d=None: p.get(k, d)) if isinstance(p, dict) else (lambda k, d=None: getattr(p, k, d))
    s = bte_params()
    for k in ("E_dc", "E_omega", "omega", "B", "mu", "alpha", "phiy_min", "phiy_max", "dt",
              "periods", "t_max", "avg_window"):
        setattr(s, k, float(g(k)))
    s.n_max = int(g("n_max"))
    s.m_points = int(g("m_points"))
    s.precision = int(g("precision", FP64))
    s.reserved = 0
    s.B_omega = float(g("B_omega", 0.0))
    s.B_phase = float(g("B_phase", 0.0))
    return s


def _tuning(tile_m=0, chunk_n=0, graph_steps=0, vec=0, resident=0, walk=0, wide_cols=0):
    t = bte_tuning()
    t.tile_m, t.chunk_n, t.graph_steps, t.vec = int(tile_m), int(chunk_n), int(graph_steps), int(vec)
    t.resident, t.walk, t.wide_cols = int(resident), int(walk), int(wide_cols)
    return t


def version() -> str:
    return lib().bte_version().decode()


def bessel_ratio(mu: float, nmax: int) -> np.ndarray:
    r = np.zeros(nmax + 1)
    _check(lib().bte_bessel_ratio(float(mu), int(nmax), _dp(r)))
    return r


def time_grid(p):
    s = to_params(p)
    dt = ctypes.c_double()
    P, K, Kw = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().bte_time_grid(ctypes.byref(s), ctypes.byref(dt), ctypes.byref(P), ctypes.byref(K),
                               ctypes.byref(Kw)))
    return dt.value, P.value, K.value, Kw.value


def workspace_size(p, tile_m=0, chunk_n=0, vec=0, resident=0, wide_cols=0) -> int:
    s = to_params(p)
    t = _tuning(tile_m, chunk_n, 0, vec, resident, 0, wide_cols)
    n = ctypes.c_size_t()
    _check(lib().bte_workspace_size(ctypes.byref(s), ctypes.byref(t), ctypes.byref(n)))
    return n.value


def launch_shape(p, tile_m=0, chunk_n=0, vec=0) -> dict:
    """tile_m, chunk_n, pitch, grid_x, grid_y the library picks for p."""
    s = to_params(p)
    t = _tuning(tile_m, chunk_n, 0, vec)
    v = [ctypes.c_int32() for _ in range(5)]
    _check(lib().bte_launch_shape(ctypes.byref(s), ctypes.byref(t), *(ctypes.byref(x) for x in v)))
    return dict(zip(("tile_m", "chunk_n", "pitch", "grid_x", "grid_y"), (x.value for x in v)))


def observe_noalloc(p, a0_row_dev: int, b1_row_dev: int, out_dev: int, stream: int = 0) -> None:
    """Queues bte_observe_noalloc on device pointers (ints): out_dev[0] =
    drift velocity, out_dev[1] = norm of the given rows; allocates nothing."""
    s = to_params(p)
    _check(lib().bte_observe_noalloc(ctypes.byref(s), ctypes.c_void_p(a0_row_dev),
                                     ctypes.c_void_p(b1_row_dev), ctypes.c_void_p(out_dev),
                                     ctypes.c_void_p(stream or None)))


@dataclass
class Observables:
    t: float
    step: int
    v_dr: float
    norm: float
    v_dc_avg: float
    absorption: float
    norm_max_abs_err: float
    dt_eff: float
    steps_total: int
    steps_per_period: int
    window_steps: int
    status: int


class Solver:
    """One solver instance (a ``bte_handle``).

    ``stream`` is a CUDA stream handle as an integer (e.g.
    ``torch.cuda.current_stream().cuda_stream``) or 0 for a private stream.
    ``workspace`` is an optional device pointer (int) of at least
    ``workspace_size(p)`` bytes, e.g. from a PyTorch uint8 tensor, which the
    caller keeps alive while the solver exists.  ``resident=1`` keeps the
    grid in the shared memory of one thread-block cluster and advances it
    with one persistent launch per step/run call (grids that fit only);
    ``resident=2`` is the persistent mode, ``resident=3`` the on-chip mode
    over several clusters (``wide_cols`` phi_y columns per cluster, 0 =
    automatic)."""

    def __init__(self, p, stream: int = 0, tile_m: int = 0, chunk_n: int = 0,
                 graph_steps: int = 0, workspace: int = 0, workspace_bytes: int = 0,
                 vec: int = 0, resident: int = 0, walk: int = 0, wide_cols: int = 0):
        self._lib = lib()
        self.params = to_params(p)
        self._h = ctypes.c_void_p()
        t = _tuning(tile_m, chunk_n, graph_steps, vec, resident, walk, wide_cols)
        _check(self._lib.bte_create_ex(ctypes.byref(self.params), ctypes.c_void_p(stream or None),
                                       ctypes.byref(t), ctypes.c_void_p(workspace or None),
                                       int(workspace_bytes), ctypes.byref(self._h)))
        self.shape = (self.params.n_max + 1, self.params.m_points)

    def close(self):
        if self._h:
            self._lib.bte_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, nsteps: int) -> None:
        _check(self._lib.bte_step(self._h, int(nsteps)))

    def run(self) -> None:
        _check(self._lib.bte_run(self._h))

    def reset(self) -> None:
        _check(self._lib.bte_reset(self._h))

    def observables(self, check: bool = True) -> Observables:
        o = bte_obs()
        rc = self._lib.bte_observables(self._h, ctypes.byref(o))
        if check:
            _check(rc)
        return _obs(o)

    def trace(self, k0: int = 0, count: int | None = None):
        if count is None:
            count = self.observables(check=False).step + 1 - k0
        v = np.zeros(count)
        n = np.zeros(count)
        _check(self._lib.bte_trace(self._h, int(k0), int(count), _dp(v), _dp(n)))
        return v, n

    def get_state(self, grid: int):
        a = np.zeros(self.shape)
        b = np.zeros(self.shape)
        _check(self._lib.bte_get_state(self._h, int(grid), _dp(a), _dp(b)))
        return a, b

    def set_state(self, grid: int, a: np.ndarray, b: np.ndarray) -> None:
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        assert a.shape == self.shape and b.shape == self.shape
        _check(self._lib.bte_set_state(self._h, int(grid), _dp(a), _dp(b)))

    def pdf(self, grid: int = 0, nphix: int = 128) -> np.ndarray:
        """f(phi_x, phi_y) of one grid on nphix x m_points points
        (``bte_pdf``); phi_x = -pi + 2 pi i / nphix."""
        out = np.zeros((int(nphix), self.shape[1]))
        _check(self._lib.bte_pdf(self._h, int(grid), int(nphix), _dp(out)))
        return out

    def wait_probe(self, limit_ns: int) -> None:
        """Queues ``bte_wait_probe``: one bounded in-kernel wait that nothing
        completes, recorded in the error word as a solver timeout (the next
        ``observables`` call reports ``ETIMEOUT`` until ``reset``)."""
        _check(self._lib.bte_wait_probe(self._h, int(limit_ns)))

    def set_step(self, k: int, v: np.ndarray, norm: np.ndarray) -> None:
        v = np.ascontiguousarray(v, dtype=np.float64)
        norm = np.ascontiguousarray(norm, dtype=np.float64)
        assert len(v) >= k + 1 and len(norm) >= k + 1
        _check(self._lib.bte_set_step(self._h, int(k), _dp(v), _dp(norm)))


def _obs(o: bte_obs) -> Observables:
    return Observables(o.t, o.step, o.v_dr, o.norm, o.v_dc_avg, o.absorption,
                       o.norm_max_abs_err, o.dt_eff, o.steps_total, o.steps_per_period,
                       o.window_steps, o.status)


def _batch_opts(tile_m=0, chunk_n=0, vec=0, graph_steps=0, max_batch=0, max_batch_bytes=0,
                stream=0, resident=0, resident_smem=0, walk=0):
    o = bte_batch_opts()
    o.tile_m, o.chunk_n, o.vec, o.graph_steps = int(tile_m), int(chunk_n), int(vec), int(graph_steps)
    o.max_batch, o.resident, o.max_batch_bytes = int(max_batch), int(resident), int(max_batch_bytes)
    o.resident_smem, o.walk = int(resident_smem), int(walk)
    o.stream = ctypes.c_void_p(stream or None)
    return o


def batch_plan(points, **opts) -> np.ndarray:
    """Tier of every point under ``batch_run`` with the same options
    (``bte_batch_plan``): CTAs per cluster on chip, 0 when streamed."""
    pts = list(points)
    n = len(pts)
    arr = (bte_params * max(n, 1))(*[to_params(q) for q in pts])
    tier = np.zeros(max(n, 1), dtype=np.int32)
    o = _batch_opts(**opts)
    _check(lib().bte_batch_plan(arr, n, ctypes.byref(o),
                                tier.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return tier[:n]


TUNE_FIELDS = ("tile_m", "chunk_n", "vec", "graph_steps", "max_batch", "max_batch_bytes",
               "resident", "resident_smem")


def batch_tune(points, sample: int = 16, steps: int = 2000, **opts):
    """``bte_batch_tune``: (best options as a dict of batch_run keywords,
    seconds of the 12 candidates)."""
    pts = list(points)
    n = len(pts)
    arr = (bte_params * n)(*[to_params(q) for q in pts])
    base = _batch_opts(**opts)
    best = bte_batch_opts()
    secs = np.zeros(12)
    _check(lib().bte_batch_tune(arr, n, ctypes.byref(base), int(sample), int(steps),
                                ctypes.byref(best), secs.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return {k: int(getattr(best, k)) for k in TUNE_FIELDS}, secs


def batch_run(points, tile_m: int = 0, chunk_n: int = 0, vec: int = 0, graph_steps: int = 0,
              max_batch: int = 0, max_batch_bytes: int = 0, stream: int = 0,
              resident: int = 0, resident_smem: int = 0, walk: int = 0,
              check: bool = True) -> list[Observables]:
    """Full solves of many parameter points (``bte_batch_run``); returns one
    ``Observables`` per point, in order.  ``resident``: 0 on chip where a
    point fits, 1 never, 2 only.  With ``check`` a non-OK overall status
    raises; without it the per-point ``status`` fields tell."""
    pts = list(points)
    n = len(pts)
    arr = (bte_params * max(n, 1))(*[to_params(q) for q in pts])
    out = (bte_obs * max(n, 1))()
    o = _batch_opts(tile_m, chunk_n, vec, graph_steps, max_batch, max_batch_bytes, stream, resident,
                    resident_smem, walk)
    rc = lib().bte_batch_run(arr, n, out, ctypes.byref(o))
    if check:
        _check(rc)
    elif rc in (EINVAL, ENOMEM, ECUDA):
        _check(rc)
    return [_obs(out[i]) for i in range(n)]


def solve(p, **kw) -> Observables:
    """Creates a solver, runs the whole protocol and returns the observables."""
    with Solver(p, **kw) as s:
        s.run()
        return s.observables()
