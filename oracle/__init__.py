"""FP64 CPU oracle of the superlattice BTE solver (arXiv:1401.6047).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package.

``bte_oracle.cpp`` holds the arithmetic (see its header for the paper sections
each function follows and the readings of the paper it takes).  This module
only compiles it with g++ and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bte_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

# planted-mistake switches (tests only; 0 = the method)
MUT_PAPER_B_SIGN = 1
MUT_ALPHA_STENCIL = 2
MUT_SIGMA0_ONE = 4
MUT_NO_CHI = 8
MUT_STALE_SOURCE = 16
MUT_THETA_START_ONLY = 32
MUT_STENCIL_INDEX = 64
MUT_NO_B0_RESET = 128
MUT_B_STENCIL_START = 256


class _Params(ctypes.Structure):
    _fields_ = [
        ("E_dc", ctypes.c_double), ("E_omega", ctypes.c_double),
        ("omega", ctypes.c_double), ("B", ctypes.c_double),
        ("mu", ctypes.c_double), ("alpha", ctypes.c_double),
        ("phiy_min", ctypes.c_double), ("phiy_max", ctypes.c_double),
        ("dt", ctypes.c_double), ("periods", ctypes.c_double),
        ("t_max", ctypes.c_double), ("avg_window", ctypes.c_double),
        ("n_max", ctypes.c_int32), ("m_points", ctypes.c_int32),
        ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("B_omega", ctypes.c_double), ("B_phase", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (g++, OpenMP, no FMA
    contraction so that x86 and Arm hosts round identically)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        ll = ctypes.c_longlong
        llp = ctypes.POINTER(ll)
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_set_threads.restype = None
        L.oracle_time_grid.argtypes = [P, dp, llp, llp, llp]
        L.oracle_bessel_ratio.argtypes = [ctypes.c_double, ctypes.c_int, dp]
        L.oracle_equilibrium.argtypes = [P, dp]
        L.oracle_init.argtypes = [P, dp, dp, dp, dp]
        L.oracle_advance.argtypes = [P, ll, ll, dp, dp, dp, dp, dp, dp]
        L.oracle_observe.argtypes = [P, dp, dp, dp, dp]
        L.oracle_window.argtypes = [P, dp, ll, dp, dp]
        L.oracle_solve.argtypes = [P, dp, dp, dp, dp, dp, dp, dp]
        for f in ("oracle_time_grid", "oracle_bessel_ratio", "oracle_equilibrium",
                  "oracle_init", "oracle_advance", "oracle_observe", "oracle_window",
                  "oracle_solve"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(p, flags: int = 0) -> _Params:
    """Accepts any object with the solver parameter attributes (the workload
    dataclass) or a dict."""
    g = (lambda k, d=None: p.get(k, d)) if isinstance(p, dict) else (lambda k, d=None: getattr(p, k, d))
    s = _Params()
    for k in ("E_dc", "E_omega", "omega", "B", "mu", "alpha", "phiy_min", "phiy_max",
              "dt", "periods", "t_max"):
        setattr(s, k, float(g(k)))
    s.avg_window = float(g("avg_window"))
    s.n_max = int(g("n_max"))
    s.m_points = int(g("m_points"))
    s.flags = int(flags)
    s.B_omega = float(g("B_omega", 0.0))
    s.B_phase = float(g("B_phase", 0.0))
    return s


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle: {what} rejected the parameters")


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def threads() -> int:
    return int(lib().oracle_threads())


def time_grid(p):
    dt = ctypes.c_double()
    P = ctypes.c_longlong()
    K = ctypes.c_longlong()
    Kw = ctypes.c_longlong()
    s = _params(p)
    _check(lib().oracle_time_grid(ctypes.byref(s), ctypes.byref(dt), ctypes.byref(P),
                                  ctypes.byref(K), ctypes.byref(Kw)), "time_grid")
    return dt.value, P.value, K.value, Kw.value


def bessel_ratio(mu: float, nmax: int) -> np.ndarray:
    r = np.zeros(nmax + 1)
    _check(lib().oracle_bessel_ratio(float(mu), int(nmax), _ptr(r)), "bessel_ratio")
    return r


def _shape(p):
    g = (lambda k: p[k]) if isinstance(p, dict) else (lambda k: getattr(p, k))
    return (int(g("n_max")) + 1, int(g("m_points")))


def equilibrium(p, flags: int = 0) -> np.ndarray:
    a0 = np.zeros(_shape(p))
    s = _params(p, flags)
    _check(lib().oracle_equilibrium(ctypes.byref(s), _ptr(a0)), "equilibrium")
    return a0


@dataclass
class State:
    aw: np.ndarray
    bw: np.ndarray
    af: np.ndarray
    bf: np.ndarray

    def copy(self) -> "State":
        return State(self.aw.copy(), self.bw.copy(), self.af.copy(), self.bf.copy())


def init(p, flags: int = 0) -> State:
    shp = _shape(p)
    st = State(*(np.zeros(shp) for _ in range(4)))
    s = _params(p, flags)
    _check(lib().oracle_init(ctypes.byref(s), _ptr(st.aw), _ptr(st.bw), _ptr(st.af),
                             _ptr(st.bf)), "init")
    return st


def advance(p, st: State, k0: int, nsteps: int, flags: int = 0):
    """Advances ``st`` in place by ``nsteps`` steps from step ``k0``; returns
    (v, norm) arrays of the whole-grid samples after each step."""
    v = np.zeros(max(nsteps, 1))
    nr = np.zeros(max(nsteps, 1))
    s = _params(p, flags)
    _check(lib().oracle_advance(ctypes.byref(s), int(k0), int(nsteps), _ptr(st.aw),
                                _ptr(st.bw), _ptr(st.af), _ptr(st.bf), _ptr(v), _ptr(nr)),
           "advance")
    return v[:nsteps], nr[:nsteps]


def observe(p, a: np.ndarray, b: np.ndarray):
    v = ctypes.c_double()
    nr = ctypes.c_double()
    s = _params(p)
    _check(lib().oracle_observe(ctypes.byref(s), _ptr(a), _ptr(b), ctypes.byref(v),
                                ctypes.byref(nr)), "observe")
    return v.value, nr.value


def window(p, v: np.ndarray):
    """A and vbar from a whole-grid trace v[0..K]."""
    A = ctypes.c_double()
    vb = ctypes.c_double()
    v = np.ascontiguousarray(v, dtype=np.float64)
    s = _params(p)
    _check(lib().oracle_window(ctypes.byref(s), _ptr(v), len(v) - 1, ctypes.byref(A),
                               ctypes.byref(vb)), "window")
    return A.value, vb.value


@dataclass
class Result:
    A: float
    v_dc: float
    norm_err: float
    dt_eff: float
    K: int
    Kw: int
    v: np.ndarray = field(repr=False)
    norm: np.ndarray = field(repr=False)
    state: State | None = field(default=None, repr=False)


def solve(p, flags: int = 0, want_state: bool = False) -> Result:
    dt, P, K, Kw = time_grid(p)
    v = np.zeros(K + 1)
    nr = np.zeros(K + 1)
    out = np.zeros(6)
    s = _params(p, flags)
    shp = _shape(p)
    st = State(*(np.zeros(shp) for _ in range(4))) if want_state else None
    _check(lib().oracle_solve(ctypes.byref(s), _ptr(v), _ptr(nr), _ptr(out),
                              _ptr(st.aw) if st else None, _ptr(st.bw) if st else None,
                              _ptr(st.af) if st else None, _ptr(st.bf) if st else None),
           "solve")
    return Result(out[0], out[1], out[2], out[3], int(out[4]), int(out[5]), v, nr, st)
