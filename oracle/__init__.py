"""FP64 CPU oracle of the MacLABSWE step (Zhou, arXiv:1902.02999).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The CUDA library never
imports, links or calls anything here, and nothing here touches the CUDA
library.

The arithmetic lives in ``maclab_oracle.c`` (plain C, double precision,
compiled with -O2 -ffp-contract=off); this module compiles it with gcc on
first use and marshals numpy arrays through ctypes.

Pins (tests/test_oracle_pins.py, tests/test_oracle_tidal.py) tie it to the
paper: the moment identities of Eq. feq-full, a 3x3 step worked by hand
from Eqs. feq-full and Mac.lb.6/7, lake at rest over an arbitrary bed,
exact mass conservation in closed basins, the uniform-flow fixed point, the
uniform-force closed form, the viscosity of Eq. mlb-viscosity, mirror
symmetry, the push form of Eq. lb.1 at tau = 1, and the asymptotic tidal
solution of Section 4.1 within the paper's level bound.  The distribution
form with a general relaxation time (``elab_run``) is pinned by its
reduction to MacLABSWE at tau = 1, the viscosity of Eq. viscosity and exact
mass conservation (tests/test_oracle_elab.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "maclab_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double),
        ("e", ctypes.c_double), ("g", ctypes.c_double),
        ("rho_w", ctypes.c_double), ("rho_a", ctypes.c_double), ("Cw", ctypes.c_double),
        ("wind_u", ctypes.c_double), ("wind_v", ctypes.c_double),
        ("Cb", ctypes.c_double), ("Omega", ctypes.c_double),
        ("edge", ctypes.c_int * 4),
        ("bc", ctypes.c_double * 48),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2,
    -ffp-contract=off, no architecture-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False) -> str:
    """The same source built with -fopenmp (rows of a step split over the
    host cores, the arithmetic per node unchanged): used only to time the
    oracle as the CPU baseline; the tests use the serial build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
                               "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def run_threads(case, nsteps: int, state=None, n0: int = 0):
    """oracle.run on the OpenMP build (all host cores unless OMP_NUM_THREADS
    says otherwise): for timing the CPU baseline."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            lib = ctypes.CDLL(build_omp())
            P = ctypes.POINTER
            lib.oracle_run.argtypes = [P(_Problem), P(ctypes.c_double), P(ctypes.c_uint8), P(ctypes.c_double),
                                       P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int64, ctypes.c_int64]
            lib.oracle_run.restype = ctypes.c_int
            _lib_omp = lib
    return _run_with(_lib_omp, case, nsteps, state, n0)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB lets the mutation tests load a deliberately broken
            # build of this same source; it is never set otherwise.
            lib = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
            P = ctypes.POINTER
            d, u8 = P(ctypes.c_double), P(ctypes.c_uint8)
            pp = P(_Problem)
            lib.oracle_feq.argtypes = [ctypes.c_double] * 5 + [d]
            lib.oracle_force.argtypes = [pp, ctypes.c_double, ctypes.c_double, ctypes.c_double, d]
            lib.oracle_step.argtypes = [pp, d, u8, d, d, d, d, d, d, ctypes.c_double]
            lib.oracle_run.argtypes = [pp, d, u8, d, d, d, ctypes.c_int64, ctypes.c_int64]
            lib.oracle_residual.argtypes = [pp, u8, d, d, d, d, d, d, ctypes.c_int, d]
            lib.oracle_step_push.argtypes = [pp, d, d, d, d, d, d, d]
            lib.oracle_step_newlevel.argtypes = [pp, d, u8, d, d, d, d, d, d, ctypes.c_double]
            lib.oracle_elab_step.argtypes = [pp, d, u8, ctypes.c_double, d, d]
            lib.oracle_elab_init.argtypes = [pp, d, d, d, d]
            lib.oracle_elab_moments.argtypes = [pp, d, d, d, d]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _problem(case) -> _Problem:
    p = _Problem()
    p.nx, p.ny, p.dx = case.nx, case.ny, case.dx
    p.e, p.g = case.e, case.g
    p.rho_w, p.rho_a, p.Cw = case.rho_w, case.rho_a, case.cw
    p.wind_u, p.wind_v = case.wind_u, case.wind_v
    p.Cb, p.Omega = case.cb, case.omega
    for k in range(4):
        p.edge[k] = int(case.edges[k])
    bc = np.ascontiguousarray(case.bc, dtype=np.float64).reshape(-1)
    for k in range(48):
        p.bc[k] = bc[k]
    return p


def _arr(a, case):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(case.ny, case.nx)).copy()


def feq(h: float, u: float, v: float, e: float, g: float) -> np.ndarray:
    """f^eq_0..8 of Eq. feq-full."""
    out = np.zeros(9)
    _load().oracle_feq(h, u, v, e, g, _dp(out))
    return out


def force(case, h: float, u: float, v: float) -> np.ndarray:
    """F of Eq. SWE-force at one node."""
    out = np.zeros(2)
    _load().oracle_force(ctypes.byref(_problem(case)), h, u, v, _dp(out))
    return out


def step(case, h, u, v, t_next: float):
    """One step from (h,u,v) at t_n; t_next = t_{n+1}.  Returns new arrays."""
    lib = _load()
    h, u, v = _arr(h, case), _arr(u, case), _arr(v, case)
    h1, u1, v1 = np.empty_like(h), np.empty_like(h), np.empty_like(h)
    zb = np.ascontiguousarray(case.zb, dtype=np.float64)
    mask = np.ascontiguousarray(case.mask, dtype=np.uint8)
    rc = lib.oracle_step(ctypes.byref(_problem(case)), _dp(zb),
                         mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                         _dp(h), _dp(u), _dp(v), _dp(h1), _dp(u1), _dp(v1), float(t_next))
    if rc != 0:
        raise ValueError("oracle_step: Dirichlet node off the grid edge")
    return h1, u1, v1


def run(case, nsteps: int, state=None, n0: int = 0):
    """Advance ``nsteps`` steps from ``state`` (default: the case's initial
    state) starting at step index n0.  Returns (h, u, v)."""
    return _run_with(_load(), case, nsteps, state, n0)


def _run_with(lib, case, nsteps, state, n0):
    if state is None:
        state = (case.h0, case.u0, case.v0)
    h, u, v = (_arr(a, case) for a in state)
    zb = np.ascontiguousarray(case.zb, dtype=np.float64)
    mask = np.ascontiguousarray(case.mask, dtype=np.uint8)
    rc = lib.oracle_run(ctypes.byref(_problem(case)), _dp(zb),
                        mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                        _dp(h), _dp(u), _dp(v), int(n0), int(nsteps))
    if rc != 0:
        raise ValueError("oracle_run failed (%d)" % rc)
    return h, u, v


def residual(case, s0, s1, interval: int = 1):
    """(r, mass, max|u|) of state s1 against state s0 taken ``interval``
    steps earlier: r = ||q1 - q0|| / (interval ||q1||) with q = (h, hu, hv)
    over non-solid nodes (the steady-state residual, reading R7)."""
    lib = _load()
    a = [_arr(x, case) for x in (*s0, *s1)]
    out = np.zeros(3)
    mask = np.ascontiguousarray(case.mask, dtype=np.uint8)
    lib.oracle_residual(ctypes.byref(_problem(case)),
                        mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                        *[_dp(x) for x in a], int(interval), _dp(out))
    return float(out[0]), float(out[1]), float(out[2])


def step_push(case, h, u, v):
    """Distribution (push) form of Eq. lb.1 at tau = 1, all-fluid periodic grids."""
    lib = _load()
    h, u, v = _arr(h, case), _arr(u, case), _arr(v, case)
    h1, u1, v1 = np.empty_like(h), np.empty_like(h), np.empty_like(h)
    zb = np.ascontiguousarray(case.zb, dtype=np.float64)
    rc = lib.oracle_step_push(ctypes.byref(_problem(case)), _dp(zb), _dp(h), _dp(u), _dp(v),
                              _dp(h1), _dp(u1), _dp(v1))
    if rc != 0:
        raise MemoryError("oracle_step_push")
    return h1, u1, v1


def elab_run(case, tau: float, nsteps: int, f=None):
    """eLABSWE (Eq. lb.1) with relaxation time tau: ``nsteps`` steps from the
    distributions f [9, ny, nx] (default: the equilibrium of the case's
    initial state).  Returns (h, u, v, f)."""
    lib = _load()
    prob = _problem(case)
    N = case.nx * case.ny
    if f is None:
        f = np.empty((9, case.ny, case.nx))
        h0, u0, v0 = (_arr(a, case) for a in (case.h0, case.u0, case.v0))
        lib.oracle_elab_init(ctypes.byref(prob), _dp(h0), _dp(u0), _dp(v0), _dp(f))
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    f1 = np.empty_like(f)
    zb = np.ascontiguousarray(case.zb, dtype=np.float64)
    mask = np.ascontiguousarray(case.mask, dtype=np.uint8)
    for _ in range(nsteps):
        rc = lib.oracle_elab_step(ctypes.byref(prob), _dp(zb), mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                  float(tau), _dp(f), _dp(f1))
        if rc != 0:
            raise ValueError("oracle_elab_step: only fluid and solid nodes (%d)" % rc)
        f, f1 = f1, f
    h, u, v = (np.empty((case.ny, case.nx)) for _ in range(3))
    lib.oracle_elab_moments(ctypes.byref(prob), _dp(f), _dp(h), _dp(u), _dp(v))
    assert f.size == 9 * N
    return h, u, v, f


def run_newlevel(case, nsteps: int, state=None, n0: int = 0):
    """Like run(), with hbar at the new time level (Eq. h-bar as written,
    solved node by node).  Returns (h, u, v)."""
    lib = _load()
    if state is None:
        state = (case.h0, case.u0, case.v0)
    h, u, v = (_arr(a, case) for a in state)
    h1, u1, v1 = np.empty_like(h), np.empty_like(h), np.empty_like(h)
    zb = np.ascontiguousarray(case.zb, dtype=np.float64)
    mask = np.ascontiguousarray(case.mask, dtype=np.uint8)
    for k in range(nsteps):
        rc = lib.oracle_step_newlevel(ctypes.byref(_problem(case)), _dp(zb),
                                      mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                      _dp(h), _dp(u), _dp(v), _dp(h1), _dp(u1), _dp(v1),
                                      float((n0 + k + 1) * case.dt))
        if rc != 0:
            raise ValueError("oracle_step_newlevel failed (%d)" % rc)
        h, h1 = h1, h
        u, u1 = u1, u
        v, v1 = v1, v
    return h, u, v
