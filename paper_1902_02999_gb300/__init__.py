"""GB300-native MacLABSWE streaming step (Zhou, arXiv:1902.02999).

Python binding of the C ABI in include/maclab.h.  This module only
marshals arguments: every step of the method runs in the library's own
sm_103a CUDA kernels (csrc/).  PyTorch supplies device memory (through the
caching allocator) and the CUDA stream; there is no CPU fallback, and
creating a Simulation fails loudly when the CUDA library or a GPU is
missing.

    sim = Simulation(nx, ny, dx, zb, mask, nu=..., precision="f32", ...)
    sim.step(1000)
    h, u, v = sim.get_state()
    r, mass, umax = sim.residual()
"""
from __future__ import annotations

import atexit
import ctypes
import weakref
from typing import Sequence

import numpy as np

from . import _abi
from . import build as _build_module

SOLID, FLUID, NOSLIP, DIR_H, DIR_Q, DIR_HU = 0, 1, 2, 3, 4, 5
BOUNCEBACK, SPECULAR, PERIODIC = 0, 1, 2
F32, F64 = 0, 1

__all__ = ["Simulation", "Batch", "MaclabError", "build_library", "lib", "measure_fp64"]


class MaclabError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("maclab error %d: %s" % (code, msg))
        self.code = code


def build_library(force: bool = False) -> str:
    """Compile csrc/ into _build/libmaclab.so for sm_103a; returns its path."""
    return _build_module.build(force=force)


def lib() -> ctypes.CDLL:
    """The loaded C library (built on first use)."""
    return _abi.load()


def measure_fp64() -> float:
    """Measured FP64 fused multiply-add rate of the current device, TFLOP/s."""
    out = ctypes.c_double()
    L = lib()
    rc = L.maclab_measure_fp64(ctypes.byref(out))
    if rc != 0:
        raise MaclabError(rc, L.maclab_last_error(None).decode())
    return out.value


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n: int) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


class _TorchAllocator:
    """maclab_allocator backed by torch's CUDA caching allocator."""

    def __init__(self, device: int, stream: int):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream

        def _alloc(nbytes, _ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                              self.stream or None))
            except Exception:  # noqa: BLE001 -- reported as MACLAB_E_NOMEM
                return None

        def _release(ptr, _ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self._alloc = _abi.ALLOC_FN(_alloc)
        self._release = _abi.RELEASE_FN(_release)
        self.struct = _abi.Allocator(self._alloc, self._release, None)


_live = weakref.WeakSet()


@atexit.register
def _close_all():
    # release device buffers while torch's allocator is still alive
    for sim in list(_live):
        try:
            sim.close()
        except Exception:  # noqa: BLE001
            pass


class Simulation:
    """One MacLABSWE problem resident on the current CUDA device.

    Arrays are [ny][nx] row-major (x fastest).  ``precision`` is "f32"
    (state stored as float perturbation eta = h - (h_ref - z_b)) or "f64".
    ``edges`` gives the W, E, S, N edge kinds; ``bc`` is an array [4][3][4]
    of (mean, amp, omega, phase) for h, q_x, q_y per edge.
    """

    def __init__(self, nx: int, ny: int, dx: float, zb, mask, *, nu: float = 0.0,
                 e: float = 0.0, precision: str = "f32", g: float = 9.81,
                 rho_w: float = 1000.0, rho_a: float = 1.293, cw: float = 0.0026,
                 wind: Sequence[float] = (0.0, 0.0), cb: float = 0.0, omega: float = 0.0,
                 h_ref: float = 0.0, edges: Sequence[int] = (0, 0, 0, 0), bc=None,
                 h0=None, u0=None, v0=None, stream=None, torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("maclab needs a CUDA GPU; no CPU fallback exists")
        self._lib = lib()
        self.nx, self.ny = int(nx), int(ny)
        N = self.nx * self.ny
        self.device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream_obj = stream
        sptr = int(getattr(stream, "cuda_stream", stream) or 0)
        grid = _abi.Grid(self.nx, self.ny, float(dx))
        prec = {"f32": F32, "f64": F64, F32: F32, F64: F64}[precision]
        params = _abi.Params(prec, float(nu), float(e), float(g), float(rho_w), float(rho_a),
                             float(cw), float(wind[0]), float(wind[1]), float(cb), float(omega),
                             float(h_ref))
        b = _abi.BC()
        for k in range(4):
            b.edge[k] = int(edges[k])
        if bc is not None:
            bcv = np.asarray(bc, dtype=np.float64).reshape(4, 3, 4)
            for k in range(4):
                b.h[k] = _abi.Wave(*bcv[k, 0])
                b.qx[k] = _abi.Wave(*bcv[k, 1])
                b.qy[k] = _abi.Wave(*bcv[k, 2])
        zb = _f64(zb, N)
        mask = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
        if mask.size != N:
            raise ValueError("mask size")
        state = [None, None, None]
        if h0 is not None:
            state = [_f64(h0, N), _f64(u0, N), _f64(v0, N)]
        self._alloc = _TorchAllocator(self.device, sptr) if torch_allocator else None
        handle = ctypes.c_void_p()
        rc = self._lib.maclab_create(
            ctypes.byref(grid), ctypes.byref(params), ctypes.byref(b), _dptr(zb),
            mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
            *[(_dptr(a) if a is not None else None) for a in state],
            ctypes.byref(self._alloc.struct) if self._alloc else None, ctypes.c_void_p(sptr),
            ctypes.byref(handle))
        if rc != 0:
            raise MaclabError(rc, self._lib.maclab_last_error(None).decode())
        self._h = handle
        _live.add(self)
        info = _abi.Info()
        self._check(self._lib.maclab_get_info(self._h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _abi.Info._fields_}
        self.precision = "f32" if prec == F32 else "f64"

    # -- construction from an ``inputs.Case``-like object ---------------------
    @classmethod
    def from_case(cls, case, precision: str = "f32", initial: bool = True, **kw):
        st = dict(h0=case.h0, u0=case.u0, v0=case.v0) if initial else {}
        return cls(case.nx, case.ny, case.dx, case.zb, case.mask, nu=case.nu,
                   precision=precision, g=case.g, rho_w=case.rho_w, rho_a=case.rho_a,
                   cw=case.cw, wind=(case.wind_u, case.wind_v), cb=case.cb, omega=case.omega,
                   h_ref=case.h_ref, edges=case.edges, bc=case.bc, **st, **kw)

    def _check(self, rc: int):
        if rc != 0:
            raise MaclabError(rc, self._lib.maclab_last_error(self._h).decode())

    @property
    def handle(self):
        return self._h

    def step(self, n: int = 1) -> None:
        self._check(self._lib.maclab_step(self._h, int(n)))

    def get_state(self, out=None):
        """(h, u, v) as [ny][nx] double arrays; ``out`` may supply three
        contiguous float64 arrays of nx*ny values to fill (e.g. pinned)."""
        N = self.nx * self.ny
        if out is not None:
            h, u, v = out
            for a in out:
                if a.dtype != np.float64 or a.size != N or not a.flags.c_contiguous:
                    raise ValueError("out arrays must be contiguous float64 of nx*ny values")
        else:
            h, u, v = np.empty(N), np.empty(N), np.empty(N)
        self._check(self._lib.maclab_get_state(self._h, _dptr(h), _dptr(u), _dptr(v)))
        shp = (self.ny, self.nx)
        return h.reshape(shp), u.reshape(shp), v.reshape(shp)

    def set_state(self, h, u, v) -> None:
        N = self.nx * self.ny
        h, u, v = _f64(h, N), _f64(u, N), _f64(v, N)
        self._check(self._lib.maclab_set_state(self._h, _dptr(h), _dptr(u), _dptr(v)))

    def residual(self):
        """(r, mass, max|u|) of the last step; raises on a non-finite state."""
        out = np.zeros(4)
        self._check(self._lib.maclab_residual(self._h, _dptr(out)))
        return float(out[0]), float(out[1]), float(out[2])

    def mark(self) -> None:
        """Keep a copy of the current state for residual_since_mark."""
        self._check(self._lib.maclab_mark(self._h))

    def residual_since_mark(self):
        """(r, mass, max|u|): r = ||q - q_mark|| / (m ||q||) over the m steps
        since the mark, q = (h, hu, hv)."""
        out = np.zeros(4)
        self._check(self._lib.maclab_residual_since_mark(self._h, _dptr(out)))
        return float(out[0]), float(out[1]), float(out[2])

    def run_to_steady(self, tol: float = 1e-8, max_steps: int = 10 ** 7, check_every: int = 100):
        """Steps until the residual over each check interval is <= tol.
        Returns (converged, steps_done, last_residual)."""
        done, r = ctypes.c_int64(), ctypes.c_double()
        rc = self._lib.maclab_run_to_steady(self._h, float(tol), int(max_steps), int(check_every),
                                           ctypes.byref(done), ctypes.byref(r))
        if rc not in (0, -5):
            self._check(rc)
        return rc == 0, int(done.value), float(r.value)

    def set_tile_rows(self, rows: int) -> None:
        self._check(self._lib.maclab_set_tile_rows(self._h, int(rows)))
        self.info["tile_rows"] = min(int(rows), self.ny)

    def set_launch(self, rows: int, blocks: int = 0) -> None:
        """Rows per warp strip and a cap on step-kernel blocks (0 = none)."""
        self._check(self._lib.maclab_set_launch(self._h, int(rows), int(blocks)))
        self.info["tile_rows"] = min(int(rows), self.ny)
        self.info["grid_blocks"] = int(blocks)

    KERNELS = {"tile": 0, "strip": 1, "tma": 2, "march": 3}

    def set_step_kernel(self, kernel) -> None:
        """Step kernel: "tile", "strip", "tma" (FP32 only) or "march", or its code."""
        code = self.KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        self._check(self._lib.maclab_set_step_kernel(self._h, code))
        self.info["step_kernel"] = code

    def set_hbar_level(self, level: int) -> None:
        """hbar of the bed term at the old (0) or the new (1) time level."""
        self._check(self._lib.maclab_set_hbar_level(self._h, int(level)))
        self.info["hbar_level"] = int(level)

    def set_relaxation(self, tau: float) -> None:
        """Relaxation time of Eq. lb.1: 1 = MacLABSWE, otherwise the
        distribution form (fluid and solid nodes only)."""
        self._check(self._lib.maclab_set_relaxation(self._h, float(tau)))
        info = _abi.Info()
        self._check(self._lib.maclab_get_info(self._h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _abi.Info._fields_}

    def set_temporal_block(self, k: int) -> None:
        """Steps per launch of clean interior tiles: 1, or 2 (FP32)."""
        self._check(self._lib.maclab_set_temporal_block(self._h, int(k)))
        info = _abi.Info()
        self._check(self._lib.maclab_get_info(self._h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _abi.Info._fields_}

    def autotune(self, trial_steps: int = 20) -> int:
        """Pick the fastest step-kernel launch shape for this grid (0 = tile
        kernel, 1..4 = strip kernel with 8/16/32/64 rows, 5 = TMA-staged tile
        kernel, 6 = tile kernel with two steps per launch on clean tiles);
        state unchanged."""
        c = ctypes.c_int()
        self._check(self._lib.maclab_autotune(self._h, int(trial_steps), ctypes.byref(c)))
        info = _abi.Info()
        self._check(self._lib.maclab_get_info(self._h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _abi.Info._fields_}
        return int(c.value)

    def set_graph_steps(self, steps: int) -> None:
        """Steps per CUDA-graph replay (even, 0 = off)."""
        self._check(self._lib.maclab_set_graph_steps(self._h, int(steps)))

    def set_profiling(self, on: bool) -> None:
        self._check(self._lib.maclab_set_profiling(self._h, 1 if on else 0))

    def get_profile(self):
        """(total step-kernel milliseconds, launches) recorded since profiling was enabled."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._check(self._lib.maclab_get_profile(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return float(ms.value), int(n.value)

    def time(self):
        t, n = ctypes.c_double(), ctypes.c_int64()
        self._check(self._lib.maclab_time(self._h, ctypes.byref(t), ctypes.byref(n)))
        return float(t.value), int(n.value)

    def device_state(self):
        """Zero-copy torch views (ny, nx) of the current device state (eta, u, v)."""
        import torch
        ptrs = [ctypes.c_void_p() for _ in range(3)]
        self._check(self._lib.maclab_device_state(self._h, *[ctypes.byref(p) for p in ptrs]))
        pitch = self.info["pitch"]
        typestr = "<f4" if self.precision == "f32" else "<f8"

        class _View:
            def __init__(self, ptr):
                self.__cuda_array_interface__ = {
                    "shape": (self.ny_, pitch), "typestr": typestr, "data": (ptr, False),
                    "version": 3, "strides": None}
        out = []
        for p in ptrs:
            _View.ny_ = self.ny
            out.append(torch.as_tensor(_View(p.value), device="cuda")[:, :self.nx])
        return tuple(out)

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.maclab_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many independent grids advanced together (maclab_batch_* of the C ABI).

    ``cases`` are objects with the attributes of ``Simulation.from_case``;
    every instance must have time-independent boundary data.  Each instance
    gets exactly the values a separate Simulation would give.
    """

    def __init__(self, cases, precision: str = "f32", initial: bool = True, stream=None,
                 torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("maclab needs a CUDA GPU; no CPU fallback exists")
        self._lib = lib()
        cases = list(cases)
        n = len(cases)
        self.count = n
        self.shapes = [(c.ny, c.nx) for c in cases]
        prec = {"f32": F32, "f64": F64}[precision]
        self.precision = precision
        grids = (_abi.Grid * n)()
        params = (_abi.Params * n)()
        bcs = (_abi.BC * n)()
        keep = []
        zbp = (ctypes.POINTER(ctypes.c_double) * n)()
        mkp = (ctypes.POINTER(ctypes.c_uint8) * n)()
        hp = (ctypes.POINTER(ctypes.c_double) * n)()
        up = (ctypes.POINTER(ctypes.c_double) * n)()
        vp = (ctypes.POINTER(ctypes.c_double) * n)()
        for i, c in enumerate(cases):
            N = c.nx * c.ny
            grids[i] = _abi.Grid(c.nx, c.ny, float(c.dx))
            params[i] = _abi.Params(prec, float(c.nu), 0.0, float(c.g), float(c.rho_w), float(c.rho_a),
                                    float(c.cw), float(c.wind_u), float(c.wind_v), float(c.cb),
                                    float(c.omega), float(c.h_ref))
            bcv = np.asarray(c.bc, dtype=np.float64).reshape(4, 3, 4)
            for k in range(4):
                bcs[i].edge[k] = int(c.edges[k])
                bcs[i].h[k] = _abi.Wave(*bcv[k, 0])
                bcs[i].qx[k] = _abi.Wave(*bcv[k, 1])
                bcs[i].qy[k] = _abi.Wave(*bcv[k, 2])
            zb = _f64(c.zb, N)
            mk = np.ascontiguousarray(np.asarray(c.mask, dtype=np.uint8).reshape(-1))
            keep += [zb, mk]
            zbp[i] = _dptr(zb)
            mkp[i] = mk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
            if initial:
                h, u, v = _f64(c.h0, N), _f64(c.u0, N), _f64(c.v0, N)
                keep += [h, u, v]
                hp[i], up[i], vp[i] = _dptr(h), _dptr(u), _dptr(v)
        self.device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream()
        sptr = int(getattr(stream, "cuda_stream", stream) or 0)
        self._alloc = _TorchAllocator(self.device, sptr) if torch_allocator else None
        handle = ctypes.c_void_p()
        rc = self._lib.maclab_batch_create(
            n, grids, params, bcs, zbp, mkp, hp if initial else None, up if initial else None,
            vp if initial else None, ctypes.byref(self._alloc.struct) if self._alloc else None,
            ctypes.c_void_p(sptr), ctypes.byref(handle))
        if rc != 0:
            raise MaclabError(rc, self._lib.maclab_batch_last_error(None).decode())
        self._h = handle
        _live.add(self)

    def _check(self, rc):
        if rc != 0:
            raise MaclabError(rc, self._lib.maclab_batch_last_error(self._h).decode())

    def step(self, n: int = 1) -> None:
        self._check(self._lib.maclab_batch_step(self._h, int(n)))

    def set_graph_steps(self, steps: int) -> None:
        self._check(self._lib.maclab_batch_set_graph_steps(self._h, int(steps)))

    def set_persistent(self, mode: int) -> None:
        """1: steps in persistent cooperative launches (grid barrier between
        steps), 0: one launch per step, replayed from a CUDA graph (the
        default)."""
        self._check(self._lib.maclab_batch_set_persistent(self._h, int(mode)))

    def set_barrier_test(self, extra: int, polls: int) -> None:
        """Failure-detection test hook of the persistent grid barrier: expect
        `extra` arrivals beyond the grid and give up after `polls` polls."""
        self._check(self._lib.maclab_batch_set_barrier_test(self._h, int(extra), int(polls)))

    def mark(self) -> None:
        """Keep a copy of every instance's state for residual_since_mark."""
        self._check(self._lib.maclab_batch_mark(self._h))

    def residual_since_mark(self) -> np.ndarray:
        """[count, 4]: residual over the steps since the mark (per step),
        mass, max|u|, non-finite count per instance."""
        out = np.zeros(4 * self.count)
        self._check(self._lib.maclab_batch_residual_since_mark(self._h, _dptr(out)))
        return out.reshape(self.count, 4)

    def residual(self) -> np.ndarray:
        """[count, 4]: residual, mass, max|u|, non-finite count per instance."""
        out = np.zeros(4 * self.count)
        self._check(self._lib.maclab_batch_residual(self._h, _dptr(out)))
        return out.reshape(self.count, 4)

    def set_active(self, flags) -> None:
        f = np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
        self._check(self._lib.maclab_batch_set_active(self._h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))

    def run_to_steady(self, tol: float = 1e-8, max_steps: int = 10 ** 7, check_every: int = 1000):
        """Returns (steps[count], residual[count], seconds[count]) -- steps is -1 for
        an instance that did not converge within max_steps."""
        steps = np.zeros(self.count, dtype=np.int64)
        r = np.zeros(self.count)
        sec = np.full(self.count, np.nan)
        rc = self._lib.maclab_batch_run_to_steady(
            self._h, float(tol), int(max_steps), int(check_every),
            steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(r), _dptr(sec))
        if rc not in (0, -5):
            self._check(rc)
        return steps, r, sec

    def get_state(self, i: int):
        ny, nx = self.shapes[i]
        h, u, v = np.empty(nx * ny), np.empty(nx * ny), np.empty(nx * ny)
        self._check(self._lib.maclab_batch_get_state(self._h, int(i), _dptr(h), _dptr(u), _dptr(v)))
        return h.reshape(ny, nx), u.reshape(ny, nx), v.reshape(ny, nx)

    def set_state(self, i: int, h, u, v) -> None:
        ny, nx = self.shapes[i]
        N = nx * ny
        h, u, v = _f64(h, N), _f64(u, N), _f64(v, N)
        self._check(self._lib.maclab_batch_set_state(self._h, int(i), _dptr(h), _dptr(u), _dptr(v)))

    def device_state(self, i: int):
        """Device pointers (eta, u, v) of instance i's current state and the
        row pitch (elements); valid until the next step or set_state."""
        ptrs = [ctypes.c_void_p() for _ in range(3)]
        pitch = ctypes.c_int()
        self._check(self._lib.maclab_batch_device_state(self._h, int(i), *[ctypes.byref(p) for p in ptrs],
                                                        ctypes.byref(pitch)))
        return ptrs[0].value, ptrs[1].value, ptrs[2].value, pitch.value

    def info(self):
        c, nodes, tiles, steps = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.maclab_batch_info(self._h, ctypes.byref(c), ctypes.byref(nodes),
                                                ctypes.byref(tiles), ctypes.byref(steps)))
        return {"count": c.value, "nodes": nodes.value, "tiles": tiles.value, "steps": steps.value}

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.maclab_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
