"""maclab_residual_noalloc: the residual for callers that cannot allocate
device memory (a runtime that owns every device buffer, or a loop that must
not allocate), computed with the library's static scratch array instead of
memory it allocates.  It must give what maclab_residual gives on the same
two states, call after call.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def pitched(view, pitch, dtype):
    """A [ny][pitch] device copy of a [ny][nx] view."""
    ny, nx = view.shape
    out = torch.zeros((ny, pitch), dtype=dtype, device="cuda")
    out[:, :nx] = view
    return out


# one reduction block (131 x 70); many blocks (2048 x 1500); exactly the
# node limit, the most blocks the scratch holds (8192 x 2048, the benchmark
# channel)
GRIDS = {"one_block": lambda: inputs.random_case(131, 70, 3),
         "many_blocks": lambda: inputs.bump_channel(2048, 1500, seed=1),
         "at_limit": lambda: inputs.bump_channel(8192, 2048, seed=0)}


@pytest.mark.parametrize("grid", sorted(GRIDS))
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_noalloc_residual_matches_handle_residual(precision, grid):
    from paper_1902_02999_gb300 import Simulation, _abi
    lib = _abi.load()
    case = GRIDS[grid]()
    sim = Simulation.from_case(case, precision=precision)
    nx, ny, pitch = case.nx, case.ny, sim.info["pitch"]
    dt = torch.float32 if precision == "f32" else torch.float64
    # still-water depth and node types in the library's [ny][pitch] layout
    D = np.zeros((ny, pitch))
    D[:, :nx] = case.h_ref - case.zb
    Dd = torch.tensor(D, device="cuda").to(dt)
    T = np.zeros((ny, pitch), dtype=np.uint8)
    T[:, :nx] = case.mask
    Td = torch.tensor(T, device="cuda")
    sum_D = float(np.sum((case.h_ref - case.zb)[case.mask != inputs.SOLID]))
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                       # two calls in a row
        sim.step(4)
        prev = [pitched(v, pitch, dt) for v in sim.device_state()]
        sim.step(1)
        cur = sim.device_state()                # views into [ny][pitch] storage
        r_ref, m_ref, u_ref = sim.residual()    # the existing entry point
        torch.cuda.synchronize()
        out = (ctypes.c_double * 4)()
        rc = lib.maclab_residual_noalloc(
            0 if precision == "f32" else 1, nx, ny, pitch,
            *[ctypes.c_void_p(t.data_ptr()) for t in prev],
            *[ctypes.c_void_p(t.data_ptr()) for t in cur],
            ctypes.c_void_p(Dd.data_ptr()),
            ctypes.cast(ctypes.c_void_p(Td.data_ptr()), ctypes.POINTER(ctypes.c_uint8)),
            sum_D, ctypes.c_void_p(stream), out)
        assert rc == 0, lib.maclab_last_error(None)
        assert r_ref > 0
        assert abs(out[0] - r_ref) <= 1e-12 * r_ref, (call, out[0], r_ref)
        assert abs(out[1] - m_ref) <= 1e-12 * m_ref, (call, out[1], m_ref)
        assert abs(out[2] - u_ref) <= 1e-12 * u_ref, (call, out[2], u_ref)
        assert out[3] == 0.0
    sim.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1902_02999_gb300 import _abi
    lib = _abi.load()
    out = (ctypes.c_double * 4)()
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    rc = lib.maclab_residual_noalloc(0, 8192, 2049, 8192, *([dummy] * 7),
                                     ctypes.cast(dummy, ctypes.POINTER(ctypes.c_uint8)),
                                     0.0, None, out)
    assert rc == -1
    assert b"16777216" in lib.maclab_last_error(None)
