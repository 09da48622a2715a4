"""The TMA-staged tile kernel (persistent blocks; interior tiles staged in
shared memory by tensor copies) against the one-block-per-tile kernel and
the warp-strip kernel (bitwise: all spell out every rounding the same way;
the tile kernels pair two nodes per FP32 instruction, the strip kernel does
not) and against the FP64 oracle (within the FP32 tolerance of the parity
tests)."""
import numpy as np
import pytest

import inputs
import oracle
from inputs import BOUNCEBACK, PERIODIC, SPECULAR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EDGES = [
    (BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR),
    (PERIODIC, PERIODIC, SPECULAR, SPECULAR),
    (SPECULAR, SPECULAR, SPECULAR, SPECULAR),
    (PERIODIC, PERIODIC, PERIODIC, PERIODIC),
    (BOUNCEBACK, BOUNCEBACK, BOUNCEBACK, BOUNCEBACK),
    (BOUNCEBACK, SPECULAR, PERIODIC, PERIODIC),
]


def sim_of(case, kernel=None, precision="f32"):
    from paper_1902_02999_gb300 import Simulation
    sim = Simulation.from_case(case, precision=precision)
    if kernel is not None:
        sim.set_step_kernel(kernel)
    return sim


def run_pair(case, steps, graph_steps=None, kernels=("tile", "tma")):
    out = []
    for kernel in kernels:
        sim = sim_of(case, kernel)
        if graph_steps is not None:
            sim.set_graph_steps(graph_steps)
        sim.step(steps)
        out.append(sim.get_state())
        assert sim.info["step_kernel"] == {"tile": 0, "strip": 1, "tma": 2}[kernel]
        sim.close()
    return out


# sizes with interior tiles (nx >= 130, ny >= 33), ragged tails and one
# tile that is all edge
@pytest.mark.parametrize("nx,ny,seed", [(131, 97, 1), (517, 301, 2), (200, 40, 3), (64, 16, 4), (1000, 35, 5)])
@pytest.mark.parametrize("edges", EDGES)
def test_tma_kernel_equals_tile_kernel(nx, ny, seed, edges):
    case = inputs.random_case(nx, ny, seed, edges=edges)
    a, b = run_pair(case, 60)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("edges", EDGES)
def test_paired_and_scalar_kernels_agree_bitwise(edges):
    """Paired FP32 arithmetic (tile kernels) against one node per
    instruction (strip kernel), specular ghosts and ragged tails included."""
    case = inputs.random_case(517, 131, 40, edges=edges)
    runs = run_pair(case, 80, kernels=("strip", "tile", "tma"))
    for other in runs[1:]:
        for x, y in zip(runs[0], other):
            assert np.array_equal(x, y)


def test_tma_kernel_force_variants_equal_tile_kernel():
    """Every compile-time force variant: wind, friction, Coriolis on / off."""
    for fm in range(8):
        case = inputs.random_case(300, 70, 30 + fm)
        if not fm & 1:
            case.wind_u = case.wind_v = 0.0
        if not fm & 2:
            case.cb = 0.0
        if not fm & 4:
            case.omega = 0.0
        runs = run_pair(case, 40, kernels=("strip", "tile", "tma"))
        for other in runs[1:]:
            for x, y in zip(runs[0], other):
                assert np.array_equal(x, y), fm


def test_tma_kernel_with_graph_replay():
    case = inputs.random_case(517, 301, 7)
    a, b = run_pair(case, 130, graph_steps=64)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_tma_kernel_against_oracle():
    case = inputs.random_case(517, 131, 11)
    want = oracle.run(case, 300)
    sim = sim_of(case, "tma")
    sim.step(300)
    got = sim.get_state()
    live = case.mask != inputs.SOLID
    eh = np.abs(got[0] - want[0])[live].max() / np.abs(want[0][live]).max()
    scale = np.hypot(want[1], want[2])[live].max()
    eu = max(np.abs(got[1] - want[1])[live].max(), np.abs(got[2] - want[2])[live].max()) / scale
    assert eh <= 2e-5 and eu <= 1e-4, (eh, eu)
    r, mass, umax = sim.residual()
    assert np.isfinite(r) and r > 0


def test_tma_kernel_full_size_channel():
    """8192 x 2048 channel: 20 steps of each kernel, bitwise equal."""
    case = inputs.bump_channel(8192, 2048, seed=0)
    a, b = run_pair(case, 20)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_tma_kernel_needs_fp32():
    from paper_1902_02999_gb300 import MaclabError
    case = inputs.random_case(131, 40, 1)
    sim = sim_of(case, precision="f64")
    with pytest.raises(MaclabError):
        sim.set_step_kernel("tma")
    sim.close()
