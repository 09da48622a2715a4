"""The row-march step kernel (one warp per 64-column strip block walking
down its rows, neighbour columns by warp shuffles) against the tile kernel
(bitwise: both finish every node with the same update_tail arithmetic and
derive sources with the same paired operations) and against the FP64
oracle (FP64 to 1e-12, FP32 to 2e-5 on h and 1e-4 on u, v)."""
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


def run(case, steps, kernel, precision="f32", graph_steps=None):
    from paper_1902_02999_gb300 import Simulation
    sim = Simulation.from_case(case, precision=precision)
    sim.set_step_kernel(kernel)
    if graph_steps is not None:
        sim.set_graph_steps(graph_steps)
    sim.step(steps)
    out = sim.get_state()
    assert sim.info["step_kernel"] == {"tile": 0, "strip": 1, "tma": 2, "march": 3}[kernel]
    sim.close()
    return out


def equal(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# strip blocks inside the grid and on every edge, ragged widths (62-column
# strips), grids narrower than one strip and one row high
@pytest.mark.parametrize("nx,ny,seed", [(131, 97, 1), (517, 301, 2), (200, 40, 3), (64, 16, 4), (1000, 35, 5),
                                        (61, 9, 6), (63, 70, 7), (125, 3, 8)])
@pytest.mark.parametrize("edges", EDGES)
def test_march_equals_tile(nx, ny, seed, edges):
    case = inputs.random_case(nx, ny, seed, edges=edges)
    equal(run(case, 60, "march"), run(case, 60, "tile"))


@pytest.mark.parametrize("edges", EDGES[:3])
def test_march_equals_tile_f64(edges):
    case = inputs.random_case(517, 131, 40, edges=edges)
    equal(run(case, 50, "march", "f64"), run(case, 50, "tile", "f64"))


def test_march_force_variants():
    """Every compile-time force variant: wind, friction, Coriolis on / off."""
    for fm in range(8):
        case = inputs.random_case(300, 70, 30 + fm)
        if not fm & 1:
            case.wind_u = case.wind_v = 0.0
        if not fm & 2:
            case.cb = 0.0
        if not fm & 4:
            case.omega = 0.0
        equal(run(case, 40, "march"), run(case, 40, "tile"))


def test_march_lake_and_graph_replay():
    """A dish lake (no-slip ring, solid outside: nodes with bounce-back links
    done by their strip block) with graph replay."""
    case = inputs.dish_lake(256, seed=3)
    equal(run(case, 130, "march", graph_steps=64), run(case, 130, "tile"))


@pytest.mark.parametrize("precision,tol_h,tol_u", [("f64", 1e-12, 1e-12), ("f32", 2e-5, 1e-4)])
def test_march_against_oracle(precision, tol_h, tol_u):
    case = inputs.random_case(517, 131, 11)
    want = oracle.run(case, 300)
    got = run(case, 300, "march", precision)
    live = case.mask != inputs.SOLID
    eh = np.abs(got[0] - want[0])[live].max() / np.abs(want[0][live]).max()
    scale = np.hypot(want[1], want[2])[live].max()
    eu = max(np.abs(got[1] - want[1])[live].max(), np.abs(got[2] - want[2])[live].max()) / scale
    print("march %s vs oracle: h %.3g, u/v %.3g" % (precision, eh, eu))
    if precision == "f64":
        # FP64: the momentum sum carries rounding of size g h^2 / (6 e) per
        # term (see test_parity_gpu); both scales are printed above
        scale64 = max(scale, case.g * np.abs(want[0][live]).max() / case.e)
        eu = eu * scale / scale64
    assert eh <= tol_h and eu <= tol_u, (eh, eu)


def test_march_full_size_channel():
    """8192 x 2048 channel: 20 steps of each kernel, bitwise equal."""
    case = inputs.bump_channel(8192, 2048, seed=0)
    equal(run(case, 20, "march"), run(case, 20, "tile"))
