"""Temporal blocking gives exactly the states of single steps, with either
step kernel: the row march (strip blocks of plain fluid taking both steps
in one pass, step_march2_kernel; the others two single steps through the
middle state, the first with a one-node fringe) and the tile kernel (clean
tiles in step_tile2_kernel).  Compared bitwise after odd and even step
counts, with and without CUDA-graph replay, on grids with every edge kind,
solids, no-slip rings and Dirichlet columns, and at the benchmark's full
size."""
import numpy as np
import pytest

import inputs
from inputs import BOUNCEBACK, PERIODIC, SPECULAR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


KERNELS = ["march", "tile"]


def run(case, steps, k, graph_steps=64, precision="f32", kernel="march"):
    from paper_1902_02999_gb300 import Simulation
    sim = Simulation.from_case(case, precision=precision)
    sim.set_step_kernel(kernel)
    sim.set_graph_steps(graph_steps)
    if k != 1:
        sim.set_temporal_block(k)
    sim.step(steps)
    out = sim.get_state()
    r = sim.residual()
    info = dict(sim.info)
    sim.close()
    return out, r, info


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("edges", [(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR),
                                   (PERIODIC, PERIODIC, PERIODIC, PERIODIC),
                                   (SPECULAR, SPECULAR, SPECULAR, SPECULAR),
                                   (BOUNCEBACK, SPECULAR, PERIODIC, PERIODIC)])
@pytest.mark.parametrize("steps", [1, 2, 7, 130])
@pytest.mark.parametrize("kernel", KERNELS)
def test_two_step_launches_equal_single_steps(edges, steps, kernel):
    case = inputs.random_case(517, 301, 11, edges=edges)
    a, ra, _ = run(case, steps, 1, kernel=kernel)
    b, rb, info = run(case, steps, 2, kernel=kernel)
    assert info["temporal_block"] == 2 and info["clean_tiles"] > 0
    if kernel == "march" and info["dirichlet_fused"]:
        assert info["two_step_blocks"] > 0
    print(kernel, edges, steps, "two-step strip blocks", info["two_step_blocks"])
    assert same(a, b)
    assert ra == rb


@pytest.mark.parametrize("kernel", KERNELS)
def test_dish_lake_and_channel(kernel):
    for case in (inputs.dish_lake(256, seed=3), inputs.bump_channel(1024, 512, seed=1),
                 inputs.random_case(517, 131, 22, edges=(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR), dirichlet_sn=True)):
        a, ra, _ = run(case, 301, 1, graph_steps=0, kernel=kernel)
        b, rb, info = run(case, 301, 2, graph_steps=0, kernel=kernel)
        assert info["clean_tiles"] > 0
        if kernel == "march" and info["dirichlet_fused"]:
            assert info["two_step_blocks"] > 0
        assert same(a, b), case.name
        assert ra == rb


@pytest.mark.parametrize("kernel", KERNELS)
def test_full_size_channel(kernel):
    case = inputs.bump_channel(8192, 2048, seed=0)
    a, _, _ = run(case, 21, 1, graph_steps=0, kernel=kernel)
    b, _, info = run(case, 21, 2, graph_steps=0, kernel=kernel)
    assert info["clean_tiles"] >= 0.9 * (8192 // 64) * (2048 // 16)
    if kernel == "march":
        assert info["two_step_blocks"] > 0
    assert same(a, b)


def test_rejected_for_fp64_and_bad_k():
    from paper_1902_02999_gb300 import MaclabError, Simulation
    sim = Simulation.from_case(inputs.random_case(131, 70, 2), precision="f64")
    with pytest.raises(MaclabError):
        sim.set_temporal_block(2)
    with pytest.raises(MaclabError):
        sim.set_temporal_block(3)
    sim.close()
