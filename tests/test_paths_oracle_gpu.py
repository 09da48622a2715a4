"""The batched paths (one launch per step, and persistent cooperative
launches) and the two-step temporal blocking path against the FP64 oracle,
element by element at the parity tolerances (FP64 <= 1e-12; FP32 <= 2e-5
on h, <= 1e-4 on u, v): not only against the single-grid kernels, so that a
mistake shared by the kernels would still show."""
import numpy as np
import pytest

import inputs
import oracle
from inputs import BOUNCEBACK, PERIODIC, SPECULAR

from test_parity_gpu import compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def steady(case):
    """The case with its Dirichlet values held at their means (a batch
    takes no time-dependent boundary values)."""
    c = case.copy()
    c.bc[:, :, 1] = 0.0
    return c


def uneven_instances():
    """Nine uneven grids: every node kind (solid, fluid, no-slip, DIR_H,
    DIR_Q, DIR_HU), every edge kind, Dirichlet nodes on all four edges."""
    hump = inputs.paper_hump(41)
    hump.nu = 75.0
    return [
        steady(inputs.random_case(70, 40, 3, edges=(BOUNCEBACK,) * 4)),
        inputs.random_case(33, 65, 4, edges=(PERIODIC, PERIODIC, SPECULAR, SPECULAR), dirichlet=False),
        inputs.dish_lake(48, seed=1),
        inputs.bump_channel(130, 40, seed=2),
        steady(inputs.random_case(97, 51, 11, edges=(SPECULAR,) * 4, dirichlet_sn=True)),
        inputs.random_case(64, 64, 12, edges=(PERIODIC,) * 4),
        steady(inputs.random_case(150, 36, 13, edges=(BOUNCEBACK, SPECULAR, PERIODIC, PERIODIC))),
        steady(inputs.random_case(45, 90, 14, edges=(PERIODIC, PERIODIC, BOUNCEBACK, BOUNCEBACK),
                                  dirichlet_sn=True)),
        hump,
    ]


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_against_oracle(precision, persistent):
    from paper_1902_02999_gb300 import Batch
    cases = uneven_instances()
    kinds = set()
    for c in cases:
        kinds |= set(np.unique(c.mask).tolist())
    assert kinds == {0, 1, 2, 3, 4, 5}
    batch = Batch(cases, precision=precision)
    batch.set_persistent(persistent)
    batch.step(300)
    for i, c in enumerate(cases):
        compare(c, batch.get_state(i), oracle.run(c, 300), precision,
                ("batch", "persistent" if persistent else "per-step", c.name))


@pytest.mark.parametrize("case_fn", [
    lambda: inputs.random_case(517, 131, 22, edges=(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR),
                               dirichlet_sn=True),
    lambda: inputs.bump_channel(1030, 130, seed=5),
], ids=["random_517x131_dirichlet_all_edges", "channel_1030x130"])
def test_two_step_path_against_oracle(case_fn):
    """k = 2 (clean tiles two steps per launch, the rest in two single
    steps, time-dependent Dirichlet values at each step's own time),
    1000 steps, FP32 against the FP64 oracle."""
    from paper_1902_02999_gb300 import Simulation
    case = case_fn()
    sim = Simulation.from_case(case, precision="f32")
    sim.set_temporal_block(2)
    assert sim.info["clean_tiles"] > 0
    sim.step(1000)
    compare(case, sim.get_state(), oracle.run(case, 1000), "f32", ("k=2", case.name))
