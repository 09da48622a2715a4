"""Batches: every instance of a batch gets exactly (bitwise) what its own
handle gives, including under graph replay and when instances are switched
off; run-to-steady per instance matches the single-grid path."""
import numpy as np
import pytest

import inputs
from inputs import BOUNCEBACK, PERIODIC, SPECULAR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def mixed_cases():
    hump = inputs.paper_hump(41)
    hump.nu = 75.0
    return [
        inputs.random_case(70, 40, 3, edges=(BOUNCEBACK,) * 4, dirichlet=False),
        inputs.random_case(33, 65, 4, edges=(PERIODIC, PERIODIC, SPECULAR, SPECULAR), dirichlet=False),
        inputs.dish_lake(48, seed=1),
        inputs.bump_channel(130, 40, seed=2),
        hump,
        inputs.random_case(9, 7, 5, edges=(SPECULAR,) * 4, solids=False, dirichlet=False),
    ]


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_batch_equals_separate_handles(precision):
    from paper_1902_02999_gb300 import Batch, Simulation
    cases = mixed_cases()
    batch = Batch(cases, precision=precision)
    batch.set_graph_steps(16)
    batch.step(37)                       # graph blocks plus single launches
    res = batch.residual()
    for i, c in enumerate(cases):
        sim = Simulation.from_case(c, precision=precision)
        sim.step(37)
        want = sim.get_state()
        got = batch.get_state(i)
        for a, b in zip(got, want):
            assert np.array_equal(a, b), (i, c.name)
        r, m, u = sim.residual()
        # same terms, summed in another order (per tile, then per instance)
        assert abs(res[i, 0] - r) <= 1e-12 * r and abs(res[i, 1] - m) <= 1e-12 * m
        assert res[i, 2] == u
        sim.close()


def test_inactive_instances_stay_put():
    from paper_1902_02999_gb300 import Batch
    cases = mixed_cases()[:3]
    batch = Batch(cases, precision="f32")
    batch.step(5)
    frozen = batch.get_state(1)
    batch.set_active([1, 0, 1])
    batch.step(7)                        # odd: the buffer parity changes
    for a, b in zip(batch.get_state(1), frozen):
        assert np.array_equal(a, b)
    batch.set_active([1, 1, 1])
    batch.step(2)
    assert not np.array_equal(batch.get_state(1)[0], frozen[0])


def test_batch_run_to_steady_matches_single():
    from paper_1902_02999_gb300 import Batch, Simulation
    cases = [inputs.dish_lake(n, seed=s) for n, s in ((40, 1), (56, 2), (64, 3))]
    batch = Batch(cases, precision="f64")
    steps, r, sec = batch.run_to_steady(tol=1e-9, max_steps=400000, check_every=500)
    assert (steps > 0).all() and (r <= 1e-9).all() and np.isfinite(sec).all()
    for i, c in enumerate(cases):
        sim = Simulation.from_case(c, precision="f64")
        ok, n, rr = sim.run_to_steady(tol=1e-9, max_steps=400000, check_every=500)
        assert ok and n == steps[i]
        for a, b in zip(batch.get_state(i), sim.get_state()):
            assert np.array_equal(a, b)
        sim.close()


def test_batch_rejects_time_dependent_boundaries():
    from paper_1902_02999_gb300 import Batch, MaclabError
    with pytest.raises(MaclabError):
        Batch([inputs.tidal_strip(60, 1)], precision="f32")


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_persistent_steps_equal_per_step_launches(precision):
    """One cooperative launch for many steps (grid barrier between steps)
    against one launch per step: bitwise the same after odd and even step
    counts, with bounce-back links, Dirichlet nodes outside their inward
    node's tile (east column of a 129-wide channel) and more tiles than
    resident blocks (a 1024 x 640 channel alone has 640 tiles)."""
    from paper_1902_02999_gb300 import Batch
    cases = mixed_cases()[:4] + [inputs.bump_channel(129, 40, seed=6), inputs.bump_channel(1024, 640, seed=3)]
    a = Batch(cases, precision=precision)
    a.set_persistent(0)
    b = Batch(cases, precision=precision)
    b.set_persistent(1)
    for n in (1, 2, 37, 120):
        a.step(n)
        b.step(n)
        for i in range(len(cases)):
            for x, y in zip(a.get_state(i), b.get_state(i)):
                assert np.array_equal(x, y), (n, i, cases[i].name)
    assert np.array_equal(a.residual(), b.residual())
    b.set_active([1, 0, 1, 1, 0, 1])
    a.set_active([1, 0, 1, 1, 0, 1])
    a.step(9)
    b.step(9)
    for i in range(len(cases)):
        for x, y in zip(a.get_state(i), b.get_state(i)):
            assert np.array_equal(x, y), ("inactive", i)
    for mode in (2, -1):
        with pytest.raises(Exception):
            b.set_persistent(mode)
    a.close()
    b.close()
