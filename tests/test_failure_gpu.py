"""Failure detection on the GPU without a fault: the persistent batch
kernel's grid barrier is made to wait for one block more than the launch
holds (a test hook), so every bounded wait runs out.  The library must
report the error status at the next residual / state read, refuse the
half-advanced state, and become usable again once every instance is
reloaded, with results equal to a batch that never failed."""
import numpy as np
import pytest

import inputs
from inputs import BOUNCEBACK, SPECULAR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MACLAB_E_CUDA, MACLAB_E_STATE = -2, -5


def cases():
    return [inputs.random_case(70, 40, 3, edges=(BOUNCEBACK,) * 4, dirichlet=False),
            inputs.dish_lake(48, seed=1),
            inputs.bump_channel(130, 40, seed=2),
            inputs.random_case(33, 65, 4, edges=(SPECULAR,) * 4, dirichlet=False)]


def test_grid_barrier_wait_runs_out_and_is_reported():
    from paper_1902_02999_gb300 import Batch, MaclabError
    cs = cases()
    batch = Batch(cs, precision="f32")
    batch.set_persistent(1)
    start = [batch.get_state(i) for i in range(len(cs))]
    # no barrier can complete: every block gives up after 2^12 polls
    batch.set_barrier_test(1, 1 << 12)
    batch.step(6)                        # asynchronous: returns before the waits run out
    with pytest.raises(MaclabError) as err:
        batch.residual()
    assert err.value.code == MACLAB_E_CUDA
    # the device state matches no step count: refused until reloaded
    for call in (lambda: batch.residual(), lambda: batch.get_state(0), lambda: batch.step(1)):
        with pytest.raises(MaclabError) as err:
            call()
        assert err.value.code == MACLAB_E_STATE
    batch.set_barrier_test(0, 1 << 22)
    for i in range(len(cs) - 1):
        batch.set_state(i, *start[i])
        with pytest.raises(MaclabError):
            batch.step(1)                # one instance still holds a half-advanced state
    batch.set_state(len(cs) - 1, *start[-1])
    # usable again, and the same as a batch that never failed
    batch.step(6)
    got = [batch.get_state(i) for i in range(len(cs))]
    ref = Batch(cs, precision="f32")
    ref.set_persistent(1)
    for i in range(len(cs)):
        ref.set_state(i, *start[i])
    ref.step(6)
    for i in range(len(cs)):
        for a, b in zip(got[i], ref.get_state(i)):
            assert np.array_equal(a, b), i
    assert np.all(np.isfinite(batch.residual()[:, 0]))
