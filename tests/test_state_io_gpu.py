"""maclab_set_state / maclab_get_state with page-locked (mapped) host arrays,
which the conversion kernels read and write directly, give exactly the
states of pageable arrays, which go through the staged copies: both
directions, FP32 and FP64, after steps on a grid with every node kind."""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def pinned_like(a):
    t = torch.empty(a.size, dtype=torch.float64, pin_memory=True)
    out = t.numpy().reshape(a.shape)
    out[...] = a
    return out, t  # keep the tensor alive with its memory


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_pinned_and_pageable_state_transfers_agree(precision):
    """Two handles with the same history (the boundary values depend on
    time, and set_state keeps the time), one fed and read through pageable
    arrays, one through pinned arrays."""
    from paper_1902_02999_gb300 import Simulation
    case = inputs.random_case(301, 187, 7)
    rng = np.random.default_rng(3)
    sims = [Simulation.from_case(case, precision=precision) for _ in range(2)]
    for sim in sims:
        sim.step(5)
    h, u, v = sims[0].get_state()
    h1 = h + 1e-3 * rng.standard_normal(h.shape) * (case.mask > 0)
    u1 = u + 1e-3 * rng.standard_normal(u.shape)
    v1 = v + 1e-3 * rng.standard_normal(v.shape)
    sims[0].set_state(h1, u1, v1)
    ph = [pinned_like(a) for a in (h1, u1, v1)]
    sims[1].set_state(*[a for a, _ in ph])
    for sim in sims:
        sim.step(7)
    want = sims[0].get_state()
    outs = [pinned_like(np.zeros_like(a)) for a in want]
    got = sims[1].get_state(out=[a.reshape(-1) for a, _ in outs])
    for g, o, w in zip(got, outs, want):
        assert np.array_equal(o[0], w)
        assert np.array_equal(np.asarray(g).reshape(w.shape), w)
    for sim in sims:
        sim.close()
