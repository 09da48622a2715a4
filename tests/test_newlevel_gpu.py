"""The new-level hbar variant (maclab_set_hbar_level(sim, 1), Eq. h-bar as
written) on the GPU against the oracle's variant, element by element;
lake at rest stays exactly at rest in FP32; level 0 restores the default
step.  Tolerances as for the default step."""
import numpy as np
import pytest

import inputs
import oracle
from inputs import BOUNCEBACK, PERIODIC, SOLID, SPECULAR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": (1e-12, 1e-12), "f32": (2e-5, 1e-4)}


def check(case, got, want, precision):
    live = case.mask != SOLID
    th, tu = TOL[precision]
    assert np.abs(got[0] - want[0])[live].max() <= th * np.abs(want[0][live]).max()
    scale = np.hypot(want[1], want[2])[live].max()
    if precision == "f64":
        scale = max(scale, case.g * np.abs(want[0][live]).max() / case.e)
    assert np.abs(got[1] - want[1])[live].max() <= tu * scale
    assert np.abs(got[2] - want[2])[live].max() <= tu * scale


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("edges", [(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR), (PERIODIC,) * 4])
def test_new_level_matches_oracle(edges, precision):
    from paper_1902_02999_gb300 import Simulation
    case = inputs.random_case(131, 70, 12, edges=edges)
    want = oracle.run_newlevel(case, 300)
    sim = Simulation.from_case(case, precision=precision)
    sim.set_hbar_level(1)
    sim.step(300)
    check(case, sim.get_state(), want, precision)
    # back to the old level: continues as the default step
    sim.set_hbar_level(0)
    sim.step(20)
    check(case, sim.get_state(), oracle.run(case, 20, want, n0=300), precision)
    sim.close()


def test_new_level_lake_at_rest_is_exact_in_fp32():
    from paper_1902_02999_gb300 import Simulation
    case = inputs.random_case(131, 70, 13)
    case.wind_u = case.wind_v = 0.0
    D = case.h_ref - case.zb
    case.h0 = np.where(case.mask == SOLID, 0.0, D)
    case.u0 = np.zeros_like(D)
    case.v0 = np.zeros_like(D)
    case.bc = np.zeros_like(np.asarray(case.bc, dtype=np.float64))
    case.mask = np.where(case.mask >= 3, 1, case.mask).astype(np.uint8)   # no Dirichlet data
    sim = Simulation.from_case(case, precision="f32")
    sim.set_hbar_level(1)
    sim.step(500)
    h, u, v = sim.get_state()
    live = case.mask != SOLID
    eta = sim.device_state()[0].cpu().numpy()[:, :case.nx]
    assert (eta[live] == 0).all() and (u[live] == 0).all() and (v[live] == 0).all()
    sim.close()
