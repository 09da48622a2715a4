"""The eLABSWE distribution form with a general relaxation time (Eq. lb.1,
maclab_set_relaxation) on the GPU against the FP64 oracle's distribution
form, element by element on h, u, v; mass conservation; argument checks.
Tolerances as for the macroscopic step: FP64 1e-12, FP32 2e-5 on h and 1e-4
on u, v (relative to max|h| and to the largest reference speed)."""
import numpy as np
import pytest

import inputs
import oracle
from inputs import BOUNCEBACK, FLUID, NOSLIP, PERIODIC, SOLID, SPECULAR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": (1e-12, 1e-12), "f32": (2e-5, 1e-4)}


def no_walls(case):
    c = case.copy()
    c.mask = np.where(c.mask == NOSLIP, FLUID, c.mask).astype(np.uint8)
    return c


_ORACLE = {}


def oracle_elab(key, case, tau, steps):
    """The oracle run, computed once per case and tau (both precisions use it)."""
    if key not in _ORACLE:
        _ORACLE[key] = oracle.elab_run(case, tau, steps)
    return _ORACLE[key]


def sim_of(case, precision, tau):
    from paper_1902_02999_gb300 import Simulation
    sim = Simulation.from_case(case, precision=precision)
    sim.set_relaxation(tau)
    assert sim.info["tau"] == tau
    return sim


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("tau", [0.7, 1.4])
@pytest.mark.parametrize("edges", [(PERIODIC,) * 4, (BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR),
                                   (SPECULAR, BOUNCEBACK, PERIODIC, PERIODIC)])
def test_distribution_form_matches_oracle(edges, tau, precision):
    case = no_walls(inputs.random_case(131, 70, 5, edges=edges, dirichlet=False))
    assert (case.mask == SOLID).any()
    steps = 300
    h, u, v, _ = oracle_elab((edges, tau), case, tau, steps)
    sim = sim_of(case, precision, tau)
    sim.step(steps)
    gh, gu, gv = sim.get_state()
    live = case.mask != SOLID
    th, tu = TOL[precision]
    assert np.abs(gh - h)[live].max() <= th * np.abs(h[live]).max()
    scale = np.hypot(u, v)[live].max()
    if precision == "f64":
        scale = max(scale, case.g * np.abs(h[live]).max() / case.e)
    assert np.abs(gu - u)[live].max() <= tu * scale and np.abs(gv - v)[live].max() <= tu * scale
    sim.close()


def test_mass_is_conserved_and_graphs_agree():
    case = no_walls(inputs.random_case(200, 90, 8, edges=(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR),
                                       dirichlet=False))
    live = case.mask != SOLID
    m0 = case.h0[live].sum()
    a = sim_of(case, "f64", 0.9)
    a.set_graph_steps(64)
    a.step(200)
    b = sim_of(case, "f64", 0.9)
    b.set_graph_steps(0)
    b.step(200)
    sa, sb = a.get_state(), b.get_state()
    assert all(np.array_equal(x[live], y[live]) for x, y in zip(sa, sb))
    assert abs(sa[0][live].sum() - m0) <= 1e-12 * m0
    r, mass, _ = a.residual()
    assert abs(mass - m0) <= 1e-12 * m0 and r > 0
    a.close()
    b.close()


def test_back_to_macroscopic_and_argument_checks():
    from paper_1902_02999_gb300 import MaclabError, Simulation
    case = no_walls(inputs.random_case(131, 70, 6, dirichlet=False))
    sim = sim_of(case, "f64", 1.2)
    sim.step(10)
    sim.set_relaxation(1.0)          # MacLABSWE from the current state
    mid = sim.get_state()
    sim.step(5)
    want = oracle.run(case, 5, mid)
    got = sim.get_state()
    live = case.mask != SOLID
    assert np.abs(got[0] - want[0])[live].max() <= 1e-12 * np.abs(want[0][live]).max()
    for bad in (0.5, 0.2, float("nan")):
        with pytest.raises(MaclabError):
            sim.set_relaxation(bad)
    sim.close()
    walled = Simulation.from_case(inputs.random_case(131, 70, 6, dirichlet=False), precision="f32")
    with pytest.raises(MaclabError):
        walled.set_relaxation(1.2)   # no-slip nodes
    walled.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_all_fluid_tiles_match_oracle(precision):
    """No solid node anywhere: every tile whose window lies in the grid
    streams without per-link checks; periodic x and specular y edges."""
    edges = (PERIODIC, PERIODIC, SPECULAR, SPECULAR)
    case = inputs.random_case(200, 70, 9, edges=edges, solids=False, dirichlet=False)
    assert (case.mask == FLUID).all()
    h, u, v, _ = oracle_elab(("dense", edges), case, 0.9, 200)
    sim = sim_of(case, precision, 0.9)
    sim.step(200)
    gh, gu, gv = sim.get_state()
    th, tu = TOL[precision]
    assert np.abs(gh - h).max() <= th * np.abs(h).max()
    scale = np.hypot(u, v).max()
    if precision == "f64":
        scale = max(scale, case.g * np.abs(h).max() / case.e)
    assert np.abs(gu - u).max() <= tu * scale and np.abs(gv - v).max() <= tu * scale
    sim.close()
