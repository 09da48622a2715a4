"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs.

Tolerances (relative max-norm over non-solid nodes):
  FP64 storage: <= 1e-12 on h, u, v after 1000 steps.
  FP32 storage: <= 2e-5 on h and <= 1e-4 on u, v after 1000 steps.
h is normalised by max|h|, u and v by the largest reference speed, and
every comparison prints its three errors (the FP32 error against the FP64
oracle, reported per result).  One exception, named by the tests that use
it (conditioned=True): on the tidal strips (h ~ 16 m, |u| < 0.06 m/s) the
momentum of Eq. Mac.lb.7 is a sum of terms of size ~g h^2 / (6 e) whose
rounding the oracle itself carries -- two builds of the same oracle, with
and without fused multiply-add, differ by 2.5e-11 relative to max|u| after
2000 steps -- so there the FP64 u, v errors are normalised by
max(largest speed, g h_max / e); the speed-normalised error is printed
beside it.  Lake at rest is checked bitwise in FP32 (the perturbation form
makes it exact).  The full-size channel (8192 x 2048) runs in the same
launch configuration as the benchmark and is compared on every node after
one step and after two; a 512 x 128 channel of the same family is
compared after 1000 steps.
"""
import functools
import math

import numpy as np
import pytest

import inputs
import oracle
from inputs import BOUNCEBACK, DIR_H, FLUID, NOSLIP, PERIODIC, SOLID, SPECULAR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": (1e-12, 1e-12), "f32": (2e-5, 1e-4)}


def sim_of(case, precision, **kw):
    from paper_1902_02999_gb300 import Simulation
    return Simulation.from_case(case, precision=precision, **kw)


def relerr(a, b, live):
    if not live.any():
        return 0.0
    scale = max(np.abs(b[live]).max(), 1e-300)
    return float(np.abs(a[live] - b[live]).max() / scale)


def compare(case, got, want, precision, label="", conditioned=False):
    live = case.mask != SOLID
    th, tu = TOL[precision]
    assert np.isfinite(got[0][live]).all()
    eh = relerr(got[0], want[0], live)
    scale = max(np.hypot(want[1], want[2])[live].max(), 1e-30)
    eu = float(np.abs(got[1] - want[1])[live].max() / scale)
    ev = float(np.abs(got[2] - want[2])[live].max() / scale)
    line = "%s %s: h %.3g, u %.3g, v %.3g (speed-normalised)" % (label, precision, eh, eu, ev)
    if conditioned and precision == "f64":
        scale_c = max(scale, case.g * np.abs(want[0][live]).max() / case.e)
        eu, ev = eu * scale / scale_c, ev * scale / scale_c
        line += "; u %.3g, v %.3g against max(speed, g h / e)" % (eu, ev)
    print(line)
    assert eh <= th, (label, "h", eh)
    assert eu <= tu and ev <= tu, (label, "u,v", eu, ev)
    if (case.mask == NOSLIP).any():
        assert (got[1][case.mask == NOSLIP] == 0).all()
    return eh, eu, ev


CASES = [
    # (nx, ny, seed, edges)  -- sizes span several 62-column warp strips and ragged tails
    (131, 97, 1, (BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR)),
    (67, 45, 2, (PERIODIC, PERIODIC, SPECULAR, SPECULAR)),
    (125, 66, 3, (SPECULAR, SPECULAR, SPECULAR, SPECULAR)),
    (64, 63, 4, (PERIODIC, PERIODIC, PERIODIC, PERIODIC)),
    (63, 40, 5, (BOUNCEBACK, BOUNCEBACK, BOUNCEBACK, BOUNCEBACK)),
    (190, 33, 6, (BOUNCEBACK, SPECULAR, PERIODIC, PERIODIC)),
]
# Dirichlet rows on the S / N edges as well (with and without W / E columns)
CASES_SN = [
    (131, 97, 7, (BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR)),
    (100, 60, 8, (PERIODIC, PERIODIC, BOUNCEBACK, BOUNCEBACK)),
]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny,seed,edges", CASES)
def test_parity_random(nx, ny, seed, edges, precision):
    case = inputs.random_case(nx, ny, seed, edges=edges)
    nsteps = 1000
    want = oracle.run(case, nsteps)
    sim = sim_of(case, precision)
    sim.step(nsteps)
    got = sim.get_state()
    compare(case, got, want, precision, (nx, ny, seed, edges))
    assert sim.time()[1] == nsteps


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny,seed,edges", CASES_SN)
def test_parity_dirichlet_rows(nx, ny, seed, edges, precision):
    case = inputs.random_case(nx, ny, seed, edges=edges, dirichlet_sn=True)
    assert (case.mask[0, 2:-2] == inputs.DIR_Q).all() and (case.mask[-1, 2:-2] == DIR_H).all()
    want = oracle.run(case, 1000)
    sim = sim_of(case, precision)
    sim.step(1000)
    compare(case, sim.get_state(), want, precision, ("SN", nx, ny, seed, edges))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_hand_step_3x3(precision):
    rows = np.loadtxt(__file__.replace("test_parity_gpu.py", "golden/hand_step_3x3.txt"))
    z = np.zeros((3, 3))
    c = inputs.Case("hand", 3, 3, 1.0, 2.0, z, np.full((3, 3), FLUID, np.uint8), np.ones((3, 3)),
                    z.copy(), z.copy(), edges=(PERIODIC,) * 4, h_ref=1.0)
    c.h0[1, 1] = 1.1
    sim = sim_of(c, precision)
    sim.step(1)
    h, u, v = sim.get_state()
    tol = 1e-14 if precision == "f64" else 2e-7
    for i, j, hn, hun, hvn in rows:
        i, j = int(i), int(j)
        assert abs(h[j, i] - hn) < tol
        assert abs(h[j, i] * u[j, i] - hun) < tol
        assert abs(h[j, i] * v[j, i] - hvn) < tol


@pytest.mark.parametrize("rows", [1, 3, 8, 1000])
def test_tile_rows_do_not_change_results(rows):
    case = inputs.random_case(131, 50, 9, edges=(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR))
    ref = sim_of(case, "f32")
    ref.step(50)
    a = ref.get_state()
    sim = sim_of(case, "f32")
    sim.set_tile_rows(rows)
    sim.step(50)
    b = sim.get_state()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_autotune_keeps_state_and_results(precision):
    case = inputs.random_case(131, 60, 21, edges=(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR))
    a = sim_of(case, precision)
    a.step(7)
    before = a.get_state()
    choice = a.autotune(4)
    assert 0 <= choice <= (6 if precision == "f32" else 4) and a.time()[1] == 7
    assert a.info["temporal_block"] == (2 if choice == 6 else 1)
    for x, y in zip(a.get_state(), before):
        assert np.array_equal(x, y)
    a.step(30)
    b = sim_of(case, precision)
    b.step(37)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_graph_replay_is_bitwise_identical(precision):
    """maclab_step replays captured CUDA graphs for steady boundary data;
    the result equals one launch per step."""
    case = inputs.dish_lake(96, seed=5)
    a = sim_of(case, precision)
    a.set_graph_steps(0)
    b = sim_of(case, precision)
    b.set_graph_steps(8)
    for n in (3, 16, 29):          # blocks of 8 plus odd remainders, both parities
        a.step(n)
        b.step(n)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert a.time() == b.time()
    ra, rb = a.residual(), b.residual()
    assert ra == rb


@pytest.mark.parametrize("n", [64, 101])
def test_lake_at_rest_bitwise_f32(n):
    case = inputs.dish_lake(n, seed=3)
    case.wind_u = case.wind_v = 0.0
    sim = sim_of(case, "f32", initial=False)   # still water: eta = 0, u = v = 0
    sim.step(1000)
    eta, u, v = (t.cpu().numpy() for t in sim.device_state())
    assert (eta == 0).all() and (u == 0).all() and (v == 0).all()
    h, _, _ = sim.get_state()
    live = case.mask != SOLID
    assert (h[live] == (case.h_ref - case.zb)[live]).all()


def test_lake_at_rest_f64_arbitrary_bed():
    case = inputs.random_case(90, 70, 12, edges=(SPECULAR,) * 4, dirichlet=False)
    live = case.mask != SOLID
    case.h0 = np.where(live, case.h_ref - case.zb, 0.0)
    case.u0[:] = 0
    case.v0[:] = 0
    case.wind_u = case.wind_v = 0.0
    sim = sim_of(case, "f64")
    sim.step(1000)
    h, u, v = sim.get_state()
    assert np.abs(h - case.h0)[live].max() < 1e-13
    assert np.abs(u).max() < 1e-13 and np.abs(v).max() < 1e-13


@pytest.mark.parametrize("precision,tol", [("f64", 1e-13), ("f32", 2e-6)])
def test_mass_conservation_closed_basin(precision, tol):
    case = inputs.random_case(140, 90, 13, edges=(BOUNCEBACK,) * 4, dirichlet=False)
    live = case.mask != SOLID
    m0 = case.h0[live].sum()
    sim = sim_of(case, precision)
    sim.step(1000)
    r, mass, umax = sim.residual()
    assert abs(mass - m0) / m0 < tol
    h, _, _ = sim.get_state()
    assert abs(h[live].sum() - m0) / m0 < tol


def test_residual_matches_oracle():
    case = inputs.random_case(77, 51, 14)
    s1 = oracle.run(case, 30)
    s2 = oracle.run(case, 1, s1, n0=30)
    r_o, m_o, u_o = oracle.residual(case, s1, s2)
    sim = sim_of(case, "f64")
    sim.step(31)
    r, m, umax = sim.residual()
    assert abs(r - r_o) <= 1e-9 * r_o
    assert abs(m - m_o) <= 1e-12 * m_o
    assert abs(umax - u_o) <= 1e-11 * u_o


def test_paper_tidal_case_on_gpu():
    """Section 4.1 at the paper's resolution, FP64 on the GPU: matches the
    oracle and keeps the level error under the paper's 0.005 %."""
    case = inputs.tidal_strip(201, 1)
    n = int(round(10800.0 / case.dt))
    sim = sim_of(case, "f64")
    sim.step(n)
    h, u, v = sim.get_state()
    want = oracle.run(case, n)
    compare(case, (h, u, v), want, "f64", "tidal", conditioned=True)
    om = 4 * math.pi / 86400
    eta = 20 - 4 * math.sin(om * n * case.dt + math.pi / 2)
    assert np.abs(h[0] + case.zb[0] - eta).max() / eta < 5e-5


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_coriolis_inertial_oscillation(precision):
    """Uniform flow on a flat periodic domain with Coriolis only: every node
    follows w_{n+1} = (1 - i dt Omega) w_n for w = u + i v (the centred force
    of a uniform state, Eq. SWE-force), so after n steps the velocity has
    turned by n atan(dt Omega) and grown by (1 + (dt Omega)^2)^(n/2)."""
    n, steps = 64, 3000
    z = np.zeros((n, n))
    c = inputs.Case("inertial", n, n, 10.0, 20.0, z, np.full((n, n), FLUID, np.uint8), np.full((n, n), 3.0),
                    np.full((n, n), 0.2), np.full((n, n), -0.1), edges=(PERIODIC,) * 4, h_ref=3.0)
    c.omega = 1.0e-4
    sim = sim_of(c, precision)
    sim.step(steps)
    h, u, v = sim.get_state()
    w = (0.2 - 0.1j) * (1 - 1j * c.dt * c.omega) ** steps
    assert abs(np.angle(w / (0.2 - 0.1j))) > 0.05          # a visible turn
    th, tu = TOL[precision]
    assert np.abs(h - 3.0).max() <= th * 3.0
    assert np.abs(u - w.real).max() <= tu * abs(w) and np.abs(v - w.imag).max() <= tu * abs(w)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_tidal_strip_400x3(precision):
    """The 400 x 3 strip with free-slip side walls, 2000 steps."""
    case = inputs.tidal_strip(400, 3)
    sim = sim_of(case, precision)
    sim.step(2000)
    compare(case, sim.get_state(), oracle.run(case, 2000), precision, "strip", conditioned=True)


@pytest.mark.parametrize("nx,ny,edges", [
    (1, 1, (PERIODIC,) * 4), (2, 3, (PERIODIC,) * 4), (1, 7, (SPECULAR,) * 4),
    (9, 1, (SPECULAR,) * 4), (65, 2, (PERIODIC, PERIODIC, SPECULAR, SPECULAR)),
    (127, 5, (SPECULAR, BOUNCEBACK, PERIODIC, PERIODIC)), (3, 3, (BOUNCEBACK,) * 4)])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_small_and_degenerate_grids(nx, ny, edges, precision):
    case = inputs.random_case(nx, ny, 40 + nx, edges=edges, solids=False, dirichlet=False, amp=0.1)
    want = oracle.run(case, 20)
    sim = sim_of(case, precision)
    sim.step(20)
    compare(case, sim.get_state(), want, precision, (nx, ny))


def test_all_solid_grid_is_inert():
    case = inputs.random_case(20, 10, 50, dirichlet=False)
    case.mask[:] = SOLID
    sim = sim_of(case, "f32")
    h0, u0, v0 = sim.get_state()
    sim.step(5)
    h1, u1, v1 = sim.get_state()
    assert np.array_equal(h0, h1) and np.array_equal(u0, u1)
    r, mass, umax = sim.residual()
    assert r == 0.0 and mass == 0.0


def test_state_roundtrip_and_time():
    case = inputs.random_case(70, 30, 60)
    sim = sim_of(case, "f64")
    h, u, v = sim.get_state()
    live = case.mask != SOLID
    assert np.abs(h - case.h0)[live].max() < 1e-15
    assert np.array_equal(u[live], case.u0[live])
    sim.step(7)
    t, n = sim.time()
    assert n == 7 and abs(t - 7 * case.dt) < 1e-12
    s7 = sim.get_state()
    sim.set_state(*s7)
    sim.step(3)
    a = sim.get_state()
    want = oracle.run(case, 3, s7, n0=7)
    compare(case, a, want, "f64", "resume")


def test_errors_are_reported():
    from paper_1902_02999_gb300 import MaclabError
    case = inputs.random_case(30, 20, 70)
    bad = case.copy()
    bad.mask[10, 10] = DIR_H                       # Dirichlet node off the edge
    with pytest.raises(MaclabError) as ei:
        sim_of(bad, "f32")
    assert ei.value.code == -1
    sim = sim_of(case, "f32")
    with pytest.raises(MaclabError) as ei:
        sim.residual()                             # no step yet
    assert ei.value.code == -5
    h = case.h0.copy()
    j, i = np.argwhere(case.mask == FLUID)[len(np.argwhere(case.mask == FLUID)) // 2]
    h[j, i] = np.nan
    sim.set_state(h, case.u0, case.v0)
    sim.step(2)
    with pytest.raises(MaclabError) as ei:
        sim.residual()
    assert ei.value.code == -4


def test_run_to_steady_converges():
    """Coarse Section 4.3 hump (41 x 41, dx = 25 m; nu = 75 m^2/s keeps the
    lattice speed e = 18 m/s above sqrt(g h) and R_le < 1) run to a residual
    of 1e-9; the steady state matches the oracle after the same steps."""
    case = inputs.paper_hump(41)
    case.nu = 75.0
    sim = sim_of(case, "f64")
    ok, steps, r = sim.run_to_steady(tol=1e-9, max_steps=200000, check_every=500)
    assert ok and r <= 1e-9 and steps % 500 == 0
    _, _, umax = sim.residual()
    assert umax * case.dx / case.nu < 1.0          # R_le < 1 (Section 3)
    compare(case, sim.get_state(), oracle.run(case, steps), "f64", "steady")


@pytest.mark.parametrize("precision", ["f32"])
def test_full_size_bump_channel(precision):
    """8192 x 2048 channel in the benchmark's launch configuration, every
    node compared with the oracle after one step and after two."""
    case = inputs.bump_channel(8192, 2048, seed=0)
    sim = sim_of(case, precision)
    sim.step(1)
    s1 = sim.get_state()
    w1 = oracle.step(case, case.h0, case.u0, case.v0, case.dt)
    compare(case, s1, w1, precision, "full-1")
    sim.step(1)
    w2 = oracle.step(case, *w1, 2 * case.dt)
    compare(case, sim.get_state(), w2, precision, "full-2")


def test_full_size_channel_1000_steps():
    """8192 x 2048, 1000 steps: the row-march kernel (the benchmark's) and
    the tile kernel agree bitwise on every node; both are compared with the
    oracle after 1000 steps on the 512 x 128 channel below and on the random
    grids above, and on the full grid after one and two steps."""
    case = inputs.bump_channel(8192, 2048, seed=0)
    out = []
    for kernel in ("march", "tile"):
        sim = sim_of(case, "f32")
        sim.set_step_kernel(kernel)
        sim.step(1000)
        out.append(sim.get_state())
        sim.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@functools.lru_cache(maxsize=1)
def channel_slice():
    case = inputs.bump_channel(512, 128, seed=0)
    return case, oracle.run(case, 1000)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_channel_slice_1000_steps(precision):
    """A 512 x 128 channel of the benchmark's family (same dx, nu, depth,
    inflow, outflow, friction; bump scaled with the grid), 1000 steps."""
    case, want = channel_slice()
    sim = sim_of(case, precision)
    sim.step(1000)
    compare(case, sim.get_state(), want, precision, "channel-512x128")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_interval_residual_matches_oracle(precision):
    """maclab_residual_since_mark over 37 steps (and the batch's) against
    the oracle's interval residual on the same two states."""
    from paper_1902_02999_gb300 import Batch
    case = inputs.random_case(90, 50, 81)
    sim = sim_of(case, precision)
    sim.step(30)
    s30 = sim.get_state()
    sim.mark()
    sim.step(37)
    r, m, umax = sim.residual_since_mark()
    r_o, m_o, u_o = oracle.residual(case, s30, sim.get_state(), interval=37)
    tol = 1e-9 if precision == "f64" else 1e-5
    assert abs(r - r_o) <= tol * r_o and abs(m - m_o) <= 1e-12 * m_o
    steady = case.copy()
    steady.bc[:, :, 1] = 0.0
    b = Batch([steady], precision=precision)
    b.step(30)
    b30 = b.get_state(0)
    b.mark()
    b.step(37)
    rb = b.residual_since_mark()[0, 0]
    rb_o = oracle.residual(steady, b30, b.get_state(0), interval=37)[0]
    assert abs(rb - rb_o) <= tol * rb_o
