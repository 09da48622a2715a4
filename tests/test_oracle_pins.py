"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets a term of the update so that a dropped term, a wrong sign,
a wrong index or a transposed operand in the oracle fails at least one:

* Eq. feq-full moments            -> f^eq, lambda_a, lattice numbering
* 3x3 step worked by hand         -> streaming sum of Eqs. Mac.lb.6/7
* lake at rest over any bed       -> bed-slope term, hbar, bounce-back
* mass in closed/periodic basins  -> antisymmetric link terms, bounce-back
* uniform flow / uniform force    -> momentum moments, force weights
* shear-wave decay                -> viscosity of Eq. mlb-viscosity
* mirror symmetry                 -> index / sign conventions
* push form of Eq. lb.1 (tau = 1) -> pull/push transposition
"""
import math
import os

import numpy as np
import pytest

import inputs
import oracle
from inputs import (BOUNCEBACK, DIR_H, DIR_HU, DIR_Q, E, FLUID, NOSLIP, PERIODIC, S, SOLID,
                    SPECULAR, W, Case)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# D2Q9 lattice vectors in the numbering of Section 3 (south-wall unknowns
# 2,3,4 pair with 6,7,8); written out here independently of the oracle.
C = np.array([(0, 0), (1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)],
             dtype=float)


def flat_periodic(nx, ny, h=1.0, u=0.0, v=0.0, e=12.0):
    z = np.zeros((ny, nx))
    return Case("flat", nx, ny, 1.0, e / 6.0, z, np.full((ny, nx), FLUID, np.uint8),
                np.full((ny, nx), h), np.full((ny, nx), u), np.full((ny, nx), v),
                edges=(PERIODIC,) * 4)


@pytest.mark.parametrize("seed", range(5))
def test_feq_moments(seed):
    """Eq. feq-full: sum f = h, sum e_a f = h u, sum e_ai e_aj f = g h^2/2 delta + h u_i u_j."""
    rng = inputs.Rng(100 + seed)
    h, u, v = rng.scalar(0.1, 20), rng.scalar(-2, 2), rng.scalar(-2, 2)
    e, g = rng.scalar(5, 60), 9.81
    f = oracle.feq(h, u, v, e, g)
    ea = e * C
    assert abs(f.sum() - h) <= 1e-13 * h
    np.testing.assert_allclose(ea.T @ f, [h * u, h * v], rtol=0, atol=1e-13 * e * h)
    second = np.einsum("ai,aj,a->ij", ea, ea, f)
    want = g * h * h / 2 * np.eye(2) + h * np.outer([u, v], [u, v])
    np.testing.assert_allclose(second, want, rtol=0, atol=1e-12 * e * e * h)


def test_feq_lambda_weights():
    """At rest f^eq_a = lambda_a g h^2/(6 e^2): lambda = 1 on axes, 1/4 on diagonals."""
    f = oracle.feq(2.0, 0.0, 0.0, 10.0, 9.81)
    base = 9.81 * 4.0 / 600.0
    np.testing.assert_allclose(f[1::2], base, rtol=1e-15)
    np.testing.assert_allclose(f[2::2], base / 4, rtol=1e-15)
    assert abs(f[0] - 2.0 * (1 - 5 * 9.81 * 2.0 / 600.0)) < 1e-15


def test_hand_step_3x3():
    """Golden values worked by hand (tests/golden/hand_step_3x3.txt)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "hand_step_3x3.txt"))
    c = flat_periodic(3, 3, e=12.0)
    c.h0[1, 1] = 1.1
    h, u, v = oracle.step(c, c.h0, c.u0, c.v0, c.dt)
    for i, j, hn, hun, hvn in rows:
        i, j = int(i), int(j)
        assert abs(h[j, i] - hn) < 1e-15
        assert abs(h[j, i] * u[j, i] - hun) < 1e-15
        assert abs(h[j, i] * v[j, i] - hvn) < 1e-15
    assert abs(h.sum() - 9.1) < 1e-14


def rest_case(seed, edges):
    c = inputs.random_case(26, 22, seed, edges=edges, dirichlet=False)
    fl = c.mask != SOLID
    c.h0 = np.where(fl, c.h_ref - c.zb, 0.0)
    c.u0[:] = 0.0
    c.v0[:] = 0.0
    c.wind_u = c.wind_v = 0.0
    return c


@pytest.mark.parametrize("edges", [(BOUNCEBACK,) * 4, (SPECULAR,) * 4,
                                   (PERIODIC, PERIODIC, SPECULAR, SPECULAR)])
@pytest.mark.parametrize("seed", [0, 1])
def test_lake_at_rest(seed, edges):
    """Still water over an arbitrary bed stays still (bed term with hbar of Eq. h-bar)."""
    c = rest_case(seed, edges)
    h, u, v = oracle.run(c, 100)
    fl = c.mask != SOLID
    assert np.abs(h - c.h0)[fl].max() < 1e-13
    assert np.abs(u).max() < 1e-13 and np.abs(v).max() < 1e-13


def test_lake_at_rest_fails_with_wrong_bed_sign():
    """Control: the at-rest balance really involves the bed term -- a still
    surface with the bed but no depth adjustment is not at rest."""
    c = rest_case(3, (BOUNCEBACK,) * 4)
    c.h0 = np.where(c.mask != SOLID, 1.0, 0.0)  # flat depth over a sloping bed
    h, _, _ = oracle.run(c, 5)
    assert np.abs(h - c.h0)[c.mask != SOLID].max() > 1e-6


@pytest.mark.parametrize("edges", [(BOUNCEBACK,) * 4, (PERIODIC,) * 4, (SPECULAR,) * 4,
                                   (PERIODIC, PERIODIC, BOUNCEBACK, SPECULAR)])
def test_mass_conservation(edges):
    """sum h is invariant with wind, friction, Coriolis, solids and walls."""
    c = inputs.random_case(24, 20, 7, edges=edges, dirichlet=False)
    fl = c.mask != SOLID
    m0 = c.h0[fl].sum()
    h, u, v = oracle.run(c, 400)
    assert abs(h[fl].sum() - m0) <= 2e-14 * m0
    assert np.abs(u[c.mask == NOSLIP]).max(initial=0) == 0.0


def test_uniform_flow_is_fixed_point():
    c = flat_periodic(7, 5, h=1.3, u=0.21, v=-0.17)
    h, u, v = oracle.run(c, 30)
    np.testing.assert_allclose(h, 1.3, rtol=1e-14)
    np.testing.assert_allclose(u, 0.21, rtol=1e-13)
    np.testing.assert_allclose(v, -0.17, rtol=1e-13)


def test_uniform_wind_force():
    """Uniform state, uniform wind: h unchanged, h u grows by dt tau_w / rho per step."""
    c = flat_periodic(5, 4, h=1.7, u=0.1, v=0.05)
    c.wind_u, c.wind_v = 6.0, -3.0
    wm = math.hypot(6.0, -3.0)
    fx = c.rho_a * c.cw * 6.0 * wm / c.rho_w
    fy = c.rho_a * c.cw * -3.0 * wm / c.rho_w
    h, u, v = oracle.run(c, 10)
    np.testing.assert_allclose(h, 1.7, rtol=1e-14)
    np.testing.assert_allclose(h * u, 1.7 * 0.1 + 10 * c.dt * fx, rtol=1e-12)
    np.testing.assert_allclose(h * v, 1.7 * 0.05 + 10 * c.dt * fy, rtol=1e-12)


def test_uniform_friction_and_coriolis_recurrence():
    """Uniform state: u_{n+1} = u_n + dt F(u_n)/h with F = -C_b u|u| + Omega h (v,-u)."""
    c = flat_periodic(4, 4, h=2.0, u=0.5, v=-0.3)
    c.cb, c.omega = 0.004, 1.2e-3
    u, v = 0.5, -0.3
    state = (c.h0, c.u0, c.v0)
    for n in range(6):
        sp = math.hypot(u, v)
        fx = -c.cb * u * sp + c.omega * 2.0 * v
        fy = -c.cb * v * sp - c.omega * 2.0 * u
        u, v = u + c.dt * fx / 2.0, v + c.dt * fy / 2.0
        state = oracle.run(c, 1, state, n0=n)
        np.testing.assert_allclose(state[0], 2.0, rtol=1e-14)
        np.testing.assert_allclose(state[1], u, rtol=1e-13)
        np.testing.assert_allclose(state[2], v, rtol=1e-13)


@pytest.mark.parametrize("ny", [32, 64])
def test_shear_wave_viscosity(ny):
    """A shear wave u = U sin(k y) decays at nu k^2 with nu = e dx / 6
    (Eq. mlb-viscosity), to second order in k dx."""
    c = flat_periodic(2, ny, h=1.0, e=12.0)
    k = 2 * math.pi / ny
    U = 1e-4
    c.u0 = np.tile((U * np.sin(k * (np.arange(ny) + 0.5)))[:, None], (1, 2))
    n = 40
    _, u, _ = oracle.run(c, n)
    amp = 2.0 / ny * np.sum(u[:, 0] * np.sin(k * (np.arange(ny) + 0.5)))
    rate = -math.log(amp / U) / (n * c.dt)
    nu = c.e * c.dx / 6.0
    err = abs(rate / (nu * k * k) - 1.0)
    assert err < 2.5 * (k * c.dx) ** 2 / 12 + 1e-6
    assert err < 2e-3


def mirror_case(c, axis):
    m = c.copy()
    flip = (lambda a: a[:, ::-1]) if axis == "x" else (lambda a: a[::-1, :])
    for f in ("zb", "mask", "h0", "u0", "v0"):
        setattr(m, f, np.ascontiguousarray(flip(getattr(m, f))))
    if axis == "x":
        m.u0, m.wind_u = -m.u0, -m.wind_u
        m.edges = (c.edges[E], c.edges[W], c.edges[S], c.edges[3])
    else:
        m.v0, m.wind_v = -m.v0, -m.wind_v
        m.edges = (c.edges[W], c.edges[E], c.edges[3], c.edges[S])
    m.omega = -m.omega  # a mirror reverses the sense of rotation
    return m, flip


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("edges", [(BOUNCEBACK, SPECULAR, PERIODIC, PERIODIC),
                                   (SPECULAR, BOUNCEBACK, BOUNCEBACK, SPECULAR)])
def test_mirror_symmetry(axis, edges):
    c = inputs.random_case(20, 17, 11, edges=edges, dirichlet=False)
    m, flip = mirror_case(c, axis)
    h, u, v = oracle.run(c, 20)
    hm, um, vm = oracle.run(m, 20)
    np.testing.assert_allclose(flip(hm), h, rtol=0, atol=1e-13)
    sx, sy = (-1, 1) if axis == "x" else (1, -1)
    np.testing.assert_allclose(sx * flip(um), u, rtol=0, atol=1e-13)
    np.testing.assert_allclose(sy * flip(vm), v, rtol=0, atol=1e-13)


def test_transpose_symmetry():
    """Swapping x and y (and u with v, wind_u with wind_v) transposes the result."""
    c = inputs.random_case(18, 18, 12, edges=(SPECULAR, BOUNCEBACK, SPECULAR, BOUNCEBACK),
                           dirichlet=False)
    t = c.copy()
    for f in ("zb", "mask", "h0"):
        setattr(t, f, np.ascontiguousarray(getattr(c, f).T))
    t.u0, t.v0 = np.ascontiguousarray(c.v0.T), np.ascontiguousarray(c.u0.T)
    t.wind_u, t.wind_v = c.wind_v, c.wind_u
    t.omega = -c.omega
    h, u, v = oracle.run(c, 15)
    ht, ut, vt = oracle.run(t, 15)
    np.testing.assert_allclose(ht.T, h, rtol=0, atol=1e-13)
    np.testing.assert_allclose(vt.T, u, rtol=0, atol=1e-13)
    np.testing.assert_allclose(ut.T, v, rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_push_form_matches(seed):
    """Pull form (Eqs. Mac.lb.6/7) equals the push form of Eq. lb.1 at tau = 1
    followed by the moments of Eqs. fea-0-h / fea-0-v."""
    c = inputs.random_case(13, 11, 20 + seed, edges=(PERIODIC,) * 4, solids=False,
                           dirichlet=False)
    a = oracle.step(c, c.h0, c.u0, c.v0, c.dt)
    b = oracle.step_push(c, c.h0, c.u0, c.v0)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-13)


def test_specular_strip_matches_periodic_and_1d():
    """For y-invariant data, free-slip side walls, periodic sides and a
    single-row strip give the same result."""
    base = inputs.tidal_strip(60, 3)
    base.mask[:] = FLUID
    base.mask[:, -1] = NOSLIP
    base.u0 = np.tile(0.3 * np.sin(np.arange(60) / 7.0), (3, 1))
    base.cb, base.wind_u = 0.003, 4.0
    per = base.copy()
    per.edges = (BOUNCEBACK, BOUNCEBACK, PERIODIC, PERIODIC)
    one = base.copy()
    for f in ("zb", "mask", "h0", "u0", "v0"):
        setattr(one, f, np.ascontiguousarray(getattr(base, f)[:1]))
    one.ny = 1
    a = oracle.run(base, 50)
    b = oracle.run(per, 50)
    d = oracle.run(one, 50)
    for x, y, z in zip(a, b, d):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-13)
        np.testing.assert_allclose(x[1], z[0], rtol=0, atol=1e-13)


def test_dirichlet_rules():
    """DIR_H takes h(t_{n+1}); DIR_Q takes q(t_{n+1}); each unprescribed
    quantity takes the new value of the first inward node."""
    c = inputs.random_case(16, 12, 31)
    s0 = (c.h0, c.u0, c.v0)
    t1 = 4 * c.dt
    h, u, v = oracle.step(c, *s0, t1)

    def wave(p):
        return p[0] + p[1] * math.sin(p[2] * t1 + p[3])

    for j in range(c.ny):
        kind = c.mask[j, 0]
        if kind == DIR_H:
            assert h[j, 0] == wave(c.bc[W, 0])
            assert u[j, 0] == u[j, 1] and v[j, 0] == v[j, 1]
        elif kind == DIR_HU:
            assert h[j, 0] == wave(c.bc[W, 0])
            assert abs(u[j, 0] * h[j, 0] - wave(c.bc[W, 1])) < 1e-15
            assert abs(v[j, 0] * h[j, 0] - wave(c.bc[W, 2])) < 1e-15
        assert c.mask[j, -1] == DIR_Q
        assert h[j, -1] == h[j, -2]
        assert abs(u[j, -1] * h[j, -1] - wave(c.bc[E, 1])) < 1e-14


def test_solid_nodes_untouched_and_residual():
    c = inputs.random_case(20, 16, 41)
    s1 = oracle.run(c, 3)
    sol = c.mask == SOLID
    assert (s1[0][sol] == c.h0[sol]).all()
    s2 = oracle.run(c, 1, s1, n0=3)
    r, mass, umax = oracle.residual(c, s1, s2)
    fl = ~sol
    dq = np.concatenate([(s2[0] - s1[0])[fl], (s2[0] * s2[1] - s1[0] * s1[1])[fl],
                         (s2[0] * s2[2] - s1[0] * s1[2])[fl]])
    q = np.concatenate([s2[0][fl], (s2[0] * s2[1])[fl], (s2[0] * s2[2])[fl]])
    assert abs(r - np.linalg.norm(dq) / np.linalg.norm(q)) < 1e-14
    assert abs(mass - s2[0][fl].sum()) < 1e-12
    assert abs(umax - np.hypot(s2[1], s2[2])[fl].max()) < 1e-15


def test_interval_residual():
    """R7 over an interval of m steps, r_m = ||q^n - q^(n-m)|| / (m ||q^n||):
    its definition restated; per step (a constant change per step gives the
    same value for every m); zero for a state that alternates with period
    two and m = 2 (a rounding flicker is not a change of the solution)."""
    c = inputs.random_case(20, 16, 41)
    fl = c.mask != SOLID
    s0 = oracle.run(c, 3)
    s7 = oracle.run(c, 7, s0, n0=3)
    r, mass, umax = oracle.residual(c, s0, s7, interval=7)
    q = lambda s: np.concatenate([s[0][fl], (s[0] * s[1])[fl], (s[0] * s[2])[fl]])
    assert abs(r - np.linalg.norm(q(s7) - q(s0)) / (7 * np.linalg.norm(q(s7)))) < 1e-14
    assert abs(mass - s7[0][fl].sum()) < 1e-12
    # a constant change per step in (h, hu, hv)
    rng = np.random.default_rng(3)
    h0 = 1.0 + 0.1 * rng.random(c.mask.shape)
    hu0, hv0 = 0.1 * rng.random(c.mask.shape), 0.1 * rng.random(c.mask.shape)
    dh, dhu, dhv = (1e-6 * rng.standard_normal(c.mask.shape) for _ in range(3))

    def at(n):
        h = h0 + n * dh
        return h, (hu0 + n * dhu) / h, (hv0 + n * dhv) / h
    r1 = oracle.residual(c, at(99), at(100))[0]
    for m in (2, 5, 40):
        assert abs(oracle.residual(c, at(100 - m), at(100), interval=m)[0] - r1) <= 1e-9 * r1
    # period-two flicker
    a, b = at(0), at(1)
    assert oracle.residual(c, a, b)[0] > 0
    assert oracle.residual(c, a, a, interval=2)[0] == 0.0
