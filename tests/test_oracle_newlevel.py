"""Pins of the oracle's new-level hbar variant (Eq. h-bar as written:
hbar = (h(x, t + dt) + h(y, t)) / 2 on the link from y = x - c_a into x).
The oracle solves the linear equation for h(x, t + dt) node by node; here
the defining sums of Eqs. Mac.lb.6 / Mac.lb.7 are evaluated directly with
that hbar, link by link, and must return the same h and h u."""
import numpy as np
import pytest

import inputs
import oracle
from inputs import BOUNCEBACK, FLUID, PERIODIC, SOLID

CX = [0, 1, 1, 0, -1, -1, -1, 0, 1]
CY = [0, 0, 1, 1, 1, 0, -1, -1, -1]


def direct_sums(case, h, u, v, h1):
    """Eq. Mac.lb.6 / 7 at every fluid node with hbar_a = (h1(x) + h(y))/2
    (periodic and bounce-back edges, solid nodes bounce back)."""
    e, g, dt = case.e, case.g, case.dt
    ny, nx = h.shape
    Sh, Sx, Sy = (np.zeros_like(h) for _ in range(3))
    for j in range(ny):
        for i in range(nx):
            if case.mask[j, i] == SOLID:
                continue
            fx = oracle.feq(h[j, i], u[j, i], v[j, i], e, g)
            Fx = oracle.force(case, h[j, i], u[j, i], v[j, i])
            acc = np.array([fx[0], 0.0, 0.0])
            for a in range(1, 9):
                ii, jj = i - CX[a], j - CY[a]
                bounce = False
                for idx, n, lo, hi in ((0, nx, 0, 1), (1, ny, 2, 3)):
                    k = ii if idx == 0 else jj
                    if k < 0 or k >= n:
                        kind = case.edges[lo if k < 0 else hi]
                        if kind == BOUNCEBACK:
                            bounce = True
                        elif idx == 0:
                            ii %= nx
                        else:
                            jj %= ny
                if not bounce and case.mask[jj, ii] == SOLID:
                    bounce = True
                if bounce:
                    fa = fx[(a + 3) % 8 + 1]
                else:
                    fs = oracle.feq(h[jj, ii], u[jj, ii], v[jj, ii], e, g)
                    Fs = oracle.force(case, h[jj, ii], u[jj, ii], v[jj, ii])
                    C = 1 / 3 if a % 2 else 1 / 12
                    hbar = 0.5 * (h1[j, i] + h[jj, ii])
                    fa = fs[a] - g * hbar / e ** 2 * C * (case.zb[j, i] - case.zb[jj, ii])
                    fa += dt / e ** 2 * C * (e * CX[a] * 0.5 * (Fx[0] + Fs[0]) + e * CY[a] * 0.5 * (Fx[1] + Fs[1]))
                acc += fa * np.array([1.0, e * CX[a], e * CY[a]])
            Sh[j, i], Sx[j, i], Sy[j, i] = acc
    return Sh, Sx, Sy


@pytest.mark.parametrize("edges", [(PERIODIC,) * 4, (BOUNCEBACK,) * 4, (PERIODIC, PERIODIC, BOUNCEBACK, BOUNCEBACK)])
def test_new_level_step_solves_its_defining_sums(edges):
    case = inputs.random_case(14, 11, 9, edges=edges, dirichlet=False)
    case.mask = np.where(case.mask == SOLID, SOLID, FLUID).astype(np.uint8)
    h, u, v = oracle.run(case, 3)               # a moving state
    h1, u1, v1 = oracle.run_newlevel(case, 1, (h, u, v), n0=3)
    Sh, Sx, Sy = direct_sums(case, h, u, v, h1)
    live = case.mask != SOLID
    assert np.abs(h1 - Sh)[live].max() <= 1e-13
    assert np.abs(h1 * u1 - Sx)[live].max() <= 1e-13 and np.abs(h1 * v1 - Sy)[live].max() <= 1e-13


def test_lake_at_rest_and_flat_bed():
    case = inputs.random_case(30, 24, 2, dirichlet=False)
    case.wind_u = case.wind_v = 0.0
    case.omega = 0.0
    rest = case.copy()
    D = rest.h_ref - rest.zb
    rest.h0 = np.where(rest.mask == SOLID, 0.0, D)
    rest.u0 = np.zeros_like(D)
    rest.v0 = np.zeros_like(D)
    h, u, v = oracle.run_newlevel(rest, 50)
    live = rest.mask != SOLID
    assert np.abs(h - D)[live].max() <= 1e-13 and np.abs(u)[live].max() <= 1e-13   # round-off only
    flat = case.copy()
    flat.zb = np.zeros_like(flat.zb)
    a = oracle.run_newlevel(flat, 20)
    b = oracle.run(flat, 20)
    assert all(np.abs(x - y)[live].max() <= 1e-14 for x, y in zip(a, b))
    # and on the sloped bed the two levels differ
    c = oracle.run_newlevel(case, 20)
    d = oracle.run(case, 20)
    assert np.abs(c[0] - d[0])[live].max() > 1e-9


def test_mass_exact_at_the_old_level_only():
    """The old-level bed terms of opposite links cancel in pairs (exact mass
    in a closed basin); with the new level they do not, and a closed basin
    gains or loses mass at the truncation level."""
    case = inputs.random_case(40, 30, 3, edges=(BOUNCEBACK,) * 4, dirichlet=False)
    live = case.mask != SOLID
    m0 = case.h0[live].sum()
    old = oracle.run(case, 200)[0][live].sum()
    new = oracle.run_newlevel(case, 200)[0][live].sum()
    assert abs(old - m0) <= 1e-13 * m0
    assert 1e-12 * m0 < abs(new - m0) < 1e-5 * m0
