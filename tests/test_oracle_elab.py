"""Pins of the oracle's distribution form with a general relaxation time
(eLABSWE, Eq. lb.1): at tau = 1 it is the MacLABSWE step (Eq. Mac.lb.3),
its shear viscosity is e^2 dt (2 tau - 1) / 6 (Eq. viscosity), and it
conserves mass exactly in a closed basin."""
import math

import numpy as np
import pytest

import inputs
import oracle
from inputs import BOUNCEBACK, FLUID, NOSLIP, PERIODIC, SOLID, SPECULAR


def no_walls(case):
    """The case with its no-slip border nodes made plain fluid (the
    distribution form has no no-slip override) and no Dirichlet data."""
    c = case.copy()
    c.mask = np.where(c.mask == NOSLIP, FLUID, c.mask).astype(np.uint8)
    return c


@pytest.mark.parametrize("edges", [(PERIODIC,) * 4, (BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR),
                                   (SPECULAR, SPECULAR, PERIODIC, PERIODIC)])
def test_tau_one_is_the_macroscopic_step(edges):
    case = no_walls(inputs.random_case(23, 17, 4, edges=edges, dirichlet=False))
    assert (case.mask == SOLID).any()
    want = oracle.run(case, 5)
    h, u, v, _ = oracle.elab_run(case, 1.0, 5)
    live = case.mask != SOLID
    for a, b in zip((h, u, v), want):
        assert np.allclose(a[live], b[live], rtol=0, atol=1e-13 * max(1.0, np.abs(b[live]).max()))


def shear_decay_error(tau, ny):
    """Relative error of the measured decay rate of u = U sin(2 pi y / ny)
    against nu k^2 with nu = e^2 dt (2 tau - 1) / 6."""
    e, dx = 12.0, 1.0
    z = np.zeros((ny, 4))
    yy = np.arange(ny)[:, None] * np.ones((1, 4))
    c = inputs.Case("shear", 4, ny, dx, e * dx / 6.0, z, np.full((ny, 4), FLUID, np.uint8), np.ones((ny, 4)),
                    1e-3 * np.sin(2 * math.pi * yy / ny), z.copy(), edges=(PERIODIC,) * 4)
    dt = dx / e
    n1, n2 = 200, 1200
    _, u1, _, f = oracle.elab_run(c, tau, n1)
    _, u2, _, _ = oracle.elab_run(c, tau, n2 - n1, f)
    rate = math.log(np.abs(u1).max() / np.abs(u2).max()) / ((n2 - n1) * dt)
    nu = e * e * dt * (2 * tau - 1) / 6.0
    k = 2 * math.pi / (ny * dx)
    return rate / (nu * k * k) - 1.0


@pytest.mark.parametrize("tau", [0.8, 1.5])
def test_shear_wave_viscosity(tau):
    """Eq. viscosity: the decay rate tends to nu k^2 with a second-order
    lattice error (a quarter when the wave is resolved twice as finely)."""
    e64, e128 = shear_decay_error(tau, 64), shear_decay_error(tau, 128)
    assert abs(e128) <= 1e-3
    assert 3.5 <= e64 / e128 <= 4.5, (e64, e128)


@pytest.mark.parametrize("tau", [0.7, 1.3])
def test_mass_is_conserved(tau):
    case = no_walls(inputs.random_case(31, 29, 7, edges=(BOUNCEBACK, BOUNCEBACK, SPECULAR, SPECULAR),
                                       dirichlet=False))
    live = case.mask != SOLID
    m0 = case.h0[live].sum()
    h, _, _, _ = oracle.elab_run(case, tau, 300)
    assert abs(h[live].sum() - m0) <= 1e-13 * m0


def test_rejects_no_slip_nodes():
    case = inputs.random_case(23, 17, 4, dirichlet=False)
    assert (case.mask == NOSLIP).any()
    with pytest.raises(ValueError):
        oracle.elab_run(case, 1.2, 1)
