"""Pins of the oracle's viscous stress, Eq. [viscstress] (first line).

Between halfway-bounce-back walls moving at -/+U the steady lattice flow is
exactly linear (Couette), and the stress must equal the Newtonian value
-rho0 nu du/dz with nu = (tau - 1/2)/3 for the shear rate of the collision
(BGK, and MRT with a bulk rate different from the shear rate).  The
Couette flow carries a stress only in the xz component pair; a state at
equilibrium carries none."""
import numpy as np
import pytest

import synth
from oracle import lattice as L
from oracle import lb as OL


def test_equilibrium_has_no_viscous_stress():
    rng = np.random.default_rng(1)
    shape = (4, 5, 6)
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    u = 0.02 * rng.standard_normal((3,) + shape)
    for p in (OL.LBParams(collision="bgk", tau=0.9),
              OL.LBParams(collision="mrt", tau=0.9, mrt_lambda=(0, 1.4, 0, 0))):
        s = OL.viscous_stress(L.equilibrium(rho, u), p)
        assert np.abs(s).max() < 1e-15      # roundoff of sums of O(1/3) terms


@pytest.mark.parametrize("coll,tau,lam", [("bgk", 0.8, (0, 0, 0, 0)), ("bgk", 1.3, (0, 0, 0, 0)),
                                          ("mrt", 0.9, (0, 1.6, 0, 0))])
def test_steady_couette_stress(coll, tau, lam):
    nz, U = 8, 0.01
    p = OL.LBParams(collision=coll, tau=tau, mrt_lambda=lam, walls=True,
                    u_bot=(-U, 0, 0), u_top=(U, 0, 0))
    shape = (nz, 1, 1)
    z = np.arange(nz)
    u = np.zeros((3,) + shape)
    u[0] = (-U + 2 * U * (z + 0.5) / nz)[:, None, None]
    f = L.equilibrium(np.ones(shape), u)
    for _ in range(2500):
        f = OL.step_recombined(f, None, None, p)
    s = OL.viscous_stress(f, p)
    nu = (tau - 0.5) / 3.0
    expect = -1.0 * nu * 2.0 * U / nz
    assert np.abs(s[0, 2] - expect).max() < 1e-12 * abs(expect)
    assert np.abs(s[2, 0] - expect).max() < 1e-12 * abs(expect)
    assert np.abs(s[0, 1]).max() < 1e-18 and np.abs(s[1, 2]).max() < 1e-18


def test_stress_is_symmetric_and_uses_its_own_moments():
    p = OL.LBParams(collision="mrt", tau=0.75)
    f = synth.random_populations((3, 4, 5), seed=6, amp=1e-2)
    s = OL.viscous_stress(f, p)
    assert np.abs(s - np.swapaxes(s, 0, 1)).max() < 1e-18
    # adding an equilibrium shift of the velocity (a force half step)
    # changes fbar but not fbar - f^eq
    rho = L.density(f)
    u = L.momentum(f) / rho
    g = L.equilibrium(rho, u + 0.003) - L.equilibrium(rho, u)
    assert np.abs(OL.viscous_stress(f + g, p) - s).max() < 1e-15
