"""Thermal fluctuations of the fluid on the GPU (Eq. [mrt-fluct],
lbc_box_set_thermal) against the oracle (oracle/fluct.py).

Both sides draw the same Philox numbers for the same (cell, step, block)
counter, so a fluctuating step agrees with the oracle's step element by
element: FP64 storage to 1e-12 (the two sides' logarithm, square root and
sine / cosine differ by a few ulp), FP32 storage to 2e-7 (FP32 arithmetic on
deviations of 1e-3 w_i).  Several steps in one call replay captured graphs:
the device step counter must advance in them.  Over a long run the GPU's
own moments settle at the equilibrium variance mu rho0 b_k.
"""
import numpy as np
import pytest

import synth
from oracle import fluct as F
from oracle import lattice as L
from oracle import lb as OL
from tests.gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu

SEED = 0x123456789ABC


def _box(shape, storage, coll, tau, lam, g=(0.0, 0.0, 0.0)):
    from paper_1406_2211_gb300 import lbc
    nz, ny, nx = shape
    lat = lbc.lattice_desc(nx, ny, nz, collision=coll, tau=tau, mrt_lambda=lam,
                           body_force=g, storage=storage)
    return lbc.Box(lat, lbc.coupling_desc("none"), max_particles=0)


@pytest.mark.parametrize("storage,coll,tau,lam,tol", [
    ("f64", "mrt", 0.8, (1.25, 1.4, 1.7, 0.6), 1e-12),
    ("f64", "bgk", 0.7, (0, 0, 0, 0), 1e-12),
    ("f32", "mrt", 1.1, (0, 1.2, 1.5, 0.8), 2e-7),
])
def test_thermal_steps_match_oracle(storage, coll, tau, lam, tol):
    require_cuda()
    shape = (5, 6, 7)
    kT = 1e-4
    g = (1e-5, 0.0, -2e-5)
    box = _box(shape, storage, coll, tau, lam, g)
    box.set_populations(synth.random_populations(shape, seed=3, amp=1e-3))
    box.set_thermal(kT, SEED)
    p = OL.LBParams(collision=coll, tau=tau, mrt_lambda=lam, body_force=g)
    f = box.get_populations()
    step = 0
    for nsteps in (1, 1, 4):                     # the last call replays graphs
        box.step(nsteps)
        for _ in range(nsteps):
            f = F.step_recombined_fluct(f, None, None, p, kT, SEED, step)
            step += 1
        got = box.get_populations()
        assert np.abs(got - f).max() < tol, np.abs(got - f).max()
        f = got                                  # the next steps start from the stored state
    # off again: the deterministic step
    box.set_thermal(0.0)
    box.step(1)
    assert np.abs(box.get_populations() - OL.step_recombined(f, None, None, p)).max() < tol


def test_thermal_mode_variances_settle_at_equilibrium():
    require_cuda()
    n = 16
    shape = (n, n, n)
    kT = 1e-5
    box = _box(shape, "f32", "mrt", 0.8, (1.25, 1.4, 1.7, 0.6))
    box.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    box.set_thermal(kT, SEED)
    box.step(200)
    feq = L.equilibrium(np.ones(shape), np.zeros((3,) + shape))
    acc = np.zeros(L.Q)
    samples = 150
    for _ in range(samples):
        box.step(2)
        m = np.tensordot(L.MRT_E, box.get_populations() - feq, axes=([1], [0]))
        acc += (m * m).reshape(L.Q, -1).mean(axis=1)
    ratio = acc / samples / (kT / L.CS2 * L.MRT_B)
    cons = L.MRT_GROUP == 0
    ratio[cons] /= 1.0 - 1.0 / n ** 3
    assert np.abs(ratio[~cons] - 1.0).max() < 0.03, ratio
    assert np.abs(ratio[cons][1:] - 1.0).max() < 0.10, ratio   # momentum modes
    m0, P, st = box.invariants()
    assert st == 0 and abs(m0 - n ** 3) < 1e-6 * n ** 3 and np.abs(P).max() < 1e-6


def test_thermal_refusals():
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    box = _box((4, 4, 4), "f32", "bgk", 0.8, (0, 0, 0, 0))
    with pytest.raises(lbc.LBCError):
        box.set_thermal(-1.0)
    box16 = _box((4, 4, 4), "bf16dev", "bgk", 0.8, (0, 0, 0, 0))
    with pytest.raises(lbc.LBCError):
        box16.set_thermal(1e-4)
    box.set_thermal(1e-4, 5)
    batch = lbc.Batch(2)
    with pytest.raises(lbc.LBCError):
        batch.add(box, 3)
    batch.close()
