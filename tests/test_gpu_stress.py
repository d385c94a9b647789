"""Viscous stress (Eq. [viscstress]) read from the GPU state against the
oracle's, after a few steps from a random non-equilibrium state."""
import numpy as np
import pytest

import synth
from oracle import lb as OL
from tests.gpu_helpers import make_pair, require_cuda

pytestmark = pytest.mark.gpu

COMP = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)]


# The stress is a difference of second moments of size rho cs^2 = 1/3, so
# the bound is absolute on that scale: FP64 roundoff ~1e-16, FP32 storage
# ~1e-7 relative on the populations
@pytest.mark.parametrize("coll,lam,walls,storage,tol", [
    ("bgk", (0, 0, 0, 0), False, "f64", 1e-15),
    ("mrt", (0, 1.5, 0, 0), True, "f64", 1e-15),
    ("mrt", (0, 0, 1.2, 1.1), False, "f64", 1e-15),
    ("bgk", (0, 0, 0, 0), True, "f32", 1e-9),
])
def test_stress_matches_oracle(coll, lam, walls, storage, tol):
    require_cuda()
    shape = (9, 10, 11)
    fbar0 = synth.random_populations(shape, seed=8, amp=2e-3)
    box, sm = make_pair(shape, fbar0, coll=coll, tau=0.85, lam=lam, walls=walls,
                        uw=((0.01, 0, 0), (-0.02, 0.01, 0)), storage=storage, g=(1e-5, 0, 2e-6))
    for _ in range(4):
        sm.step()
    box.step(4)
    sig = box.get_stress()
    ref = OL.viscous_stress(sm.fbar, sm.p)
    assert np.abs(ref).max() > 1e-6                 # a non-trivial stress
    for k, (a, b) in enumerate(COMP):
        err = np.abs(sig[k] - ref[a, b]).max()
        assert err <= tol, (k, err)
