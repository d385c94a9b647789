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


@pytest.mark.parametrize("coll,lam,walls,storage,tol", [
    ("bgk", (0, 0, 0, 0), False, "f64", 1e-15),
    ("mrt", (0, 1.5, 1.3, 0.7), True, "f64", 1e-15),       # general MRT
    ("mrt", (0, 1.4, 0, 0), False, "f64", 1e-15),          # ghosts fully relaxed
    ("mrt", (0, 0, 0, 0), False, "f32", 1e-9),
    ("bgk", (0, 0, 0, 0), True, "f32", 1e-9),
    # no walls with 16-bit storage: reading the state back rounds the
    # bounced-back values of wall cells to 16 bits, the kernel does not
    ("bgk", (0, 0, 0, 0), False, "bf16dev", 1e-9),
])
def test_stress_epilogue_matches_oracle(coll, lam, walls, storage, tol):
    """The stress epilogue of the fused step (lbc_box_set_stress_output): the
    stress of the populations each step collides, element by element against
    oracle.lb.viscous_stress of the state before the step, and the step
    itself unchanged (bit for bit against a box without the epilogue)."""
    require_cuda()
    shape = (9, 10, 11)
    fbar0 = synth.random_populations(shape, seed=18, amp=2e-3)
    kw = dict(coll=coll, tau=0.85, lam=lam, walls=walls, uw=((0.01, 0, 0), (-0.02, 0.01, 0)),
              storage=storage, g=(1e-5, 0, 2e-6))
    box, sm = make_pair(shape, fbar0, **kw)
    twin, _ = make_pair(shape, fbar0, **kw)
    sig = box.stress_output()
    for nsteps in (1, 3):                          # the second call replays graphs
        f_before = box.get_populations()
        if nsteps > 1:
            box.step(nsteps - 1)
            twin.step(nsteps - 1)
            f_before = box.get_populations()
        box.step(1)
        twin.step(1)
        import torch
        torch.cuda.synchronize()
        got = sig.double().cpu().numpy()
        ref = OL.viscous_stress(f_before, sm.p)
        assert np.abs(ref).max() > 1e-6
        for k, (a, b) in enumerate(COMP):
            err = np.abs(got[k] - ref[a, b]).max()
            assert err <= tol, (k, err)
        assert np.array_equal(box.get_populations(), twin.get_populations())
    box.stress_output(False)
    box.close()
    twin.close()
