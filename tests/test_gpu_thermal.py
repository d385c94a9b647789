"""Thermal fluctuations of the fluid on the GPU (Eq. [mrt-fluct],
lbc_box_set_thermal) against the oracle (oracle/fluct.py).

Both sides draw the same Philox numbers for the same (cell, step, block)
counter, so a fluctuating step agrees with the oracle's step element by
element: FP64 storage to 1e-12 (the two sides' logarithm, square root and
sine / cosine differ by a few ulp), FP32 storage to 2e-7 (FP32 arithmetic on
deviations of 1e-3 w_i), 16-bit storage to that plus one 16-bit spacing of
each stored deviation.  The kicks run inside the fused LB kernel (single box
and batched); force-coupled particles get the random force zeta of
Eq. [modified-force] from their own counters.  Several steps in one call replay captured graphs:
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


# one 16-bit spacing of a stored value relative to its deviation from w_i rho0
# (FP16: 10 mantissa bits, BF16: 7), plus the FP32 bound
SPACING = {"f16dev": 2.0 ** -10, "bf16dev": 2.0 ** -7}


def _close(got, ref, storage, tol, nsteps=1):
    """Bound of one call of nsteps steps: tol, plus for 16-bit storage (each
    stored value rounded stochastically to one of its two neighbours) one
    16-bit spacing of each element's deviation after one step; over several
    steps the rounding errors of large deviations reach every population
    through the density and momentum, so there the bound is nsteps x 4
    spacings of the largest deviation."""
    w0 = L.W.reshape((L.Q,) + (1,) * (ref.ndim - 1))
    sp = SPACING.get(storage, 0.0)
    dev = np.abs(ref - w0)
    bound = tol + (sp * dev if nsteps == 1 else 4.0 * nsteps * sp * dev.max())
    return float((np.abs(got - ref) / bound).max())


@pytest.mark.parametrize("storage,coll,tau,lam,tol", [
    ("f64", "mrt", 0.8, (1.25, 1.4, 1.7, 0.6), 1e-12),
    ("f64", "bgk", 0.7, (0, 0, 0, 0), 1e-12),
    ("f64", "mrt", 0.9, (0, 0, 0, 0), 1e-12),          # ghosts fully relaxed
    ("f32", "mrt", 1.1, (0, 1.2, 1.5, 0.8), 2e-7),
    ("f16dev", "mrt", 0.8, (0, 0, 0, 0), 2e-7),
    ("bf16dev", "bgk", 0.9, (0, 0, 0, 0), 2e-7),
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
        assert _close(got, f, storage, tol, nsteps) <= 1.0
        f = got                                  # the next steps start from the stored state
    # off again: the deterministic step
    box.set_thermal(0.0)
    box.step(1)
    assert _close(box.get_populations(), OL.step_recombined(f, None, None, p), storage, tol) <= 1.0


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


def test_printed_amplitude_option_matches_oracle():
    """LBC_OPT_THERMAL_AMPLITUDE = 1: the amplitude as printed in
    Eq. [mrt-fluct], sqrt(mu b_k lambda_k^2), on the GPU and in the oracle."""
    require_cuda()
    shape = (4, 5, 6)
    kT = 1e-4
    p = OL.LBParams(collision="mrt", tau=0.8, mrt_lambda=(0, 1.3, 1.6, 0.7))
    box = _box(shape, "f64", "mrt", 0.8, (0, 1.3, 1.6, 0.7))
    box.set_populations(synth.random_populations(shape, seed=5, amp=1e-3))
    f = box.get_populations()
    box.set_thermal(kT, SEED, printed_amplitude=True)
    box.step(3)
    for s in range(3):
        f = F.step_recombined_fluct(f, None, None, p, kT, SEED, s, printed=True)
    assert np.abs(box.get_populations() - f).max() < 1e-12


def test_counter_continues_when_switched_off_and_on():
    """Switching the fluctuations off and on with the same seed continues the
    step counter (steps in between do not advance it): the kicks of the
    steps after that are those of counter values 2, 3, not 0, 1 again.  A new
    seed restarts at 0."""
    require_cuda()
    shape = (4, 4, 5)
    kT = 1e-4
    p = OL.LBParams(collision="bgk", tau=0.8)
    box = _box(shape, "f64", "bgk", 0.8, (0, 0, 0, 0))
    box.set_populations(synth.random_populations(shape, seed=6, amp=1e-3))
    f = box.get_populations()
    box.set_thermal(kT, SEED)
    box.step(2)                                  # counter 0, 1
    for s in range(2):
        f = F.step_recombined_fluct(f, None, None, p, kT, SEED, s)
    box.set_thermal(0.0)
    box.step(3)                                  # plain steps, odd count: parity flips
    for _ in range(3):
        f = OL.step_recombined(f, None, None, p)
    box.set_thermal(kT, SEED)
    box.step(2)                                  # counter 2, 3
    for s in (2, 3):
        f = F.step_recombined_fluct(f, None, None, p, kT, SEED, s)
    assert np.abs(box.get_populations() - f).max() < 1e-12
    box.set_thermal(kT, SEED + 1)
    box.step(1)
    f = F.step_recombined_fluct(f, None, None, p, kT, SEED + 1, 0)
    assert np.abs(box.get_populations() - f).max() < 1e-12


@pytest.mark.parametrize("kind,order,split,n,stencil", [
    ("fc", 2, "base", 1, "trilinear"),
    ("fc", 2, "inside", 2, "trilinear"),
    ("fc", 2, "outside", 2, "peskin4"),
    ("fc", 1, "base", 1, "trilinear"),
    ("ebf", 2, "base", 1, "peskin4"),
    ("mebf", 2, "base", 1, "trilinear"),
    ("ibm", 2, "base", 1, "peskin4"),
])
def test_thermal_coupled_steps_match_oracle(kind, order, split, n, stencil):
    """Thermal fluid plus the particles' random force zeta (FC, original EBF;
    none for the modified EBF; IBM markers have no velocity): the same Philox
    counters on both sides, FP64 storage, trajectories to 1e-11 over steps
    that include graph replays."""
    require_cuda()
    from tests.gpu_helpers import make_pair
    from oracle import coupling as OC
    shape = (8, 9, 10)
    rng = np.random.default_rng(13)
    M = 12
    parts = dict(pos=rng.uniform(0, 8, (M, 3)), vel=0.01 * rng.standard_normal((M, 3)),
                 mass=rng.uniform(0.5, 2.0, M))
    if kind == "ibm":
        parts = dict(pos=parts["pos"], bonds=np.array([[0, 1], [1, 2]]), bond_k=0.02,
                     bond_r0=1.2)
    box, sm = make_pair(shape, synth.random_populations(shape, seed=12, amp=1e-3),
                        coll="mrt", tau=0.9, g=(1e-5, 0, 0), storage="f64", kind=kind,
                        order=order, stencil=stencil, gamma=1.4, split=split, n=n, parts=parts)
    kT = 1e-5
    box.set_thermal(kT, SEED)
    sm.set_thermal(kT, SEED)
    for nsteps in (1, 4):
        box.step(nsteps)
        for _ in range(nsteps):
            sm.step()
        pos, vel, _ = box.get_particles()
        d = OC.min_image(pos - sm.parts.pos, shape, False)
        assert np.abs(d).max() < 1e-11, np.abs(d).max()
        if kind != "ibm":
            assert np.abs(vel - sm.parts.vel).max() < 1e-11
    _, u = box.get_fields()
    ref = sm.fluid_velocity()
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-10
    box.close()


def test_thermal_box_in_batch_equals_alone():
    """Thermal boxes join batches: their LB steps run in the batched thermal
    launch (their own group) with their own counters; a member in a mixed
    batch equals the same box advanced alone in a batch, bit for bit."""
    require_cuda()
    from paper_1406_2211_gb300 import lbc

    def member(seed, thermal):
        nz, ny, nx = 6, 7, 9
        lat = lbc.lattice_desc(nx, ny, nz, collision="bgk", tau=0.8, storage="f32")
        cpl = lbc.coupling_desc("fc", 2, "trilinear", gamma=1.0)
        b = lbc.Box(lat, cpl, max_particles=4)
        b.set_populations(synth.random_populations((nz, ny, nx), seed=seed, amp=1e-3))
        r = np.random.default_rng(seed)
        b.set_particles(r.uniform(0, 6, (4, 3)), vel=np.zeros((4, 3)), mass=1.0)
        if thermal:
            b.set_thermal(1e-4, SEED + seed)
        return b

    results = []
    for mix in (False, True):
        batch = lbc.Batch(4)
        a = member(1, True)
        others = [member(2, False), member(3, True)] if mix else []
        batch.add(a, 7)
        for o in others:
            batch.add(o, 7)
        while len(batch) > 0:
            batch.advance(3)
        results.append((a.get_populations(), a.get_particles()[1]))
        for b in [a] + others:
            b.close()
        batch.close()
    assert np.array_equal(results[0][0], results[1][0])
    assert np.array_equal(results[0][1], results[1][1])


def test_thermal_refusals():
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    box = _box((4, 4, 4), "f32", "bgk", 0.8, (0, 0, 0, 0))
    with pytest.raises(lbc.LBCError):
        box.set_thermal(-1.0)
    with pytest.raises(lbc.LBCError):
        box.set_thermal(float("nan"))
    # the stress epilogue and the thermal step are separate variants
    box.stress_output()
    with pytest.raises(lbc.LBCError) as e:
        box.set_thermal(1e-4, 5)
    assert e.value.status == lbc.LBC_ERR_UNSUPPORTED
    box.stress_output(False)
    box.set_thermal(1e-4, 5)
    with pytest.raises(lbc.LBCError):
        box.stress_output()
    # a member's thermal state changes only outside the batch
    batch = lbc.Batch(2)
    batch.add(box, 3)
    with pytest.raises(lbc.LBCError) as e:
        box.set_thermal(0.0)
    assert e.value.status == lbc.LBC_ERR_STATE
    batch.close()
