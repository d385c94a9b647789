"""Pins of the fluctuating collision (Sec. 3.2, Eq. [mrt-fluct]) in the oracle.

* The counter-based generator: the published Philox4x32-10 known-answer
  vectors (tests/golden/philox4x32_10_kat.txt), uniform outputs (chi-square), every output
  bit balanced, one flipped counter bit changes about half the output bits
  (ten rounds of mixing), distinct counters give distinct outputs, and the
  Box-Muller Gaussians have the normal's first four moments.
* Fluctuation-dissipation: in a periodic box at rest every moment settles
  at the variance mu rho0 b_k (k_B T per degree of freedom; the conserved
  ones scaled by 1 - 1/N since the box's totals are fixed), for BGK and for
  MRT with distinct eigenvalues, by the recombined step and by the literal
  two-half-step form; the amplitude as printed, sqrt(mu b lambda^2), does
  not give these variances.
* Without temperature the steps are the deterministic ones; with it, mass
  and momentum stay conserved to roundoff (the kicks act on non-conserved
  moments only).
"""
import numpy as np
import pytest

import synth
from oracle import fluct as F
from oracle import lattice as L
from oracle import lb as OL


def test_philox_known_answer_vectors():
    """The three published Philox4x32-10 known-answer vectors (counter, key ->
    output) of the Random123 distribution: a wrong round constant, key
    increment, word permutation or round count changes every output."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(t, 16) for t in row]
        ctr = [np.array([c], dtype=np.uint64) for c in v[:4]]
        out = F.philox4x32(ctr, (v[4], v[5]))
        assert [int(w[0]) for w in out] == v[6:10]
    # nine rounds is not Philox4x32-10
    v = [int(t, 16) for t in rows[2]]
    out9 = F.philox4x32([np.array([c], dtype=np.uint64) for c in v[:4]], (v[4], v[5]), rounds=9)
    assert [int(w[0]) for w in out9] != v[6:10]


def test_uniforms_are_uniform():
    u = F.uniforms(np.arange(40000), 7, 0, 0, 2024).ravel()
    assert u.min() > 0.0 and u.max() < 1.0
    counts, _ = np.histogram(u, bins=32, range=(0.0, 1.0))
    expect = u.size / 32
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 70.0, chi2                  # 31 degrees of freedom: 99.99 % below ~70
    assert abs(u.mean() - 0.5) < 5.0 * np.sqrt(1.0 / 12.0 / u.size)


def test_output_bits_are_balanced_and_mixed():
    n = 20000
    ctr = np.stack([np.arange(n), np.full(n, 3), np.zeros(n, int), np.zeros(n, int)]).astype(np.uint64)
    out = F.philox4x32(ctr, (11, 13))
    bits = (out[..., None] >> np.arange(32, dtype=np.uint32)) & 1
    freq = bits.mean(axis=1)                  # per word and bit
    assert np.abs(freq - 0.5).max() < 5.0 * 0.5 / np.sqrt(n)
    # avalanche: flip each counter bit of word 0; about 64 of 128 output bits change
    flips = []
    for b in range(32):
        c2 = ctr.copy()
        c2[0] = c2[0] ^ np.uint64(1 << b)
        diff = np.bitwise_xor(out, F.philox4x32(c2, (11, 13)))
        flips.append(np.unpackbits(diff.view(np.uint8)).reshape(-1).mean() * 128)
    assert abs(np.mean(flips) - 64.0) < 0.5
    # distinct counters and distinct keys give distinct outputs
    rows = {tuple(r) for r in out.T}
    assert len(rows) == n
    assert not np.any(np.all(F.philox4x32(ctr, (11, 14)) == out, axis=0))


def test_gaussian_moments():
    g = F.gaussians(np.arange(60000), 2, 5, 8, 99).ravel()
    n = g.size
    assert abs(g.mean()) < 5.0 / np.sqrt(n)
    assert abs(g.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert abs((g ** 3).mean()) < 5.0 * np.sqrt(15.0 / n)
    assert abs((g ** 4).mean() - 3.0) < 5.0 * np.sqrt(96.0 / n)


def test_draws_depend_on_every_counter_field():
    base = F.gaussians(np.arange(64), 5, 0, 19, 1)
    for args in ((5, 1, 19, 1), (6, 0, 19, 1), (5, 0, 19, 2)):
        other = F.gaussians(np.arange(64), *args)
        assert np.abs(other - base).min() > 0.0
    assert np.array_equal(F.gaussians(np.arange(64), 5, 0, 19, 1), base)


def _stationary_ratios(p, kT, steps, warm, literal=False, printed=False, n=6):
    """<m_k^2> / (mu rho0 b_k) per moment, averaged over cells and steps."""
    shape = (n, n, n)
    rho0 = p.rho0
    f = L.equilibrium(np.full(shape, rho0), np.zeros((3,) + shape))
    mu = kT / L.CS2
    acc = np.zeros(L.Q)
    cnt = 0
    for s in range(steps):
        if literal:
            f = F.step_literal_fluct(f, None, None, p, kT, seed=77, step=s)
        else:
            f = F.step_recombined_fluct(f, None, None, p, kT, seed=77, step=s, printed=printed)
        if s >= warm:
            m = np.tensordot(L.MRT_E, f - L.equilibrium(np.full(shape, rho0),
                                                        np.zeros((3,) + shape)),
                             axes=([1], [0]))
            acc += (m * m).reshape(L.Q, -1).mean(axis=1)
            cnt += 1
    ratio = acc / cnt / (mu * rho0 * L.MRT_B)
    cons = L.MRT_GROUP == 0
    ratio[cons] /= 1.0 - 1.0 / n ** 3          # the box's mass and momentum are fixed
    return ratio


@pytest.mark.parametrize("coll,tau,lam", [
    ("bgk", 0.8, (0, 0, 0, 0)),
    ("mrt", 0.8, (1.25, 1.4, 1.7, 0.6)),
])
def test_fluctuation_dissipation_recombined(coll, tau, lam):
    p = OL.LBParams(collision=coll, tau=tau, mrt_lambda=lam)
    r = _stationary_ratios(p, kT=1e-6, steps=1400, warm=200)
    noncons = L.MRT_GROUP != 0
    assert np.abs(r[noncons] - 1.0).max() < 0.03, r
    assert np.abs(r[~noncons] - 1.0).max() < 0.10, r


def test_fluctuation_dissipation_literal_half_steps():
    # C^1/2 needs 1 - lambda >= 0: tau >= 1, rates below 1
    p = OL.LBParams(collision="mrt", tau=1.25, mrt_lambda=(0.8, 0.6, 0.9, 0.5))
    r = _stationary_ratios(p, kT=1e-6, steps=1200, warm=200, literal=True)
    noncons = L.MRT_GROUP != 0
    assert np.abs(r[noncons] - 1.0).max() < 0.03, r
    assert np.abs(r[~noncons] - 1.0).max() < 0.10, r


def test_printed_amplitude_is_not_stationary():
    # shear and bulk rate 1.25: the printed amplitude puts lambda^2 /
    # (1 - gamma^2) = 1.67 times the variance the relaxation removes into the
    # stress modes; streaming shares the surplus with the other modes, so the
    # stress settles well above its equilibrium variance (but below 1.67)
    p = OL.LBParams(collision="mrt", tau=0.8)
    r = _stationary_ratios(p, kT=1e-6, steps=600, warm=100, printed=True)
    stress = (L.MRT_GROUP == 1) | (L.MRT_GROUP == 2)
    assert r[stress].min() > 1.15, r
    assert r[stress].max() < 1.5625 / 0.9375, r


def test_zero_temperature_is_the_deterministic_step():
    shape = (4, 5, 6)
    fbar = synth.random_populations(shape, seed=5, amp=1e-3)
    rng = np.random.default_rng(3)
    Fa, Fb = 1e-4 * rng.standard_normal((2, 3) + shape)
    for coll, tau, lam in (("bgk", 0.8, (0, 0, 0, 0)), ("mrt", 1.3, (0.7, 0.9, 1.0, 1.0))):
        p = OL.LBParams(collision=coll, tau=tau, mrt_lambda=lam, body_force=(1e-5, 0, -2e-5))
        a = F.step_recombined_fluct(fbar, Fa, Fb, p, 0.0, seed=1, step=0)
        assert np.abs(a - OL.step_recombined(fbar, Fa, Fb, p)).max() < 1e-15
        if tau >= 1.0:                         # the half collisions exist
            b = F.step_literal_fluct(fbar, Fa, Fb, p, 0.0, seed=1, step=0)
            assert np.abs(b - OL.step_literal(fbar, Fa, Fb, p)).max() < 1e-15
        else:
            with pytest.raises(ValueError):
                F.step_literal_fluct(fbar, Fa, Fb, p, 0.0, seed=1, step=0)


def test_kicks_conserve_mass_and_momentum():
    shape = (5, 5, 5)
    f = synth.random_populations(shape, seed=8, amp=1e-3)
    p = OL.LBParams(collision="mrt", tau=0.7, mrt_lambda=(0, 1.1, 1.5, 0.4))
    m0, j0 = L.density(f).sum(), L.momentum(f).reshape(3, -1).sum(axis=1)
    for s in range(20):
        f = F.step_recombined_fluct(f, None, None, p, kT=1e-4, seed=9, step=s)
    assert abs(L.density(f).sum() - m0) < 1e-12
    assert np.abs(L.momentum(f).reshape(3, -1).sum(axis=1) - j0).max() < 1e-12


# ------------------------------------------------------- particle noise zeta
# Pins of the random force of the force coupling (Sec. 5.2,
# Eq. [viscous-coupling], Eq. [modified-force]).  On a one-cell periodic box
# the trilinear stencil puts a particle on one node, and the fluid's kicks
# leave its momentum alone, so the relative velocity w = v - u follows the
# linear recurrence of the coupling alone.  Each Crank-Nicolson half step
# (x = (alpha + beta)/2) maps w -> (1 - x)/(1 + x) w + 2x/(gamma (1 + x)) zeta,
# and with <zeta^2> = 2 k_B T gamma / s its stationary variance is
#   <w_a^2> = k_B T (1/m + 1/rho),
# the canonical value of the two-body system, for any step; the explicit
# first-order step (y = gamma h (1/m + 1/rho)) gives k_B T (1/m + 1/rho)
# 2/(2 - y).  A wrong amplitude, a missing factor of two, the noise applied
# to one side only or with the wrong sign, or a noise repeated from step to
# step fails these (the last also breaks the momentum budget below).

def _one_cell_variance(order, mode, n, gamma, mass, steps, kind="fc"):
    from oracle import coupling as OC
    from oracle import sim as OS
    p = OL.LBParams(collision="mrt", tau=1.0)
    parts = OC.Particles(np.array([[0.3, 0.6, 0.2]]), vel=np.zeros((1, 3)),
                         mass=np.array([mass]))
    sm = OS.Sim((1, 1, 1), p, OS.CouplingParams(kind, order, "trilinear", gamma=gamma,
                                                substeps=n, mode=mode), parts)
    kT = 1e-4
    sm.set_thermal(kT, 77)
    w = []
    for _ in range(steps):
        sm.step()
        w.append(sm.parts.vel[0] - sm.fluid_velocity()[:, 0, 0, 0])
    w = np.array(w[100:])
    return (w * w).mean() / (kT * (1.0 / mass + 1.0)), sm


@pytest.mark.parametrize("order,mode,n,gamma,mass", [
    (2, "base", 1, 1.0, 1.0), (2, "base", 1, 3.0, 0.5), (2, "inside", 3, 2.0, 1.0),
    (2, "outside", 2, 1.5, 1.0), (1, "base", 1, 0.5, 1.0)])
def test_particle_noise_one_cell_equipartition(order, mode, n, gamma, mass):
    ratio, _ = _one_cell_variance(order, mode, n, gamma, mass, 4000)
    if order == 1:
        y = gamma * (1.0 / mass + 1.0)
        ratio /= 2.0 / (2.0 - y)
    # 4000 steps of a recurrence with memory g <= 1/9 per step: about 1.3 %
    # standard error on three components
    assert abs(ratio - 1.0) < 0.06, ratio


def test_original_ebf_noise_uses_its_friction():
    """The original EBF is force coupling with gamma = rho a^3 / h: its noise
    has that friction's amplitude (the one-cell variance is canonical)."""
    ratio, _ = _one_cell_variance(2, "base", 1, 0.0, 1.0, 4000, kind="ebf")
    assert abs(ratio - 1.0) < 0.06, ratio


@pytest.mark.parametrize("order,mode,n", [(2, "base", 1), (2, "inside", 2), (2, "outside", 2),
                                          (1, "base", 1)])
def test_thermal_coupled_momentum_budget(order, mode, n):
    """Fluid kicks act on non-conserved moments, and the fluid receives
    exactly -F^h including the particles' random force: fluid plus particle
    momentum grows by t g N to roundoff."""
    from oracle import coupling as OC
    from oracle import sim as OS
    shape = (6, 5, 7)
    rng = np.random.default_rng(4)
    M = 9
    g = np.array([1e-5, -2e-5, 3e-6])
    p = OL.LBParams(collision="mrt", tau=0.9, body_force=g)
    parts = OC.Particles(rng.uniform(0, 5, (M, 3)), vel=0.01 * rng.standard_normal((M, 3)),
                         mass=rng.uniform(0.5, 2.0, M))
    sm = OS.Sim(shape, p, OS.CouplingParams("fc", order, "trilinear", gamma=1.3, substeps=n,
                                            mode=mode), parts,
                fbar=synth.random_populations(shape, seed=2, amp=1e-3))
    sm.set_thermal(1e-4, 9)
    P0 = sm.total_momentum()
    for t in range(1, 6):
        sm.step()
        assert np.abs(sm.total_momentum() - P0 - t * g * np.prod(shape)).max() < 1e-13


def test_thermal_off_is_deterministic_and_counter_keeps_running():
    """kT = 0 gives the deterministic coupled step; switching off and on with
    the same seed continues the counter (no kick is repeated); a new seed
    restarts it."""
    from oracle import coupling as OC
    from oracle import sim as OS
    shape = (4, 4, 4)
    rng = np.random.default_rng(6)

    def make():
        parts = OC.Particles(rng.uniform(0, 4, (3, 3)), vel=np.zeros((3, 3)), mass=np.ones(3))
        return OS.Sim(shape, OL.LBParams(collision="bgk", tau=0.8),
                      OS.CouplingParams("fc", 2, "trilinear", gamma=1.0), parts)
    a, b = make(), make()
    b.parts.pos = a.parts.pos.copy()
    b.set_thermal(0.0, 3)
    a.step(); b.step()
    assert np.array_equal(a.fbar, b.fbar) and np.array_equal(a.parts.vel, b.parts.vel)
    b.set_thermal(1e-4, 3)
    b.step()
    assert b.tstep == 1
    b.set_thermal(0.0, 3)
    b.step()
    b.set_thermal(1e-4, 3)
    assert b.tstep == 1                 # continues: the next kicks are step 1's
    b.set_thermal(1e-4, 4)
    assert b.tstep == 0                 # a new seed restarts the sequence
