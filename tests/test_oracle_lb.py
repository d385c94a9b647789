"""Pins for oracle/lb.py: step forms, collision algebra, hydrodynamic limits.

Closed forms used (none is a retyping of the oracle's formulas):
  * literal CSC (O1) == recombined step (O2) to roundoff where O1 exists
    (Sec. 4: the CSC scheme is the standard scheme with collision
    (1 - Lambda_1/2)^2, Eq. [force-transformation]);
  * C^1/2 C^1/2 = C exactly with 1 - lambda_1/2 = sqrt(1 - lambda) (Sec. 3.2);
  * shear-wave decay gives nu = (tau - 1/2)/3 (Navier-Stokes limit, k -> 0);
  * the (1 + C)/2 half collision changes the viscosity (Sec. 4, negative test);
  * body-force Poiseuille flow between halfway bounce-back walls: parabolic
    profile with the closed-form BGK slip (16(tau-1/2)^2 - 3)/24 g/(rho nu),
    second difference -g/(rho nu) for any collision model;
  * moving-wall Couette flow: exactly linear profile.
"""
import numpy as np
import pytest

from oracle import lattice as L
from oracle import lb
from oracle import sim as S


def _random_state(rng, shape, amp=1e-3):
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    u = 0.02 * rng.standard_normal((3,) + shape)
    f = L.equilibrium(rho, u) + amp * rng.standard_normal((19,) + shape)
    return f


@pytest.mark.parametrize("coll,tau,lam", [
    ("bgk", 1.0, (0, 0, 0, 0)),
    ("bgk", 1.7, (0, 0, 0, 0)),
    ("mrt", 1.2, (0, 0.8, 0.9, 0.6)),
    ("mrt", 1.0, (0, 0, 0, 0)),
])
@pytest.mark.parametrize("walls", [False, True])
def test_literal_equals_recombined(rng, coll, tau, lam, walls):
    shape = (5, 4, 6)
    f = _random_state(rng, shape)
    Fa = 1e-3 * rng.standard_normal((3,) + shape)
    Fb = 1e-3 * rng.standard_normal((3,) + shape)
    p = lb.LBParams(collision=coll, tau=tau, mrt_lambda=lam,
                    body_force=(1e-4, -2e-4, 3e-5), walls=walls,
                    u_bot=(0.01, 0.0, 0.0), u_top=(-0.02, 0.005, 0.0))
    a = lb.step_literal(f, Fa, Fb, p)
    b = lb.step_recombined(f, Fa, Fb, p)
    assert np.abs(a - b).max() < 1e-15


def test_half_collisions_compose_to_full(rng):
    shape = (3, 3, 3)
    f = _random_state(rng, shape)
    for coll, lam in (("bgk", (0, 0, 0, 0)), ("mrt", (0, 0.7, 0.8, 0.5))):
        p = lb.LBParams(collision=coll, tau=1.4, mrt_lambda=lam)
        twice = lb.relax(lb.relax(f, p.gamma_half(), p), p.gamma_half(), p)
        once = lb.relax(f, p.gamma_full(), p)
        assert np.abs(twice - once).max() < 1e-16


def test_mrt_with_equal_rates_is_bgk(rng):
    shape = (4, 3, 5)
    f = _random_state(rng, shape)
    Fa = 1e-3 * rng.standard_normal((3,) + shape)
    Fb = 1e-3 * rng.standard_normal((3,) + shape)
    tau = 0.7
    pb = lb.LBParams(collision="bgk", tau=tau, body_force=(1e-5, 0, 0))
    pm = lb.LBParams(collision="mrt", tau=tau, mrt_lambda=(1 / tau,) * 4,
                     body_force=(1e-5, 0, 0))
    a = lb.step_recombined(f, Fa, Fb, pb)
    b = lb.step_recombined(f, Fa, Fb, pm)
    assert np.abs(a - b).max() < 1e-15


@pytest.mark.parametrize("walls", [False, True])
def test_step_conserves_mass_and_adds_force_impulse(rng, walls):
    shape = (6, 4, 5)
    f = _random_state(rng, shape)
    Fa = 1e-3 * rng.standard_normal((3,) + shape)
    Fb = 1e-3 * rng.standard_normal((3,) + shape)
    g = np.array([1e-4, 2e-4, -3e-4])
    p = lb.LBParams(collision="mrt", tau=0.9, body_force=g, walls=walls)
    b = lb.step_recombined(f, Fa, Fb, p)
    assert abs(L.density(b).sum() - L.density(f).sum()) < 1e-12
    if not walls:
        dj = L.momentum(b).reshape(3, -1).sum(1) - L.momentum(f).reshape(3, -1).sum(1)
        expect = 0.5 * (Fa + Fb).reshape(3, -1).sum(1) + g * np.prod(shape)
        assert np.abs(dj - expect).max() < 1e-14


def _shear_wave_nu(stepper, L_, tau, nsteps=60):
    """Per-step decay of u_y = U sin(2 pi x / L) -> nu_eff = -ln(ratio)/k^2."""
    shape = (1, 1, L_)
    x = np.arange(L_)
    k = 2 * np.pi / L_
    u = np.zeros((3,) + shape)
    u[1, 0, 0, :] = 1e-6 * np.sin(k * x)
    f = L.equilibrium(np.ones(shape), u)
    amps = []
    for _ in range(nsteps):
        f = stepper(f)
        uy = (L.momentum(f) / L.density(f))[1, 0, 0, :]
        amps.append((uy * np.sin(k * x)).sum() * 2 / L_)
    ratio = amps[-1] / amps[-2]
    return -np.log(ratio) / k ** 2


@pytest.mark.parametrize("coll,tau,lam_s", [("bgk", 0.8, 0), ("bgk", 1.6, 0),
                                            ("bgk", 0.7, 0), ("mrt", 1.0, 1.3)])
def test_shear_wave_viscosity(coll, tau, lam_s):
    """nu = (1/lambda_s - 1/2)/3 after Richardson extrapolation in k^2."""
    p = lb.LBParams(collision=coll, tau=tau, mrt_lambda=(lam_s, 0.9, 0.8, 0.7))
    zero = np.zeros((3, 1, 1, 1))
    step = lambda f: lb.step_recombined(f, zero, zero, p)
    L1, L2 = 48, 96
    n1 = _shear_wave_nu(step, L1, tau)
    n2 = _shear_wave_nu(step, L2, tau)
    k1, k2 = (2 * np.pi / L1) ** 2, (2 * np.pi / L2) ** 2
    nu0 = (n1 * k2 - n2 * k1) / (k2 - k1)
    # the remainder is O(k^4): 3e-4 at L = 24/48 and tau = 1.6, 16x less here
    lam = lam_s if lam_s else 1.0 / tau
    expect = (1.0 / lam - 0.5) / 3.0
    assert abs(nu0 / expect - 1.0) < 5e-5


def test_approximate_half_collision_changes_viscosity():
    """With C^1/2 = (1 + C)/2 the shear eigenvalue becomes ((1 + gamma)/2)^2,
    so nu is not (tau - 1/2)/3 (Sec. 4, Eq. [half-col-approx])."""
    tau = 0.8
    p = lb.LBParams(collision="bgk", tau=tau)
    step = lambda f: lb.step_literal_approx_half(f, p)
    L1, L2 = 48, 96
    n1 = _shear_wave_nu(step, L1, tau)
    n2 = _shear_wave_nu(step, L2, tau)
    k1, k2 = (2 * np.pi / L1) ** 2, (2 * np.pi / L2) ** 2
    nu0 = (n1 * k2 - n2 * k1) / (k2 - k1)
    gam = 1.0 - 1.0 / tau
    lam_eff = 1.0 - ((1.0 + gam) / 2.0) ** 2
    assert abs(nu0 / ((tau - 0.5) / 3.0) - 1.0) > 0.5
    assert abs(nu0 / ((1.0 / lam_eff - 0.5) / 3.0) - 1.0) < 5e-5


def _channel(p, nz, g, nsteps):
    """Steady flow in a 1 x 1 x nz channel, started from the parabola."""
    nu = (p.tau - 0.5) / 3.0
    z = np.arange(nz)
    u0 = np.zeros((3, nz, 1, 1))
    u0[0, :, 0, 0] = g / (2 * nu) * ((nz / 2) ** 2 - (z - (nz - 1) / 2) ** 2)
    f = L.equilibrium(np.ones((nz, 1, 1)), u0)
    sm = S.Sim((nz, 1, 1), p, fbar=f)
    for _ in range(nsteps):
        sm.step()
    return sm.fluid_velocity()[0, :, 0, 0]


@pytest.mark.parametrize("tau", [0.8, 0.5 + np.sqrt(3.0 / 16.0), 1.3])
def test_poiseuille_closed_form(tau):
    nz, g = 8, 1e-5
    p = lb.LBParams(collision="bgk", tau=tau, walls=True, body_force=(g, 0, 0))
    u = _channel(p, nz, g, 4000)
    nu = (tau - 0.5) / 3.0
    z = np.arange(nz)
    para = g / (2 * nu) * ((nz / 2) ** 2 - (z - (nz - 1) / 2) ** 2)
    slip = (16 * (tau - 0.5) ** 2 - 3) / 24 * g / nu
    assert np.abs(u - para - slip).max() / u.max() < 1e-10
    if abs(tau - (0.5 + np.sqrt(3.0 / 16.0))) < 1e-12:
        assert abs(slip) < 1e-20
        assert np.abs(u - para).max() / u.max() < 1e-10


def test_poiseuille_mrt_second_difference():
    # g small enough that the O(u^2) ghost-mode corrections (1e-8 relative at
    # g = 1e-5 with ghost rates != 1) stay below the tolerance
    nz, g, tau = 10, 1e-8, 1.0
    p = lb.LBParams(collision="mrt", tau=tau, mrt_lambda=(0, 0.7, 0.8, 0.9),
                    walls=True, body_force=(g, 0, 0))
    u = _channel(p, nz, g, 4000)
    nu = (tau - 0.5) / 3.0
    d2 = u[2:] - 2 * u[1:-1] + u[:-2]
    assert np.abs(d2 / (-g / nu) - 1.0).max() < 1e-8


def test_couette_linear():
    nz, tau = 8, 0.9
    ub, ut = -0.01, 0.02
    p = lb.LBParams(collision="bgk", tau=tau, walls=True,
                    u_bot=(ub, 0, 0), u_top=(ut, 0, 0))
    z = np.arange(nz)
    exact = ub + (ut - ub) * (z + 0.5) / nz
    u0 = np.zeros((3, nz, 1, 1))
    u0[0, :, 0, 0] = exact
    sm = S.Sim((nz, 1, 1), p, fbar=L.equilibrium(np.ones((nz, 1, 1)), u0))
    for _ in range(3000):
        sm.step()
    u = sm.fluid_velocity()[0, :, 0, 0]
    assert np.abs(u - exact).max() < 1e-10 * abs(ut)


# ---------------------------------------------------------------- MRT groups
# The pins above see only the shear rate (shear wave, Couette stress, the
# Poiseuille second difference) or compare MRT with itself (equal rates ==
# BGK).  The two tests below pin which moments the oracle relaxes with the
# bulk rate and with each ghost rate, against facts that do not depend on
# the oracle's basis or group table:
#   * sound attenuation.  Linearised Navier-Stokes with shear viscosity nu
#     and bulk viscosity nu_b damps a longitudinal wave of wavenumber k at
#     the rate Gamma = k^2 (2 nu / 3 + nu_b / 2).  For a lattice-Boltzmann
#     fluid whose stress trace relaxes at lambda_b and whose traceless stress
#     relaxes at lambda_s, nu = cs2 (1/lambda_s - 1/2) and
#     nu_b = (2/3) cs2 (1/lambda_b - 1/2) (Duenweg, Schiller and Ladd, Phys.
#     Rev. E 76, 036704 (2007), eta_b = rho cs2 h (1 + gamma_b)/(3 (1 -
#     gamma_b))).  Moment 4 relaxed at the shear rate would give nu_b of
#     lambda_s instead.
#   * the k = 0 spectrum.  On one periodic cell the step is the collision
#     alone; the 19 populations split into the 4 conserved moments, the
#     stress (1 trace + 5 traceless), and 9 kinetic ("ghost") modes, 6 odd
#     and 3 even under c -> -c.  With four distinct rates the eigenvalues
#     1 - lambda come with multiplicities 1 (bulk), 5 (shear), 6 (odd
#     ghosts), 3 (even ghosts), and each eigenspace has the stated parity.
#     Swapped ghost groups would give multiplicities 3 and 6.


def _linear_step_matrix(p, L_):
    """19 x 19 complex matrix of one recombined step acting on a plane-wave
    perturbation exp(i k x), k = 2 pi / L_, of a fluid at rest (rho = 1),
    built column by column from one real run each: the response to
    delta_ij cos(k x) projected on cos gives Re M[:, j], on sin gives
    -Im M[:, j]."""
    shape = (1, 1, L_)
    x = np.arange(L_)
    k = 2 * np.pi / L_
    base = L.equilibrium(np.ones(shape), np.zeros((3,) + shape))
    zero = np.zeros((3,) + shape)
    eps = 1e-7
    M = np.zeros((19, 19), dtype=np.complex128)
    cosk, sink = np.cos(k * x), np.sin(k * x)
    for j in range(19):
        f = base.copy()
        f[j, 0, 0, :] += eps * cosk
        r = (lb.step_recombined(f, zero, zero, p) - base)[:, 0, 0, :] / eps
        M[:, j] = (r @ cosk) * (2.0 / L_) - 1j * (r @ sink) * (2.0 / L_)
    return M


def _sound_damping(p, L_):
    """Gamma / k^2 of the least damped complex-conjugate pair (sound)."""
    mu = np.linalg.eigvals(_linear_step_matrix(p, L_))
    cplx = mu[np.abs(mu.imag) > 1e-6]
    best = cplx[np.argmax(np.abs(cplx))]
    k2 = (2 * np.pi / L_) ** 2
    return -np.log(np.abs(best)) / k2


@pytest.mark.parametrize("lam_s,lam_b", [(1.25, 0.6), (0.8, 1.5), (1.0, 1.0)])
def test_sound_attenuation_pins_bulk_rate(lam_s, lam_b):
    p = lb.LBParams(collision="mrt", tau=1.0, mrt_lambda=(lam_s, lam_b, 1.3, 0.7))
    L1, L2 = 64, 128
    g1, g2 = _sound_damping(p, L1), _sound_damping(p, L2)
    k1, k2 = (2 * np.pi / L1) ** 2, (2 * np.pi / L2) ** 2
    g0 = (g1 * k2 - g2 * k1) / (k2 - k1)          # Richardson in k^2
    nu = (1.0 / lam_s - 0.5) / 3.0
    nu_b = (2.0 / 3.0) * (1.0 / lam_b - 0.5) / 3.0
    expect = 2.0 * nu / 3.0 + nu_b / 2.0
    assert abs(g0 / expect - 1.0) < 1e-4
    if lam_b != lam_s:
        # what the same wave would give with the trace relaxed at the shear rate
        wrong = 2.0 * nu / 3.0 + (2.0 / 3.0) * (1.0 / lam_s - 0.5) / 3.0 / 2.0
        assert abs(g0 / wrong - 1.0) > 1e-2


def test_zero_wavenumber_spectrum_pins_ghost_groups():
    lam = {"shear": 1.3, "bulk": 0.6, "odd": 1.7, "even": 0.45}
    p = lb.LBParams(collision="mrt", tau=1.0,
                    mrt_lambda=(lam["shear"], lam["bulk"], lam["odd"], lam["even"]))
    # one cell: streaming is the identity, the step is the collision
    shape = (1, 1, 1)
    base = L.equilibrium(np.ones(shape), np.zeros((3,) + shape))
    zero = np.zeros((3,) + shape)
    eps = 1e-7
    M = np.zeros((19, 19))
    for j in range(19):
        f = base.copy()
        f[j] += eps
        M[:, j] = (lb.step_recombined(f, zero, zero, p) - base)[:, 0, 0, 0] / eps
    mu, vecs = np.linalg.eig(M)
    assert np.abs(mu.imag).max() < 1e-9
    mu = mu.real
    expect = {"conserved": (1.0, 4), "bulk": (1 - lam["bulk"], 1),
              "shear": (1 - lam["shear"], 5), "odd": (1 - lam["odd"], 6),
              "even": (1 - lam["even"], 3)}
    for name, (val, mult) in expect.items():
        sel = np.abs(mu - val) < 1e-6
        assert sel.sum() == mult, (name, val, np.sort(mu))
        V = vecs[:, sel].real
        flipped = V[L.OPP]
        if name == "odd":
            assert np.abs(flipped + V).max() < 1e-6 * np.abs(V).max()
        elif name in ("even", "bulk", "shear"):
            assert np.abs(flipped - V).max() < 1e-6 * np.abs(V).max()
        if name == "even":
            # kinetic modes carry no density, momentum or stress: orthogonal
            # to every polynomial of degree <= 2 in c
            polys = [np.ones(19)] + [L.CF[:, a] for a in range(3)] + \
                    [L.CF[:, a] * L.CF[:, b] for a in range(3) for b in range(a, 3)]
            for q in polys:
                assert np.abs(q @ V).max() < 1e-6 * np.abs(V).max()
        if name == "shear":
            # traceless stress: no trace, no density
            c2 = (L.CF ** 2).sum(axis=1)
            assert np.abs(c2 @ V).max() < 1e-6 * np.abs(V).max()
            assert np.abs(np.ones(19) @ V).max() < 1e-6 * np.abs(V).max()
