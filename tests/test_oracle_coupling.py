"""Pins for the coupling schemes in oracle/sim.py and oracle/coupling.py.

On a periodic box of ONE cell every stencil node is the same node, so the
interpolation returns the node velocity and the spreading puts the whole
force on it: the coupled system reduces exactly to the two-variable ODE of
Sec. 5.2, Eq. [fc-vel],
    m dv/dt = -gamma (v - u) + F_int,   rho du/dt = gamma (v - u).
Closed forms used:
  * Crank-Nicolson half step with s = h/2: w = v - u is multiplied by
    (1 - x)/(1 + x), x = (alpha + beta)/2 = gamma s (1/m + 1/rho)/2
    (Eqs. [fc-cn], [modified-force]); a full step of the split scheme is two
    such factors, the first-order scheme one factor 1 - gamma h (1/m + 1/rho);
  * the exact solution w(t) = w0 exp(-gamma (1/m + 1/rho) t): second-order
    versus first-order error when the step is refined;
  * rho u + m v is conserved (Sec. 5.2, the coupling force "must not change
    the total momentum");
  * slip h'/(2m) F_int with the friction of Eq. [gamma-cond] (Eq. [slip]);
  * modified EBF: v = u after every force application (Sec. 5.3);
  * immersion number r -> 1 (m -> 0): the modified EBF tends to the IBM
    (Sec. 5.3, Eq. [immersion]) with an O(m) difference;
  * uniform acceleration: IBM second order advects tracers exactly
    (trapezoidal rule on a linear-in-time velocity), first order lags by g t/2;
  * periodic box with bonds and a body force: total momentum grows by
    exactly h g N per step for every coupling kind and scheme.
"""
import numpy as np
import pytest

from oracle import lattice as L
from oracle import lb
from oracle import sim as S
from oracle import coupling as CP
from oracle import delta


def _one_cell(kind, order, gamma, m, v0, mode="base", n=1, tau=0.8,
              stencil="trilinear", ext=None, rho0=1.0):
    p = lb.LBParams(tau=tau, rho0=rho0)
    parts = CP.Particles([[0.37, 0.61, 0.18]], vel=[v0], mass=[m],
                         ext_force=None if ext is None else [ext])
    cpl = S.CouplingParams(kind, order, stencil, gamma=gamma, substeps=n,
                           mode=mode)
    fbar = L.equilibrium(np.full((1, 1, 1), rho0), np.zeros((3, 1, 1, 1)))
    return S.Sim((1, 1, 1), p, cpl, parts, fbar=fbar)


def _w(sm):
    return sm.parts.vel[0] - sm.fluid_velocity()[:, 0, 0, 0]


@pytest.mark.parametrize("mode,n", [("base", 1), ("inside", 1), ("inside", 3),
                                    ("outside", 1), ("outside", 2)])
@pytest.mark.parametrize("stencil", ["trilinear", "peskin4", "peskin3"])
def test_one_cell_split_scheme_recurrence(mode, n, stencil):
    gamma, m, rho = 1.3, 0.7, 1.0
    sm = _one_cell("fc", 2, gamma, m, [0.01, -0.004, 0.002], mode=mode, n=n,
                   stencil=stencil)
    if mode == "inside":
        s, k = 0.5 / n, 2 * n
    else:
        s, k = 0.5, 2
    x = gamma * s * (1.0 / m + 1.0 / rho) / 2.0
    gfac = ((1.0 - x) / (1.0 + x)) ** k
    P0 = sm.total_momentum()
    w0 = _w(sm)
    for step in range(1, 8):
        sm.step()
        assert np.abs(_w(sm) - w0 * gfac ** step).max() < 1e-15
    assert np.abs(sm.total_momentum() - P0).max() < 1e-16


def test_one_cell_first_order_recurrence():
    gamma, m, rho = 0.4, 1.5, 1.0
    sm = _one_cell("fc", 1, gamma, m, [0.01, 0.0, -0.02])
    gfac = 1.0 - gamma * (1.0 / m + 1.0 / rho)
    P0 = sm.total_momentum()
    w0 = _w(sm)
    for step in range(1, 8):
        sm.step()
        assert np.abs(_w(sm) - w0 * gfac ** step).max() < 1e-16
    assert np.abs(sm.total_momentum() - P0).max() < 1e-16


def test_one_cell_ebf_is_fc_with_rho_over_h():
    a = _one_cell("ebf", 2, 123.0, 2.0, [0.01, 0, 0], rho0=1.0)
    gamma = 1.0                     # rho0 a^3 / h
    x = gamma * 0.5 * (1.0 / 2.0 + 1.0) / 2.0
    gfac = ((1.0 - x) / (1.0 + x)) ** 2
    w0 = _w(a)
    a.step()
    assert np.abs(_w(a) - w0 * gfac).max() < 1e-16


@pytest.mark.parametrize("order,expect", [(2, 2.0), (1, 1.0)])
def test_order_of_accuracy_in_the_step(order, expect):
    """Halving gamma and doubling the steps halves the step in units of the
    relaxation time; the error at fixed time falls by 2^order."""
    m, rho = 1.0, 1.0
    errs = []
    for refine in (1, 2, 4, 8):
        gamma = 0.1 / refine
        nsteps = 10 * refine
        sm = _one_cell("fc", order, gamma, m, [0.01, 0, 0])
        w0 = _w(sm)[0]
        for _ in range(nsteps):
            sm.step()
        exact = w0 * np.exp(-gamma * (1 / m + 1 / rho) * nsteps)
        errs.append(abs(_w(sm)[0] - exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - expect) < 0.1), rates


def test_slip_with_no_slip_friction():
    """Eq. [gamma-cond] with h -> h/2 leaves exactly v - u = (h/2)/(2m) F_int
    after every closing half step (Eq. [slip])."""
    m, rho = 0.8, 1.0
    s = 0.5
    gamma = (rho / s) * 2.0 / (1.0 + rho / m)
    F = np.array([1e-4, -2e-4, 5e-5])
    sm = _one_cell("fc", 2, gamma, m, [0.0, 0.0, 0.0], ext=F)
    for _ in range(5):
        sm.step()
        assert np.abs(_w(sm) - s / (2 * m) * F).max() < 1e-17


def test_modified_ebf_no_slip_after_each_step():
    F = np.array([3e-4, 1e-4, -2e-4])
    sm = _one_cell("mebf", 2, 0.0, 0.9, [0.02, -0.01, 0.0], ext=F)
    P = [sm.total_momentum()]
    for _ in range(6):
        sm.step()
        assert np.abs(_w(sm)).max() < 1e-17
        P.append(sm.total_momentum())
    # the external force is the only momentum source: dP = F per step
    assert np.abs(np.diff(np.array(P), axis=0) - F).max() < 1e-16


def test_one_cell_immersion_limit_is_ibm():
    """m -> 0 (r -> 1): modified EBF positions and fluid velocity converge to
    the IBM scheme with differences O(m)."""
    F = np.array([2e-4, -1e-4, 5e-5])

    def run(kind, m):
        sm = _one_cell(kind, 2, 0.0, m, [0.0, 0.0, 0.0], ext=F)
        if kind == "mebf":
            sm.parts.vel[0] = sm.fluid_velocity()[:, 0, 0, 0]
        for _ in range(20):
            sm.step()
        d = sm.parts.pos[0]
        return d, sm.fluid_velocity()[:, 0, 0, 0]

    xi, ui = run("ibm", 0.0)
    errs = []
    for m in (1e-2, 1e-3, 1e-4):
        x, u = run("mebf", m)
        errs.append(max(np.abs(x - xi).max(), np.abs(u - ui).max()))
    assert errs[-1] < 1e-5          # 0.04 m after 20 steps
    assert 5 < errs[0] / errs[1] < 20 and 5 < errs[1] / errs[2] < 20


def test_immersion_limit_converges_on_a_box(rng):
    """On a real grid the m -> 0 limit of the modified EBF exists (Cauchy
    differences shrink like m) and the fluid receives the whole intrinsic
    force (F^h -> -F_int)."""
    shape = (8, 8, 8)
    u = np.zeros((3,) + shape)
    u[0] = 0.01 * np.sin(2 * np.pi * np.arange(8) / 8)[:, None, None]
    f0 = L.equilibrium(np.ones(shape), u)
    pos0 = rng.uniform(0, 8, (4, 3))
    bonds = [[0, 1], [1, 2], [2, 3]]

    def run(m):
        p = lb.LBParams(tau=0.8)
        parts = CP.Particles(pos0.copy(), mass=np.full(4, m), bonds=bonds,
                             bond_k=0.01, bond_r0=1.0)
        sm = S.Sim(shape, p, S.CouplingParams("mebf", 2, "peskin4"), parts,
                   fbar=f0.copy())
        parts.vel = delta.interpolate(sm.fluid_velocity(), parts.pos, "peskin4")
        for _ in range(15):
            sm.step()
        return parts.pos.copy(), sm.last_Fh, sm

    prev = None
    diffs = []
    for m in (1e-2, 1e-3, 1e-4):
        X, Fh, sm = run(m)
        if prev is not None:
            diffs.append(np.abs(CP.min_image(X - prev, shape, False)).max())
        prev = X
    assert 5 < diffs[0] / diffs[1] < 20
    # F^h + r F_int -> the (m/s)(u - v) term, which vanishes with m
    X, Fh, sm = run(1e-8)
    # the closing half step acted at the mid-step positions r - (h/2) v
    r_mid = CP.wrap_positions(sm.parts.pos - 0.5 * sm.parts.vel, shape, False)
    fint = CP.intrinsic_forces(sm.parts, r_mid, shape, False)
    assert np.abs(Fh + fint).max() < 1e-6


def test_heavy_particle_limit_is_the_original_ebf(rng):
    """The other end of the immersion number (Sec. 5.3, Eq. [immersion]):
    m >> rho a^3 gives r -> 0, and the modified EBF becomes the original
    EBF of Eq. [ebf] (gamma = rho a^3 / h, intrinsic forces on the particles
    only), here the explicit first-order forms of both on a grid with bonds
    and a body force: differences shrink like 1/m."""
    shape = (6, 7, 8)
    u = np.zeros((3,) + shape)
    u[0] = 0.01 * np.sin(2 * np.pi * np.arange(6) / 6)[:, None, None]
    f0 = L.equilibrium(np.ones(shape), u)
    pos0 = rng.uniform(0, 6, (4, 3))
    vel0 = 0.01 * rng.standard_normal((4, 3))
    bonds = [[0, 1], [1, 2], [2, 3]]

    def run(kind, m):
        p = lb.LBParams(tau=0.8, body_force=(1e-5, 0.0, 0.0))
        parts = CP.Particles(pos0.copy(), vel=vel0.copy(), mass=np.full(4, m), bonds=bonds,
                             bond_k=0.05, bond_r0=1.0)
        sm = S.Sim(shape, p, S.CouplingParams(kind, 1, "trilinear"), parts, fbar=f0.copy())
        for _ in range(6):
            sm.step()
        return sm

    ref_last = None
    diffs = []
    for m in (1e5, 1e6, 1e7):
        a, b = run("mebf", m), run("ebf", m)
        d = max(np.abs(a.fbar - b.fbar).max(), np.abs(a.parts.vel - b.parts.vel).max(),
                np.abs(CP.min_image(a.parts.pos - b.parts.pos, shape, False)).max())
        diffs.append(d)
        ref_last = d
    assert ref_last < 1e-8, diffs
    assert 5 < diffs[0] / diffs[1] < 20 and 5 < diffs[1] / diffs[2] < 20, diffs


def test_ibm_uniform_acceleration():
    """Body force g on a periodic box: u_phys(t) = u_phys(0) + g t exactly, so
    the trapezoidal IBM update is exact and the first-order one lags by
    g t/2 (per unit h)."""
    shape = (4, 4, 4)
    g = np.array([1e-5, -2e-5, 0.5e-5])
    u0 = np.array([0.01, 0.0, -0.003])
    f0 = L.equilibrium(np.ones(shape), np.broadcast_to(u0[:, None, None, None],
                                                       (3,) + shape).copy())
    X0 = np.array([[1.3, 2.6, 0.4], [3.2, 0.1, 2.9]])
    N = 30
    for order in (2, 1):
        p = lb.LBParams(tau=0.9, body_force=g)
        parts = CP.Particles(X0.copy())
        sm = S.Sim(shape, p, S.CouplingParams("ibm", order, "peskin4"), parts,
                   fbar=f0.copy())
        U0 = sm.fluid_velocity()[:, 0, 0, 0]
        for _ in range(N):
            sm.step()
        exact = X0 + N * U0 + 0.5 * g * N * N
        d = CP.min_image(sm.parts.pos - exact, shape, False)
        if order == 2:
            assert np.abs(U0 - (u0 + 0.5 * g)).max() < 1e-16
            assert np.abs(d).max() < 1e-13
        else:
            assert np.abs(d - 0.5 * g * N).max() < 1e-13


SCHEMES = [("fc", 2, "base", 1), ("fc", 2, "inside", 2), ("fc", 2, "outside", 2),
           ("ebf", 2, "base", 1), ("mebf", 2, "base", 1), ("mebf", 2, "inside", 2),
           ("fc", 1, "base", 1), ("mebf", 1, "base", 1), ("ibm", 2, "base", 1),
           ("ibm", 1, "base", 1)]


@pytest.mark.parametrize("kind,order,mode,n", SCHEMES)
@pytest.mark.parametrize("stencil", ["trilinear", "peskin4"])
def test_total_momentum_budget(kind, order, mode, n, stencil, rng):
    shape = (6, 5, 7)
    g = np.array([1e-5, 0.0, -2e-5])
    M = 6
    pos = rng.uniform(0, 1, (M, 3)) * np.array([7, 5, 6])
    vel = 0.01 * rng.standard_normal((M, 3))
    bonds = [[i, i + 1] for i in range(M - 1)]
    parts = CP.Particles(pos, vel=vel, mass=rng.uniform(0.5, 2.0, M),
                         bonds=bonds, bond_k=0.05, bond_r0=1.0)
    p = lb.LBParams(collision="mrt", tau=0.75, body_force=g)
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    u = 0.01 * rng.standard_normal((3,) + shape)
    sm = S.Sim(shape, p, S.CouplingParams(kind, order, stencil, gamma=2.0,
                                          substeps=n, mode=mode),
               parts, fbar=L.equilibrium(rho, u))
    P0 = sm.total_momentum()
    N = np.prod(shape)
    for t in range(1, 6):
        sm.step()
        assert np.abs(sm.total_momentum() - P0 - t * g * N).max() < 1e-14
    assert abs(sm.mass() - L.density(L.equilibrium(rho, u)).sum()) < 1e-11


@pytest.mark.parametrize("kind", ["fc", "mebf", "ibm"])
def test_literal_and_recombined_lb_give_same_trajectories(kind, rng):
    shape = (6, 6, 6)
    pos = rng.uniform(0, 6, (5, 3))
    bonds = [[0, 1], [1, 2], [3, 4]]
    sims = []
    for form in ("literal", "recombined"):
        parts = CP.Particles(pos.copy(), vel=0.01 * np.ones((5, 3)),
                             bonds=bonds, bond_k=0.02, bond_r0=1.0)
        p = lb.LBParams(collision="mrt", tau=1.25, mrt_lambda=(0, 0.9, 0.8, 1.0),
                        body_force=(1e-5, 0, 0))
        sm = S.Sim(shape, p, S.CouplingParams(kind, 2, "peskin4", gamma=1.5),
                   parts, lb_form=form)
        for _ in range(6):
            sm.step()
        sims.append(sm)
    a, b = sims
    assert np.abs(a.fbar - b.fbar).max() < 1e-15
    assert np.abs(a.parts.pos - b.parts.pos).max() < 1e-13
    assert np.abs(a.parts.vel - b.parts.vel).max() < 1e-15


@pytest.mark.parametrize("kind,order", [("fc", 2), ("fc", 1), ("mebf", 2), ("ebf", 2), ("ibm", 2),
                                        ("ibm", 1)])
def test_empty_particle_set_is_the_fluid_step(kind, order):
    """Degenerate case: with no particles every coupling operator is the
    identity and spreads nothing, so the coupled step is the fluid step with
    its body force, bit for bit."""
    shape = (6, 7, 9)
    rng = np.random.default_rng(4)
    fbar = L.equilibrium(np.ones(shape), np.zeros((3,) + shape)) * (1.0 + 1e-3 * rng.standard_normal((19,) + shape))
    p = lb.LBParams(collision="mrt", tau=0.9, body_force=(2e-5, -1e-5, 0.0))
    parts = CP.Particles(np.zeros((0, 3)), vel=np.zeros((0, 3)), mass=np.ones(0))
    sm = S.Sim(shape, p, S.CouplingParams(kind, order, "peskin4", gamma=1.0), parts,
                fbar=fbar.copy())
    ref = S.Sim(shape, p, S.CouplingParams("none", order, "trilinear"), None, fbar=fbar.copy())
    for _ in range(3):
        sm.step()
        ref.step()
    assert np.array_equal(sm.fbar, ref.fbar)
    assert sm.parts.pos.shape == (0, 3)
