"""Lattice-Boltzmann sub-operators and the two LB step forms (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Arrays: populations f[i, z, y, x] (shape (19, nz, ny, nx)); vector fields
F[a, z, y, x] with a = (x, y, z) component; lattice units h = a = 1.

Operators (Sec. 3):
  S       streaming, f_i(x + h c_i, t + h) = f_i(x, t)            (Sec. 3.1)
  C       full collision, f^neq -> (1 - Lambda) f^neq             (Sec. 3.2,
          Eq. [CN-coll], Eq. [collision-operator]; MRT: Eq. [mrt-coll])
  C^1/2   half collision with 1 - lambda_1/2 = sqrt(1 - lambda)   (Sec. 3.2,
          after Eq. [collision-operator2]); exists only when every
          1 - lambda >= 0
  F^s     force operator over a step s with the midpoint rule
          f -> f + s G(t + s/2)                 (Sec. 3.3, Eq. [force-midpoint])

Two step forms, checked against each other in the tests:
  (O1) literal: S C^1/2 F^1/2_b F^1/2_a C^1/2 applied operator by operator to
       the post-streaming populations fbar (Sec. 4, Eqs. [force-second-halfstep]
       to [force-first-halfstep]); F_a is the force of the previous step's
       closing half, F_b the force of this step's opening half.
  (O2) recombined: fbar_new(x + c_i) = f_i^eq(rho, u1) + [(1 - Lambda)(fbar -
       f^eq(rho, u0))]_i with u0 = sum fbar c / rho and
       u1 = u0 + (h/2)(F_a + F_b)/rho.  This is (O1) with the two half
       collisions merged, which is exact because each half force step only
       shifts the equilibrium velocity (see force_half_step); it needs no
       square root of (1 - Lambda), so it also holds for tau < 1.

Readings of the paper taken here:
  * tau is the standard lattice relaxation time, lambda = 1/tau for BGK
    (full step), nu = (tau - 1/2)/3.  The paper's continuous tau of
    Eq. [BGKlambda] is tau_paper = tau - 1/2 to O(h^2).
  * G in each force half-step is evaluated at the midpoint velocity
    u + s F/(2 rho) of that half-step (Sec. 3.3 says only "midpoint"); with
    this choice F^s maps f^eq(rho, u) to exactly f^eq(rho, u + s F/rho) and
    leaves f - f^eq unchanged (the statement after Eq. [LB-force-moments],
    made exact).
  * Each collision uses the equilibrium of the populations it acts on
    (collisions conserve rho and rho u).
  * A uniform body force g is part of the force operator: each half step
    applies (h/2) g in addition to the spread coupling forces.
  * Walls (not in the paper): halfway bounce-back at z = -1/2 and
    z = nz - 1/2, moving-wall term 2 w_i rho0 (c_i . u_w)/cs2 added to the
    reflected population.
"""
import numpy as np

from . import lattice as L


class LBParams:
    """Lattice description: relaxation, reference density, body force, walls.

    collision: 'bgk' or 'mrt'.  tau: lattice BGK relaxation time (shear
    rate 1/tau for MRT unless mrt_lambda overrides).  walls: halfway
    bounce-back in z with wall velocities u_bot, u_top (3-vectors).
    """

    def __init__(self, collision='bgk', tau=1.0, mrt_lambda=(0, 0, 0, 0),
                 rho0=1.0, body_force=(0.0, 0.0, 0.0), walls=False,
                 u_bot=(0.0, 0.0, 0.0), u_top=(0.0, 0.0, 0.0)):
        self.collision = collision
        self.tau = float(tau)
        self.mrt_lambda = tuple(float(v) for v in mrt_lambda)
        self.rho0 = float(rho0)
        self.g = np.array(body_force, dtype=np.float64)
        self.walls = bool(walls)
        self.u_bot = np.array(u_bot, dtype=np.float64)
        self.u_top = np.array(u_top, dtype=np.float64)

    def gamma_full(self):
        """Eigenvalues 1 - lambda of the full-step collision C."""
        if self.collision == 'bgk':
            return 1.0 - 1.0 / self.tau
        return 1.0 - L.mrt_rates(self.tau, self.mrt_lambda)

    def gamma_half(self):
        """Eigenvalues of C^1/2: sqrt(1 - lambda) (Sec. 3.2)."""
        gam = np.asarray(self.gamma_full(), dtype=np.float64)
        if np.any(gam < 0.0):
            raise ValueError("C^1/2 needs 1 - lambda >= 0 (tau >= 1); "
                             "use the recombined step")
        return np.sqrt(gam)


def velocity(f):
    return L.momentum(f) / L.density(f)


def relax(f, gam, p):
    """Collision f -> f^eq + Gamma (f - f^eq) about the moments of f.

    BGK: Gamma = gam (scalar).  MRT: Gamma = diag(gam_k) in the moment basis
    (Eq. [mrt-coll]); back-transform by the inverse basis matrix.
    """
    rho = L.density(f)
    feq = L.equilibrium(rho, L.momentum(f) / rho)
    fneq = f - feq
    if p.collision == 'bgk':
        return feq + gam * fneq
    m = np.tensordot(L.MRT_E, fneq, axes=([1], [0]))
    m = np.asarray(gam).reshape((L.Q,) + (1,) * (f.ndim - 1)) * m
    Einv = np.linalg.inv(L.MRT_E)
    return feq + np.tensordot(Einv, m, axes=([1], [0]))


def force_step(f, F, s):
    """Force operator over a step s: f + s G(u_mid, F), u_mid = u + sF/(2rho).

    Sec. 3.3, Eq. [force-midpoint]; F is a force density field (3, ...).
    """
    rho = L.density(f)
    u = L.momentum(f) / rho
    umid = u + 0.5 * s * F / rho
    return f + s * L.force_term(umid, F)


def stream(fs, p):
    """S: fbar_i(x + c_i) = f*_i(x); periodic, or bounce-back walls in z."""
    out = np.empty_like(fs)
    nz = fs.shape[1]
    for i in range(L.Q):
        cx, cy, cz = L.C[i]
        if not p.walls:
            out[i] = np.roll(fs[i], (cz, cy, cx), axis=(0, 1, 2))
            continue
        rolled = np.roll(fs[i], (cy, cx), axis=(1, 2))
        if cz == 0:
            out[i] = rolled
        elif cz == 1:
            out[i, 1:] = rolled[:-1]
        else:
            out[i, :-1] = rolled[1:]
    if p.walls:
        for i in range(L.Q):
            cz = L.C[i][2]
            if cz == 0:
                continue
            j = L.OPP[i]
            # population i leaves the boundary layer towards the wall and
            # comes back, at the same node, as population j = -c_i
            if cz == 1:
                zb, uw = nz - 1, p.u_top
            else:
                zb, uw = 0, p.u_bot
            out[j, zb] = fs[i, zb] + 2.0 * L.W[j] * p.rho0 * \
                (L.CF[j] @ uw) / L.CS2
    return out


def _field(F, shape):
    if F is None:
        return np.zeros((3,) + shape)
    return F


def step_literal(fbar, Fa, Fb, p):
    """(O1) S C^1/2 F^1/2(F_b + g) F^1/2(F_a + g) C^1/2 acting on fbar.

    Sec. 4, Eqs. [force-second-halfstep]-[force-first-halfstep]: the closing
    half of the previous step (C^1/2 then F^1/2 with F_a) gives the physical
    f(t); the opening half of this step (F^1/2 with F_b, C^1/2) and the
    streaming give the next post-streaming populations.
    """
    shape = fbar.shape[1:]
    g = p.g.reshape(3, 1, 1, 1)
    gh = p.gamma_half()
    f = relax(fbar, gh, p)
    f = force_step(f, _field(Fa, shape) + g, 0.5)
    f = force_step(f, _field(Fb, shape) + g, 0.5)
    f = relax(f, gh, p)
    return stream(f, p)


def step_recombined(fbar, Fa, Fb, p):
    """(O2) fbar_new(x + c) = f^eq(rho, u1) + (1 - Lambda)(fbar - f^eq(rho, u0)).

    u1 = u0 + (h/2)(F_a + F_b + 2 g)/rho.  Equal to step_literal whenever the
    latter exists (tests), and valid for every tau > 1/2.
    """
    shape = fbar.shape[1:]
    g = p.g.reshape(3, 1, 1, 1)
    rho = L.density(fbar)
    u0 = L.momentum(fbar) / rho
    u1 = u0 + 0.5 * (_field(Fa, shape) + _field(Fb, shape) + 2.0 * g) / rho
    gam = p.gamma_full()
    neq = fbar - L.equilibrium(rho, u0)
    if p.collision == 'bgk':
        post_neq = gam * neq
    else:
        m = np.tensordot(L.MRT_E, neq, axes=([1], [0]))
        m = np.asarray(gam).reshape((L.Q, 1, 1, 1)) * m
        post_neq = np.tensordot(np.linalg.inv(L.MRT_E), m, axes=([1], [0]))
    return stream(L.equilibrium(rho, u1) + post_neq, p)


def step_first_order(fbar, F, p):
    """First-order fluid part of the P S C F schemes (Sec. 5.1, 5.2).

    A full force step F^h with F + g, then the full collision C, then S.
    The fluid velocity seen by the particles is sum fbar c / rho.
    """
    shape = fbar.shape[1:]
    g = p.g.reshape(3, 1, 1, 1)
    f = force_step(fbar, _field(F, shape) + g, 1.0)
    f = relax(f, p.gamma_full(), p)
    return stream(f, p)


def physical_velocity(fbar, Fa, p, order=2):
    """Hydrodynamic velocity of the fluid at integer times.

    Second order: rho u = sum fbar c + (h/2)(F_a + g) (Sec. 4, the velocity
    redefinition after Eq. [force-transformation]; the paper's "c_i c_i"
    there is read as c_i).  First order: rho u = sum fbar c.
    """
    rho = L.density(fbar)
    j = L.momentum(fbar)
    if order == 2:
        j = j + 0.5 * (_field(Fa, fbar.shape[1:]) + p.g.reshape(3, 1, 1, 1))
    return j / rho


def viscous_stress(fbar, p):
    """Viscous stress of the post-streaming populations, Eq. [viscstress]
    (first line, Sec. 3.4):

        sigma = 1/2 (1 + (1 - Lambda_1/2)^2) sum_i (fbar_i - f^eq_i) c_i c_i

    with (1 - Lambda_1/2)^2 = 1 - Lambda the full-step collision eigenvalues
    (gamma for BGK, diag(gamma_k) in the moment basis for MRT) and f^eq at
    the density and velocity of fbar (a force half step leaves fbar - f^eq
    unchanged).  Returns sigma[a, b, z, y, x].
    """
    rho = L.density(fbar)
    feq = L.equilibrium(rho, L.momentum(fbar) / rho)
    fneq = fbar - feq
    gam = p.gamma_full()
    if p.collision == 'bgk':
        scaled = 0.5 * (1.0 + gam) * fneq
    else:
        m = np.tensordot(L.MRT_E, fneq, axes=([1], [0]))
        m = 0.5 * (1.0 + np.asarray(gam)).reshape((L.Q,) + (1,) * (fbar.ndim - 1)) * m
        scaled = np.tensordot(np.linalg.inv(L.MRT_E), m, axes=([1], [0]))
    return np.einsum('ia,ib,i...->ab...', L.CF, L.CF, scaled)


def half_collision_approx(f, p):
    """The O(h^2) half collision (1 + C)/2 of Eq. [half-col-approx].

    Kept only for the negative test: with it the CSC scheme no longer has the
    viscosity of the standard scheme (Sec. 4, discussion of
    Eq. [half-collision]).
    """
    return 0.5 * (f + relax(f, p.gamma_full(), p))


def step_literal_approx_half(fbar, p):
    """S C~ C~ fbar with C~ = (1 + C)/2, no forces (negative test only)."""
    return stream(half_collision_approx(half_collision_approx(fbar, p), p), p)
