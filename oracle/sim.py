"""Simulation box: the paper's time-marching schemes, operator by operator.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

State between steps: the post-streaming populations fbar and, for the
second-order schemes, the force density F_a spread in the closing half of the
previous step (the physical fluid state at an integer time is
F^1/2(F_a) C^1/2 fbar, see oracle/lb.py).  Particles carry FP64 position,
velocity and mass.

Schemes (h = 1), one call of Sim.step():

  none      fluid only: the second-order LB step with the body force.
  fc / ebf / mebf, order 2, mode 'base'  (Sec. 5.2 Eq. [fc-splitting], Alg. 3)
      P^1/2 F^1/2 (C^1/2 S C^1/2) F^1/2 P^1/2:
      r += h/2 v; F_int(r); u = I[r] u_phys; F^h; v += (h/2m)(F^h + F_int);
      F_b = I*[r](-F^h); LB(F_a, F_b); u = I[r] (sum fbar c / rho);
      F^h; F_a = I*[r](-F^h); v += (h/2m)(F^h + F_int); r += h/2 v.
  ... mode 'inside', n >= 1  (Sec. 6, Eq. [multistep])
      [P^1/4n F^1/2n P^1/4n]^n (C^1/2 S C^1/2) [P^1/4n F^1/2n P^1/4n]^n with
      dt = h/2n: every sub-step couples with the fluid as it stands and
      spreads dt-weighted forces into F_b (or F_a).
  ... mode 'outside', n >= 1  (Sec. 6, the split with F_h^1/2 outside)
      F_h^1/2 [P^1/4n F_int^1/2n P^1/4n]^n (C^1/2 S C^1/2) [...]^n F_h^1/2:
      coupling-only half steps at the ends, intrinsic-force Verlet
      sub-steps in between.
  ibm, order 2  (Sec. 5.1, Eq. [IBM-scheme] with the predictor scheme that
      follows it; Alg. 2 read through that scheme):
      Xt = X + h/2 I[X] u(t); F = F_int(Xt); X += h/2 I[Xt] u(t);
      F_b = I*[Xt] F; LB(F_a, F_b); F_a = F_b; X += h/2 I[Xt] u(t+h),
      u(t+h) including the new F_a.
  order 1 (P S C F, Sec. 5.1 and 5.2):
      fc/ebf/mebf: F_int(r); u = I[r](sum fbar c/rho); F^h (explicit);
      v += (h/m)(F^h + F_int); F = I*[r](-F^h); S C F(F); r += h v.
      ibm: F = F_int(X); S C F(I*[X] F); X += h I[X] u(t+h).

u_phys (second order) = (sum fbar c + (h/2)(F_a + g) + the forces already
applied in the current half step) / rho, the velocity redefinition of Sec. 4.
"""
import numpy as np

from . import lattice as L
from . import lb
from . import delta
from . import coupling as CP
from . import fluct


class CouplingParams:
    def __init__(self, kind='none', order=2, stencil='trilinear', gamma=1.0,
                 substeps=1, mode='base'):
        assert kind in CP.KINDS
        assert mode in ('base', 'inside', 'outside')
        self.kind = kind
        self.order = int(order)
        self.stencil = stencil
        self.gamma = float(gamma)
        self.substeps = int(substeps)
        self.mode = mode


class Sim:
    """One box: LB populations, pending force, particles, coupling."""

    def __init__(self, shape, lbp, cpl=None, parts=None, fbar=None,
                 lb_form='recombined'):
        self.shape = tuple(int(v) for v in shape)        # (nz, ny, nx)
        self.p = lbp
        self.cpl = cpl if cpl is not None else CouplingParams()
        self.parts = parts
        if fbar is None:
            rho = np.full(self.shape, lbp.rho0)
            fbar = L.equilibrium(rho, np.zeros((3,) + self.shape))
        self.fbar = np.array(fbar, dtype=np.float64)
        self.Fa = np.zeros((3,) + self.shape)
        self.lb_form = lb_form
        self.last_Fh = None
        self.t = 0
        self.kT = 0.0            # thermal fluctuations (set_thermal)
        self.seed = None
        self.tstep = 0           # thermal LB steps since the seed was set
        self.printed = False

    def set_thermal(self, kT, seed=0, printed=False):
        """Thermal fluctuations at k_B T (0: off): the fluctuating collision
        of Eq. [mrt-fluct] (stationary amplitude, or the printed one) and the
        random force zeta of force-coupled particles (FC and original EBF).
        The thermal step counter restarts when the seed changes and keeps
        running otherwise (steps without fluctuations do not advance it)."""
        if kT > 0.0 and seed != self.seed:
            self.tstep = 0
            self.seed = seed
        self.kT = float(kT)
        self.printed = bool(printed)

    # ----------------------------------------------------------- helpers
    def _lb(self, Fa, Fb):
        if self.kT > 0.0:
            zero = np.zeros((3,) + self.shape)
            if self.cpl.order == 1:
                # first order: the whole force F_b for the step (u1 = u0 + (F + g)/rho)
                Fa = Fb = zero if Fb is None else Fb
            if self.lb_form == 'literal':
                out = fluct.step_literal_fluct(self.fbar, Fa, Fb, self.p, self.kT, self.seed,
                                               self.tstep)
            else:
                out = fluct.step_recombined_fluct(self.fbar, Fa, Fb, self.p, self.kT, self.seed,
                                                  self.tstep, self.printed)
            self.tstep += 1
            return out
        if self.cpl.order == 1:
            return lb.step_first_order(self.fbar, Fb, self.p)
        if self.lb_form == 'literal':
            return lb.step_literal(self.fbar, Fa, Fb, self.p)
        return lb.step_recombined(self.fbar, Fa, Fb, self.p)

    def _fluid_velocity(self, *pending):
        """(sum fbar c + (h/2) sum(pending)) / rho; pending are force
        densities (3, ...) or uniform 3-vectors already applied for half a
        step each (with their weights folded in)."""
        rho = L.density(self.fbar)
        j = L.momentum(self.fbar)
        for F in pending:
            F = np.asarray(F)
            if F.ndim == 1:
                F = F.reshape(3, 1, 1, 1)
            j = j + 0.5 * F
        return j / rho

    def _interp(self, field, pos):
        return delta.interpolate(field, pos, self.cpl.stencil, self.p.walls)

    def _spread(self, forces, pos):
        return delta.spread(forces, pos, self.shape, self.cpl.stencil,
                            self.p.walls)

    def _wrap(self, pos):
        return CP.wrap_positions(pos, self.shape, self.p.walls)

    def _fint(self, pos):
        return CP.intrinsic_forces(self.parts, pos, self.shape, self.p.walls)

    def _couple(self, v, u, Fint, s, include_int=True, sub=0):
        """F^h of coupling (sub-)step number `sub` of the current step (its
        random force when thermal: FC and original EBF)."""
        c = self.cpl
        zeta = None
        if self.kT > 0.0 and c.kind in ('fc', 'ebf'):
            gam = self.p.rho0 if c.kind == 'ebf' else c.gamma
            zeta = fluct.particle_noise(len(v), self._tnow, sub, s, gam, self.kT, self.seed)
        return CP.coupling_force(c.kind, c.order, v, u, Fint, self.parts.mass,
                                 s, c.gamma, self.p.rho0, include_int, zeta)

    # ------------------------------------------------------------- steps
    def step(self):
        c = self.cpl
        self._tnow = self.tstep          # the thermal counter of this step
        if c.kind == 'none' or self.parts is None:
            self._step_fluid_only()
        elif c.kind == 'ibm':
            self._step_ibm1() if c.order == 1 else self._step_ibm2()
        elif c.order == 1:
            self._step_fc1()
        elif c.mode == 'base':
            self._step_fc2_base()
        elif c.mode == 'inside':
            self._step_fc2_inside()
        else:
            self._step_fc2_outside()
        self.t += 1

    def _step_fluid_only(self):
        if self.cpl.order == 1:
            self.fbar = self._lb(None, None)
            return
        zero = np.zeros((3,) + self.shape)
        self.fbar = self._lb(zero, zero)
        self.Fa = zero

    def _step_fc2_base(self):
        P = self.parts
        g = self.p.g
        r = self._wrap(P.pos + 0.5 * P.vel)
        Fint = self._fint(r)
        u = self._interp(self._fluid_velocity(self.Fa, g), r)
        Fh = self._couple(P.vel, u, Fint, 0.5, sub=0)
        v = P.vel + (0.5 / P.mass[:, None]) * (Fh + Fint)
        Fb = self._spread(-Fh, r)
        self.fbar = self._lb(self.Fa, Fb)
        u = self._interp(self._fluid_velocity(), r)
        Fh = self._couple(v, u, Fint, 0.5, sub=1)
        self.Fa = self._spread(-Fh, r)
        v = v + (0.5 / P.mass[:, None]) * (Fh + Fint)
        P.pos = self._wrap(r + 0.5 * v)
        P.vel = v
        self.last_Fh = Fh

    def _half_inside(self, r, v, before):
        """n sub-steps [P^1/4n F^1/2n P^1/4n] of one half (Eq. [multistep])."""
        P = self.parts
        n = self.cpl.substeps
        dt = 0.5 / n
        g = self.p.g
        acc = np.zeros((3,) + self.shape)
        Fh = None
        for s in range(n):
            r = self._wrap(r + 0.5 * dt * v)
            Fint = self._fint(r)
            if before:
                field = self._fluid_velocity(self.Fa, g, acc, (s / n) * g)
            else:
                field = self._fluid_velocity(acc, (s / n) * g)
            u = self._interp(field, r)
            Fh = self._couple(v, u, Fint, dt, sub=(0 if before else n) + s)
            v = v + (dt / P.mass[:, None]) * (Fh + Fint)
            acc = acc + (1.0 / n) * self._spread(-Fh, r)
            r = self._wrap(r + 0.5 * dt * v)
        return r, v, acc, Fh

    def _step_fc2_inside(self):
        P = self.parts
        r, v, Fb, _ = self._half_inside(P.pos, P.vel, True)
        self.fbar = self._lb(self.Fa, Fb)
        r, v, self.Fa, Fh = self._half_inside(r, v, False)
        P.pos, P.vel = r, v
        self.last_Fh = Fh

    def _verlet_int(self, r, v):
        """[P^1/4n F_int^1/2n P^1/4n]^n: particle-only sub-steps."""
        P = self.parts
        n = self.cpl.substeps
        dt = 0.5 / n
        for _ in range(n):
            r = self._wrap(r + 0.5 * dt * v)
            v = v + (dt / P.mass[:, None]) * self._fint(r)
            r = self._wrap(r + 0.5 * dt * v)
        return r, v

    def _step_fc2_outside(self):
        P = self.parts
        g = self.p.g
        r, v = P.pos, P.vel
        zero = np.zeros_like(v)
        u = self._interp(self._fluid_velocity(self.Fa, g), r)
        Fh = self._couple(v, u, zero, 0.5, include_int=False, sub=0)
        v = v + (0.5 / P.mass[:, None]) * Fh
        Fb = self._spread(-Fh, r)
        r, v = self._verlet_int(r, v)
        self.fbar = self._lb(self.Fa, Fb)
        r, v = self._verlet_int(r, v)
        u = self._interp(self._fluid_velocity(), r)
        Fh = self._couple(v, u, zero, 0.5, include_int=False, sub=1)
        self.Fa = self._spread(-Fh, r)
        v = v + (0.5 / P.mass[:, None]) * Fh
        P.pos, P.vel = r, v
        self.last_Fh = Fh

    def _step_fc1(self):
        P = self.parts
        r = P.pos
        Fint = self._fint(r)
        u = self._interp(self._fluid_velocity(), r)
        Fh = self._couple(P.vel, u, Fint, 1.0, sub=0)
        v = P.vel + (1.0 / P.mass[:, None]) * (Fh + Fint)
        F = self._spread(-Fh, r)
        self.fbar = self._lb(None, F)
        P.pos = self._wrap(r + v)
        P.vel = v
        self.last_Fh = Fh

    def _step_ibm2(self):
        P = self.parts
        g = self.p.g
        X = P.pos
        ut = self._fluid_velocity(self.Fa, g)
        Xt = self._wrap(X + 0.5 * self._interp(ut, X))
        F = self._fint(Xt)
        Xh = self._wrap(X + 0.5 * self._interp(ut, Xt))
        Fb = self._spread(F, Xt)
        self.fbar = self._lb(self.Fa, Fb)
        self.Fa = Fb
        u1 = self._fluid_velocity(self.Fa, g)
        P.pos = self._wrap(Xh + 0.5 * self._interp(u1, Xt))
        self.last_Fh = F

    def _step_ibm1(self):
        P = self.parts
        X = P.pos
        F = self._fint(X)
        self.fbar = self._lb(None, self._spread(F, X))
        u1 = self._fluid_velocity()
        P.pos = self._wrap(X + self._interp(u1, X))
        self.last_Fh = F

    # ------------------------------------------------------- observables
    def fluid_velocity(self):
        """Physical fluid velocity (3, nz, ny, nx) at the current time."""
        return lb.physical_velocity(self.fbar, self.Fa, self.p,
                                    order=self.cpl.order)

    def density(self):
        return L.density(self.fbar)

    def fluid_momentum(self):
        rho = self.density()
        return (rho[None] * self.fluid_velocity()).reshape(3, -1).sum(axis=1)

    def particle_momentum(self):
        if self.parts is None or self.cpl.kind == 'ibm':
            return np.zeros(3)
        return (self.parts.mass[:, None] * self.parts.vel).sum(axis=0)

    def total_momentum(self):
        return self.fluid_momentum() + self.particle_momentum()

    def mass(self):
        return self.density().sum()
