"""Coupling operators for immersed particles (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Coupling force over a (sub-)step of length s, particle i with velocity v,
interpolated fluid velocity u, intrinsic force F_int, mass m, reference
density rho0 (a = 1):

  force coupling, Crank-Nicolson midpoint force      Sec. 5.2, Eq. [modified-force]
      alpha = gamma s / m, beta = gamma s / rho0, D = 1 + alpha/2 + beta/2
      F^h = -[gamma (v - u) + (alpha/2) F_int] / D       (zeta = 0)
  original external boundary force                   Sec. 5.3, Eq. [ebf]
      force coupling with gamma = rho0 a^3 / h
  modified external boundary force                   Sec. 5.3, Eq. [modified-ebf]
      F^h = -gamma/(alpha+beta) (v - u) - alpha/(alpha+beta) F_int
          = -(v - u) / (s (1/m + 1/rho0)) - r F_int,  r = 1/(1 + m/rho0)
      (r is the immersion number of Eq. [immersion]; gamma cancels)
  first-order force coupling (the P S C F scheme)    Sec. 5.2
      F^h = -gamma (v - u)     (u held constant over the step)

A force half-step F^1/2 is the same formula with s = h/2 (Sec. 5.2, "a
half-step is achieved by substituting h by h/2").  The particle is then
kicked with v += (s/m)(F^h + F_int) (Alg. 3 writes dt/2 and drops 1/m_i;
read as the Newton equation of Sec. 5.2) and the fluid receives -F^h through
the spreading operator.

Intrinsic forces (the paper's CalculateForces, Alg. 2/3) are model input;
provided here: harmonic bonds U = k/2 (|d| - r0)^2 between listed pairs
(minimum-image distance on periodic axes), a constant external force per
particle, and rigid bodies made of tethered markers (below).  All are
pairwise, external, or sum to zero per body, so sum F_int has no internal
part.

Rigid bodies (a model; the paper has none): body b owns markers
first_b .. first_b + count_b - 1 with reference sites q_k (body frame,
centred: sum q_k = 0).  Its frame is the least-squares fit of the markers,
  X_b = mean of the markers (unwrapped around the first one),
  R_b = the rotation closest to A = sum_k (y_k - X_b) q_k^T (polar factor,
        from the SVD A = U S V^T: R = U diag(1, 1, det(U V^T)) V^T),
and every marker is tethered to its site by a spring,
  F_k = -k_t (y_k - X_b - R_b q_k).
X_b and R_b minimise U = k_t/2 sum_k |y_k - X_b - R_b q_k|^2, so F = -grad U
and the reactions on the (massless) frame vanish: sum_k F_k = 0 and
sum_k (y_k - X_b) x F_k = 0.  Bodies whose surfaces come closer than one
lattice unit repel: gap = |X_c - X_b| - (rad_b + rad_c), for gap < 1 a
force k_rep (1 - gap) along the centre line on each (opposite signs),
shared equally by the body's markers.
"""
import numpy as np

KINDS = ('none', 'ibm', 'fc', 'ebf', 'mebf')


def wrap_positions(pos, shape, walls):
    """Wrap x, y (and z unless walls) into [0, n): r = fmod(X, n), +n if < 0,
    -n if the result rounded up to n."""
    nz, ny, nx = shape
    out = pos.copy()
    for a, n in enumerate((nx, ny, nz)):
        if a == 2 and walls:
            continue
        r = np.fmod(out[:, a], n)
        r = np.where(r < 0.0, r + n, r)
        r = np.where(r >= n, r - n, r)
        out[:, a] = r
    return out


def min_image(d, shape, walls):
    nz, ny, nx = shape
    out = d.copy()
    for a, n in enumerate((nx, ny, nz)):
        if a == 2 and walls:
            continue
        out[:, a] = out[:, a] - n * np.rint(out[:, a] / n)
    return out


class RigidBodies:
    """Bodies of tethered markers: first (B,), count (B,), reference sites
    ref (M, 3) relative to the body centre (centred per body), tether
    stiffness k_t, repulsion stiffness k_rep, radius (B,)."""

    def __init__(self, first, count, ref, k_t, k_rep, radius):
        self.first = np.array(first, dtype=np.int64).reshape(-1)
        self.count = np.array(count, dtype=np.int64).reshape(-1)
        self.ref = np.array(ref, dtype=np.float64).reshape(-1, 3)
        self.k_t = float(k_t)
        self.k_rep = float(k_rep)
        self.radius = np.broadcast_to(np.asarray(radius, dtype=np.float64),
                                      self.first.shape).copy()

    @staticmethod
    def from_positions(pos, first, count, k_t, k_rep, radius, shape, walls):
        """Reference sites from a configuration taken as the rest shape."""
        ref = np.zeros((pos.shape[0], 3))
        for f, c in zip(first, count):
            y = _unwrapped(pos[f:f + c], shape, walls)
            ref[f:f + c] = y - y.mean(axis=0)
        return RigidBodies(first, count, ref, k_t, k_rep, radius)

    def copy(self):
        return RigidBodies(self.first, self.count, self.ref, self.k_t, self.k_rep,
                           self.radius)


def _unwrapped(x, shape, walls):
    """Marker positions of one body as a connected set: the first one as
    is, the others at their minimum image relative to it."""
    return x[0] + min_image(x - x[0], shape, walls)


def rigid_frames(bodies, pos, shape, walls):
    """Centre X (B, 3) and rotation R (B, 3, 3) of every body, and the
    unwrapped marker positions y (M, 3)."""
    B = bodies.first.shape[0]
    X = np.zeros((B, 3))
    R = np.zeros((B, 3, 3))
    y = pos.copy()
    for b in range(B):
        f, c = bodies.first[b], bodies.count[b]
        yb = _unwrapped(pos[f:f + c], shape, walls)
        y[f:f + c] = yb
        X[b] = yb.mean(axis=0)
        A = (yb - X[b]).T @ bodies.ref[f:f + c]
        U, _, Vt = np.linalg.svd(A)
        d = np.sign(np.linalg.det(U @ Vt))
        R[b] = U @ np.diag([1.0, 1.0, d]) @ Vt
    return X, R, y


def rigid_forces(bodies, pos, shape, walls):
    """Tether forces of every marker plus the pairwise body repulsion."""
    F = np.zeros_like(pos)
    X, R, y = rigid_frames(bodies, pos, shape, walls)
    B = X.shape[0]
    for b in range(B):
        f, c = bodies.first[b], bodies.count[b]
        sites = X[b] + bodies.ref[f:f + c] @ R[b].T
        F[f:f + c] = -bodies.k_t * (y[f:f + c] - sites)
    for b in range(B):
        for c2 in range(b + 1, B):
            d = min_image((X[c2] - X[b])[None, :], shape, walls)[0]
            dist = np.sqrt(d @ d)
            gap = dist - (bodies.radius[b] + bodies.radius[c2])
            if gap < 1.0:
                fc = bodies.k_rep * (1.0 - gap) * d / dist        # on body c2
                F[bodies.first[c2]:bodies.first[c2] + bodies.count[c2]] += fc / bodies.count[c2]
                F[bodies.first[b]:bodies.first[b] + bodies.count[b]] -= fc / bodies.count[b]
    return F


class Particles:
    """Lagrangian points: positions, velocities, masses, bonds, external
    force, rigid bodies."""

    def __init__(self, pos, vel=None, mass=None, bonds=None, bond_k=None,
                 bond_r0=None, ext_force=None, rigid=None):
        self.pos = np.array(pos, dtype=np.float64).reshape(-1, 3)
        M = self.pos.shape[0]
        self.vel = np.zeros((M, 3)) if vel is None else \
            np.array(vel, dtype=np.float64).reshape(M, 3)
        self.mass = np.ones(M) if mass is None else \
            np.array(mass, dtype=np.float64).reshape(M)
        self.bonds = np.zeros((0, 2), dtype=np.int64) if bonds is None else \
            np.array(bonds, dtype=np.int64).reshape(-1, 2)
        nb = self.bonds.shape[0]
        self.bond_k = np.zeros(nb) if bond_k is None else \
            np.broadcast_to(np.asarray(bond_k, dtype=np.float64), (nb,)).copy()
        self.bond_r0 = np.zeros(nb) if bond_r0 is None else \
            np.broadcast_to(np.asarray(bond_r0, dtype=np.float64), (nb,)).copy()
        self.ext_force = np.zeros((M, 3)) if ext_force is None else \
            np.array(ext_force, dtype=np.float64).reshape(M, 3)
        self.rigid = rigid

    def copy(self):
        return Particles(self.pos, self.vel, self.mass, self.bonds, self.bond_k,
                         self.bond_r0, self.ext_force,
                         None if self.rigid is None else self.rigid.copy())


def intrinsic_forces(parts, pos, shape, walls):
    """F_int(X): harmonic bonds, constant external forces, rigid bodies."""
    F = parts.ext_force.copy()
    if parts.rigid is not None:
        F += rigid_forces(parts.rigid, pos, shape, walls)
    if parts.bonds.shape[0]:
        i, j = parts.bonds[:, 0], parts.bonds[:, 1]
        d = min_image(pos[j] - pos[i], shape, walls)
        dist = np.sqrt((d * d).sum(axis=1))
        mag = parts.bond_k * (dist - parts.bond_r0) / dist
        fij = d * mag[:, None]             # force on i, pulling towards j
        np.add.at(F, i, fij)
        np.add.at(F, j, -fij)
    return F


def coupling_force(kind, order, v, u, Fint, mass, s, gamma, rho0,
                   include_int=True, zeta=None):
    """Hydrodynamic force F^h on each particle for a (sub-)step of length s.

    kind in ('fc', 'ebf', 'mebf'); v, u, Fint (M, 3); mass (M,).
    include_int=False gives the coupling-only operator F_h of the split in
    Sec. 6 (intrinsic forces integrated separately).  zeta (M, 3): the
    random force of Eq. [viscous-coupling], entering the midpoint force of
    Eq. [modified-force] as -[gamma (v - u) - zeta + alpha/2 F_int] / D, and
    the explicit first-order force as -gamma (v - u) + zeta.  The modified
    EBF takes none (its no-slip condition determines F^h).
    """
    m = mass[:, None]
    Fi = Fint if include_int else np.zeros_like(Fint)
    if kind == 'ebf':
        gamma = rho0 / 1.0          # gamma = rho a^3 / h with a = h = 1
    if kind == 'mebf':
        r = 1.0 / (1.0 + m / rho0)
        return -(v - u) / (s * (1.0 / m + 1.0 / rho0)) - r * Fi
    if order == 1:
        F = -gamma * (v - u)
        return F if zeta is None else F + zeta
    alpha = gamma * s / m
    beta = gamma * s / rho0
    D = 1.0 + 0.5 * alpha + 0.5 * beta
    if zeta is None:
        return -(gamma * (v - u) + 0.5 * alpha * Fi) / D
    return -((gamma * (v - u) + 0.5 * alpha * Fi) - zeta) / D
