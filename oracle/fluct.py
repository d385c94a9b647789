"""Fluctuating MRT collision (Sec. 3.2, Eq. [mrt-fluct]) and its random
numbers, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Random numbers.  A counter-based generator, so that any cell's draws at any
step can be recomputed on their own: Philox4x32 with ten rounds, written
from its published definition (Salmon, Moraes, Dror and Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC 2011).  Each round multiplies words
0 and 2 of the 128-bit counter by two fixed odd 32-bit constants, keeps the
high and low halves of the 64-bit products, and mixes them with the other
two words and the 64-bit key; the key advances by two fixed Weyl increments
between rounds.  Uniforms in (0, 1) are (x + 1/2) 2^-32 of the 32-bit
outputs; Gaussians come from pairs of uniforms by the Box-Muller transform.
Counter layout: (cell, step, stream, block), key = the two halves of the
seed; a cell's Gaussians for one collision are blocks 0.. of its counter.

Collision (Eq. [mrt-fluct]): in the moment basis of oracle.lattice, the
non-equilibrium part of every non-conserved moment relaxes and receives a
Gaussian kick,
    m_k^neq <- gamma_k m_k^neq + sqrt(rho) phi_k r_k,   gamma_k = 1 - lambda_k,
with mu = k_B T / (a^3 cs2).

Reading (the printed amplitude): the paper prints phi_k = sqrt(mu b_k
lambda_k^2).  Stationary fluctuations need the variance a mode loses by the
relaxation, (1 - gamma_k^2) <m_k^2>, to be put back by the kick, and the
equilibrium variance of a mode is mu rho b_k (equipartition: <j_x^2> =
rho k_B T / a^3 for the momentum mode, b = cs2).  So phi_k^2 = mu b_k
(1 - gamma_k^2) = mu b_k lambda_k (2 - lambda_k), the amplitude of the
references the paper cites for Eq. [mrt-fluct]; it equals the printed one
only at lambda_k = 1.  The tests pin the stationary variances, which the
printed amplitude misses (test_printed_amplitude_is_not_stationary).

Recombination: the force half steps leave m^neq unchanged and the noise
acts on non-conserved moments only, so two half collisions of eigenvalues
sqrt(gamma_k) with kicks of the half-step amplitude compose, in
distribution, to one full collision with the full-step amplitude (the
kicks' variances add as gamma mu b (1 - gamma) + mu b (1 - gamma) =
mu b (1 - gamma^2)).  step_recombined_fluct uses one kick per step;
step_literal_fluct applies the two half steps.
"""
import numpy as np

from . import lattice as L
from . import lb as OL

_M0, _M1 = 0xD2511F53, 0xCD9E8D57            # round multipliers
_W0, _W1 = 0x9E3779B9, 0xBB67AE85            # key increments
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32(counter, key, rounds=10):
    """Philox4x32-R.  counter: (4, n) integers < 2^32; key: 2 integers.
    Returns (4, n) uint32."""
    x = [np.asarray(c, dtype=np.uint64) & _MASK for c in counter]
    k0, k1 = np.uint64(key[0]) & _MASK, np.uint64(key[1]) & _MASK
    m0, m1 = np.uint64(_M0), np.uint64(_M1)
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + np.uint64(_W0)) & _MASK
            k1 = (k1 + np.uint64(_W1)) & _MASK
        p0 = m0 * x[0]                        # exact: both factors < 2^32
        p1 = m1 * x[2]
        x = [((p1 >> np.uint64(32)) ^ x[1] ^ k0) & _MASK, p1 & _MASK,
             ((p0 >> np.uint64(32)) ^ x[3] ^ k1) & _MASK, p0 & _MASK]
    return np.stack(x).astype(np.uint32)


def uniforms(cells, step, stream, block, seed):
    """Four uniforms in (0, 1) per counter (cell, step, stream, block):
    (4, n); block may be one value or one per cell."""
    cells = np.asarray(cells, dtype=np.uint64)
    n = cells.shape[0]
    ctr = [cells, np.full(n, step, dtype=np.uint64), np.full(n, stream, dtype=np.uint64),
           np.broadcast_to(np.asarray(block, dtype=np.uint64), (n,))]
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return (philox4x32(ctr, key).astype(np.float64) + 0.5) * 2.0 ** -32


def gaussians(cells, step, stream, count, seed):
    """count standard normal numbers per cell, (count, ncells): Box-Muller
    on the uniforms of blocks 0, 1, ... (block b gives Gaussians 4b .. 4b+3:
    uniforms 0, 1 make the cosine and sine pair 4b, 4b+1; uniforms 2, 3 the
    pair 4b+2, 4b+3)."""
    cells = np.asarray(cells, dtype=np.uint64)
    n = cells.shape[0]
    nblk = (count + 3) // 4
    blocks = np.repeat(np.arange(nblk, dtype=np.uint64), n)
    u = uniforms(np.tile(cells, nblk), step, stream, blocks, seed).reshape(4, nblk, n)
    out = np.empty((nblk, 4, n))
    for a, b, k in ((0, 1, 0), (2, 3, 2)):
        r = np.sqrt(-2.0 * np.log(u[a]))
        out[:, k] = r * np.cos(2.0 * np.pi * u[b])
        out[:, k + 1] = r * np.sin(2.0 * np.pi * u[b])
    return out.reshape(4 * nblk, n)[:count]


def particle_noise(nparticles, step, substep, s, gamma, kT, seed):
    """Random force zeta of the force coupling for one coupling (sub-)step of
    length s (Sec. 5.2, Eq. [viscous-coupling]): white noise of intensity
    <zeta_a(t) zeta_b(t')> = 2 k_B T gamma delta_ab delta(t - t') averaged
    over the step, i.e. independent normals of variance 2 k_B T gamma / s
    per component (the fluctuation-dissipation relation of the friction
    gamma).  Counter (particle index, step, 8 + substep, 0); the components
    are the first three Gaussians of the block.  Returns (M, 3)."""
    r = gaussians(np.arange(nparticles), step, 8 + substep, 3, seed)   # (3, M)
    return np.sqrt(2.0 * kT * gamma / s) * r.T


def amplitudes(gam, kT, printed=False):
    """phi_k for the eigenvalues gam_k = 1 - lambda_k (0 for the conserved
    moments).  printed=True takes the amplitude as printed in the paper,
    sqrt(mu b_k lambda_k^2) (for the negative test only)."""
    mu = kT / L.CS2
    gam = np.broadcast_to(np.asarray(gam, dtype=np.float64), (L.Q,))
    lam = 1.0 - gam
    var = mu * L.MRT_B * (lam * lam if printed else 1.0 - gam * gam)
    var = np.where(L.MRT_GROUP == 0, 0.0, var)
    return np.sqrt(var)


def _mode_gammas(p):
    """Full-step eigenvalues per moment (BGK: the same for every moment)."""
    return np.broadcast_to(np.asarray(p.gamma_full(), dtype=np.float64), (L.Q,)).copy()


def relax_fluct(f, gam, phi, noise):
    """Collision with kicks: moments of f - f^eq(f) relaxed by gam_k and
    kicked by sqrt(rho) phi_k noise_k (Eq. [mrt-fluct]).  noise (19, ...)."""
    rho = L.density(f)
    feq = L.equilibrium(rho, L.momentum(f) / rho)
    m = np.tensordot(L.MRT_E, f - feq, axes=([1], [0]))
    shape = (L.Q,) + (1,) * (f.ndim - 1)
    m = gam.reshape(shape) * m + np.sqrt(rho) * phi.reshape(shape) * noise
    return feq + np.tensordot(np.linalg.inv(L.MRT_E), m, axes=([1], [0]))


def _noise(shape, step, stream, seed, cells=None):
    """Standard normal kicks for the 19 moments of every cell (the four
    conserved ones are drawn and multiplied by phi = 0).  cells: the flat
    cell indices x + nx (y + ny z) that number the counters (default: the
    cells of this array in order; a block cut out of a larger box passes the
    indices the cells have there)."""
    ncell = int(np.prod(shape))
    idx = np.arange(ncell) if cells is None else np.asarray(cells).reshape(-1)
    r = gaussians(idx, step, stream, L.Q, seed)
    return r.reshape((L.Q,) + tuple(shape))


def step_recombined_fluct(fbar, Fa, Fb, p, kT, seed, step, printed=False, cells=None):
    """(O2) with thermal fluctuations: fbar_new(x + c) = f^eq(rho, u1) +
    E^-1 [gamma m^neq(u0) + sqrt(rho) phi r] (one kick of the full-step
    amplitude per step).  cells: as for _noise."""
    shape = fbar.shape[1:]
    g = p.g.reshape(3, 1, 1, 1)
    rho = L.density(fbar)
    u0 = L.momentum(fbar) / rho
    zero = np.zeros((3,) + shape)
    Fa = zero if Fa is None else Fa
    Fb = zero if Fb is None else Fb
    u1 = u0 + 0.5 * (Fa + Fb + 2.0 * g) / rho
    gam = _mode_gammas(p)
    phi = amplitudes(gam, kT, printed)
    m = np.tensordot(L.MRT_E, fbar - L.equilibrium(rho, u0), axes=([1], [0]))
    m = gam.reshape((L.Q, 1, 1, 1)) * m + np.sqrt(rho) * phi.reshape((L.Q, 1, 1, 1)) * \
        _noise(shape, step, 0, seed, cells)
    post = np.tensordot(np.linalg.inv(L.MRT_E), m, axes=([1], [0]))
    return OL.stream(L.equilibrium(rho, u1) + post, p)


def step_literal_fluct(fbar, Fa, Fb, p, kT, seed, step):
    """(O1) with thermal fluctuations: two half collisions of eigenvalues
    sqrt(gamma_k), each with its own kick of the half-step amplitude, around
    the two force half steps (valid for gamma_k >= 0)."""
    shape = fbar.shape[1:]
    g = p.g.reshape(3, 1, 1, 1)
    zero = np.zeros((3,) + shape)
    Fa = zero if Fa is None else Fa
    Fb = zero if Fb is None else Fb
    gh = np.broadcast_to(np.asarray(p.gamma_half(), dtype=np.float64), (L.Q,)).copy()
    phih = amplitudes(gh, kT)
    f = relax_fluct(fbar, gh, phih, _noise(shape, step, 1, seed))
    f = OL.force_step(f, Fa + g, 0.5)
    f = OL.force_step(f, Fb + g, 0.5)
    f = relax_fluct(f, gh, phih, _noise(shape, step, 2, seed))
    return OL.stream(f, p)
