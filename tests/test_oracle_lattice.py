"""Pins for oracle/lattice.py against the lattice and Hermite identities.

The checks below are properties fixed by the mathematics (quadrature
isotropy, the moments listed in Sec. 2 and Eq. [force-moments] of the paper,
the exact-shift property of the half force step), not re-evaluations of the
oracle's own formulas.
"""
import itertools

import numpy as np
import pytest

from oracle import lattice as L
from oracle import lb


def test_velocity_set_and_weights():
    # 19 distinct velocities with |c|^2 in {0, 1, 2}, closed under c -> -c
    assert len({tuple(c) for c in L.C}) == 19
    c2 = (L.C ** 2).sum(axis=1)
    assert sorted(set(c2.tolist())) == [0, 1, 2]
    for i in range(19):
        assert np.all(L.C[L.OPP[i]] == -L.C[i])
    assert abs(L.W.sum() - 1.0) < 1e-15


def test_quadrature_isotropy():
    """sum w c_a c_b = cs2 delta; 4th moment = cs2^2 (dd + dd + dd); odd = 0."""
    cf = L.CF
    d = np.eye(3)
    assert np.allclose(np.einsum('i,ia->a', L.W, cf), 0, atol=1e-16)
    assert np.allclose(np.einsum('i,ia,ib->ab', L.W, cf, cf), L.CS2 * d,
                       atol=1e-16)
    assert np.allclose(np.einsum('i,ia,ib,ic->abc', L.W, cf, cf, cf), 0,
                       atol=1e-16)
    m4 = np.einsum('i,ia,ib,ic,id->abcd', L.W, cf, cf, cf, cf)
    iso = L.CS2 ** 2 * (np.einsum('ab,cd->abcd', d, d)
                        + np.einsum('ac,bd->abcd', d, d)
                        + np.einsum('ad,bc->abcd', d, d))
    assert np.allclose(m4, iso, atol=1e-16)


def test_equilibrium_moments(rng):
    """rho, rho u and Pi = rho cs2 I + rho u u of f^eq (Sec. 2)."""
    rho = 1.0 + 0.1 * rng.standard_normal(7)
    u = 0.05 * rng.standard_normal((3, 7))
    feq = L.equilibrium(rho, u)
    assert np.allclose(feq.sum(axis=0), rho, rtol=0, atol=1e-15)
    assert np.allclose(L.momentum(feq), rho * u, rtol=0, atol=1e-15)
    Pi = np.einsum('ia,ib,in->abn', L.CF, L.CF, feq)
    expect = L.CS2 * np.eye(3)[:, :, None] * rho + np.einsum('an,bn->abn', u, u) * rho
    assert np.allclose(Pi, expect, rtol=0, atol=1e-15)


def test_force_term_moments(rng):
    """Eq. [force-moments]: sum G = 0, sum c G = F, sum c c G = F u + u F."""
    u = 0.05 * rng.standard_normal((3, 9))
    F = 1e-2 * rng.standard_normal((3, 9))
    G = L.force_term(u, F)
    assert np.allclose(G.sum(axis=0), 0, atol=1e-17)
    assert np.allclose(L.momentum(G), F, rtol=0, atol=1e-17)
    Pi = np.einsum('ia,ib,in->abn', L.CF, L.CF, G)
    expect = np.einsum('an,bn->abn', F, u) + np.einsum('an,bn->abn', u, F)
    assert np.allclose(Pi, expect, rtol=0, atol=1e-17)


def test_half_force_step_is_exact_equilibrium_shift(rng):
    """F^s with the midpoint-velocity G maps f^eq(rho,u) to f^eq(rho,u+sF/rho)
    and leaves f - f^eq unchanged (Sec. 3.3, statement after
    Eq. [LB-force-moments], exact for this choice of G)."""
    shape = (2, 3, 4)
    rho = 1.0 + 0.05 * rng.standard_normal(shape)
    u = 0.05 * rng.standard_normal((3,) + shape)
    F = 1e-2 * rng.standard_normal((3,) + shape)
    neq = 1e-3 * rng.standard_normal((19,) + shape)
    neq -= neq.mean(axis=0)          # remove mass
    # remove momentum from neq: project out c components with the weights
    j = L.momentum(neq)
    neq -= np.einsum('i,ia,a...->i...', L.W, L.CF, j) / L.CS2
    assert np.abs(L.momentum(neq)).max() < 1e-17
    f = L.equilibrium(rho, u) + neq
    for s in (0.5, 1.0):
        g = lb.force_step(f, F, s)
        u_new = u + s * F / rho
        assert np.abs(g - (L.equilibrium(rho, u_new) + neq)).max() < 2e-16


def test_mrt_basis_orthogonal_full_rank():
    E, b = L.MRT_E, L.MRT_B
    gram = E @ np.diag(L.W) @ E.T
    assert np.abs(gram - np.diag(b)).max() < 1e-15
    assert np.linalg.matrix_rank(E) == 19
    assert np.all(E[0] == 1) and np.all(E[1:4] == L.CF.T)
    # conserved rows are the density and momentum moments
    assert list(L.MRT_GROUP[:4]) == [0, 0, 0, 0]


def test_mrt_second_order_modes_span_stress():
    """Moments 4..9 are a basis of the symmetric second-rank tensors c c,
    i.e. (with 1) they carry exactly the stress."""
    cf = L.CF
    pairs = list(itertools.combinations_with_replacement(range(3), 2))
    cc = np.array([cf[:, a] * cf[:, b] for a, b in pairs])      # 6 x 19
    span = np.vstack([L.MRT_E[0:1], L.MRT_E[4:10]])            # 7 x 19
    both = np.vstack([span, cc])
    assert np.linalg.matrix_rank(span) == 7
    assert np.linalg.matrix_rank(both) == 7
