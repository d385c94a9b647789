"""Pins of the oracle's rigid-body model (tethered markers on a best-fit
rigid frame, soft repulsion between bodies).

The pins do not restate the formulas: rigid motions carry no force, the
frame reactions vanish (force and torque), the forces are minus the
gradient of the tether energy (finite differences), the repulsion has the
stated magnitude and range, and a coupled run conserves total momentum.
"""
import numpy as np
import pytest

import synth
from oracle import coupling as CP
from oracle import lb as OL
from oracle import sim as OS

SHAPE = (24, 24, 24)          # (nz, ny, nx)


def _random_rotation(rng):
    Q, Rr = np.linalg.qr(rng.standard_normal((3, 3)))
    Q = Q * np.sign(np.diag(Rr))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def _bodies(rng, centres, radius=3.0, markers=40, k_t=0.7, k_rep=0.2):
    v = synth.fibonacci_sphere(markers)
    pos = np.concatenate([c + radius * v for c in centres])
    n = len(centres)
    first, count = np.arange(n) * markers, np.full(n, markers)
    body = CP.RigidBodies.from_positions(CP.wrap_positions(pos, SHAPE, False), first, count,
                                         k_t, k_rep, radius, SHAPE, False)
    return body, pos


def test_rigid_motions_carry_no_force():
    rng = np.random.default_rng(1)
    body, pos = _bodies(rng, [np.array([5.0, 6.0, 7.0]), np.array([15.0, 16.0, 17.0])])
    moved = pos.copy()
    for b in range(2):
        sl = slice(body.first[b], body.first[b] + body.count[b])
        c = pos[sl].mean(axis=0)
        Q = _random_rotation(rng)
        moved[sl] = c + (pos[sl] - c) @ Q.T + rng.uniform(-30, 30, 3)   # across the boundary
    F = CP.rigid_forces(body, CP.wrap_positions(moved, SHAPE, False), SHAPE, False)
    assert np.abs(F).max() < 1e-12


def test_frame_reactions_vanish():
    rng = np.random.default_rng(2)
    body, pos = _bodies(rng, [np.array([4.0, 12.0, 20.0]), np.array([14.0, 3.0, 9.0])])
    y = CP.wrap_positions(pos + 0.2 * rng.standard_normal(pos.shape), SHAPE, False)
    F = CP.rigid_forces(body, y, SHAPE, False)
    X, R, yu = CP.rigid_frames(body, y, SHAPE, False)
    for b in range(2):
        sl = slice(body.first[b], body.first[b] + body.count[b])
        assert np.abs(F[sl].sum(axis=0)).max() < 1e-12
        torque = np.cross(yu[sl] - X[b], F[sl]).sum(axis=0)
        assert np.abs(torque).max() < 1e-12
        assert abs(np.linalg.det(R[b]) - 1.0) < 1e-12
        assert np.abs(R[b] @ R[b].T - np.eye(3)).max() < 1e-12


def _energy(body, y):
    X, R, yu = CP.rigid_frames(body, y, SHAPE, False)
    U = 0.0
    for b in range(len(body.first)):
        sl = slice(body.first[b], body.first[b] + body.count[b])
        d = yu[sl] - X[b] - body.ref[sl] @ R[b].T
        U += 0.5 * body.k_t * (d * d).sum()
    return U


def test_forces_are_minus_the_energy_gradient():
    rng = np.random.default_rng(3)
    body, pos = _bodies(rng, [np.array([12.0, 12.0, 12.0])], radius=2.5, markers=12)
    y = pos + 0.15 * rng.standard_normal(pos.shape)
    F = CP.rigid_forces(body, y, SHAPE, False)
    eps = 1e-6
    G = np.zeros_like(y)
    for k in range(y.shape[0]):
        for a in range(3):
            yp, ym = y.copy(), y.copy()
            yp[k, a] += eps
            ym[k, a] -= eps
            G[k, a] = (_energy(body, yp) - _energy(body, ym)) / (2 * eps)
    assert np.abs(F + G).max() < 1e-7 * max(1.0, np.abs(F).max())


@pytest.mark.parametrize("gap,expect", [(0.4, 0.6), (0.99, 0.01), (1.0, 0.0), (1.5, 0.0)])
def test_repulsion_magnitude_and_range(gap, expect):
    rng = np.random.default_rng(4)
    radius = 3.0
    c0 = np.array([6.0, 11.0, 12.0])
    c1 = c0 + np.array([2 * radius + gap, 0.0, 0.0])
    body, pos = _bodies(rng, [c0, c1], radius=radius, k_rep=0.2)
    F = CP.rigid_forces(body, CP.wrap_positions(pos, SHAPE, False), SHAPE, False)
    f1 = F[body.first[1]:body.first[1] + body.count[1]].sum(axis=0)
    f0 = F[:body.count[0]].sum(axis=0)
    assert np.allclose(f1, [0.2 * expect, 0.0, 0.0], atol=1e-12)
    assert np.allclose(f0, -f1, atol=1e-12)


def test_coupled_run_conserves_momentum():
    rng = np.random.default_rng(5)
    shape = (16, 16, 16)
    v = synth.fibonacci_sphere(30)
    centres = [np.array([4.0, 5.0, 6.0]), np.array([11.0, 10.0, 9.5])]
    pos = CP.wrap_positions(np.concatenate([c + 2.0 * v for c in centres]), shape, False)
    first, count = np.array([0, 30]), np.array([30, 30])
    body = CP.RigidBodies.from_positions(pos, first, count, 0.5, 0.1, 2.0, shape, False)
    pos = pos + 0.05 * rng.standard_normal(pos.shape)         # not at rest shape
    parts = CP.Particles(CP.wrap_positions(pos, shape, False),
                         vel=0.005 * rng.standard_normal(pos.shape), mass=np.full(60, 0.6),
                         rigid=body)
    g = (2e-5, -1e-5, 0.0)
    p = OL.LBParams(collision="bgk", tau=0.8, body_force=g)
    sm = OS.Sim(shape, p, OS.CouplingParams("mebf", 2, "trilinear"), parts)
    P0 = sm.total_momentum()
    N = np.prod(shape)
    for t in range(1, 16):
        sm.step()
        assert np.allclose(sm.total_momentum(), P0 + t * N * np.array(g), rtol=0, atol=1e-12)
