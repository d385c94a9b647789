"""Rigid bodies of tethered markers on the GPU against the FP64 oracle: the
best-fit frames, tether forces and body repulsion enter F_int of the
modified-EBF coupling (tau = 0.7 through the recombined step).

FP64 storage: particles to 1e-11, fluid to 1e-10 (relative L2), total
momentum budget to 1e-12.  FP32 storage on the reduced rigid-sphere
workload (32^3, 8 spheres of radius 4.5 with 400 markers): bounds stated in
the test."""
import numpy as np
import pytest

import synth
from oracle import coupling as OC
from tests.gpu_helpers import make_pair, rel_l2, require_cuda

pytestmark = pytest.mark.gpu


def _two_bodies(shape, gap, seed, markers=60, radius=3.0):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    v = synth.fibonacci_sphere(markers)
    c0 = np.array([nx * 0.3, ny * 0.5, nz * 0.45])
    c1 = c0 + np.array([2 * radius + gap, 0.4, -0.3])
    rest = OC.wrap_positions(np.concatenate([c0 + radius * v, c1 + radius * v]), shape, False)
    first, count = np.array([0, markers]), np.array([markers, markers])
    body = OC.RigidBodies.from_positions(rest, first, count, 0.8, 0.3, radius, shape, False)
    pos = rest + 0.05 * rng.standard_normal(rest.shape)
    M = 2 * markers
    return dict(pos=pos, vel=0.004 * rng.standard_normal((M, 3)), mass=0.7,
                rigid=dict(first=first, count=count, radius=radius, k=0.8, repulsion_k=0.3,
                           ref=body.ref))


@pytest.mark.parametrize("gap", [0.5, 3.0])
@pytest.mark.parametrize("stencil", ["peskin4", "trilinear"])
def test_rigid_bodies_match_oracle_fp64(gap, stencil):
    require_cuda()
    shape = (20, 20, 24)
    fbar0 = synth.random_populations(shape, seed=3, amp=1e-3)
    parts = _two_bodies(shape, gap, seed=7)
    box, sm = make_pair(shape, fbar0, tau=0.7, storage="f64", kind="mebf", stencil=stencil,
                        parts=parts, g=(1e-5, 0, 0))
    for _ in range(12):
        sm.step()
    box.step(12)
    pos, vel, fh = box.get_particles()
    d = OC.min_image(pos - sm.parts.pos, shape, False)
    assert np.abs(d).max() < 1e-11
    assert np.abs(vel - sm.parts.vel).max() < 1e-11
    rho, u = box.get_fields()
    assert rel_l2(u, sm.fluid_velocity()) < 1e-10


def test_rigid_bodies_momentum_budget():
    require_cuda()
    shape = (20, 20, 24)
    g = (2e-5, -1e-5, 0.0)
    fbar0 = synth.random_populations(shape, seed=4, amp=1e-3)
    parts = _two_bodies(shape, 0.5, seed=9)
    box, sm = make_pair(shape, fbar0, tau=0.7, storage="f64", kind="mebf", stencil="peskin4",
                        parts=parts, g=g)
    _, P0, _ = box.invariants()
    N = np.prod(shape)
    box.step(20)
    _, P, st = box.invariants()
    assert st == 0
    expect = P0 + 20 * N * np.array(g)
    # the tether forces of a body sum to zero up to the roundoff of its
    # frame centre (a floating-point mean): about count * eps * |y| * k =
    # 60 * 1.1e-16 * 20 * 0.8 ~ 1e-13 per body and force evaluation, over
    # 2 bodies and 40 half steps: ~1e-11 (a real leak would be ~k * 0.05)
    assert np.abs(P - expect).max() < 2e-11, P - expect


def test_rigid_spheres_reduced_fp32():
    require_cuda()
    c = synth.config("mebf_rigid_spheres_128", scale=4)
    nx, ny, nz = c["box"]
    shape = (nz, ny, nx)
    pos, first, count = synth.rigid_spheres(c["nspheres"], c["radius"], c["markers"], c["box"],
                                            seed=c["seed"])
    body = OC.RigidBodies.from_positions(pos, first, count, c["rigid_k"], c["repulsion_k"],
                                         c["radius"], shape, False)
    mass = c["rho0"] * 4.0 / 3.0 * np.pi * c["radius"] ** 3 / c["markers"]
    rng = np.random.default_rng(1)
    parts = dict(pos=pos, vel=np.tile([0.002, 0.0, 0.0], (len(pos), 1)) +
                 0.001 * rng.standard_normal(pos.shape), mass=mass,
                 rigid=dict(first=first, count=count, radius=c["radius"], k=c["rigid_k"],
                            repulsion_k=c["repulsion_k"], ref=body.ref))
    fbar0 = synth.random_populations(shape, seed=2, amp=1e-4)
    box, sm = make_pair(shape, fbar0, tau=c["tau"], storage="f32", kind=c["kind"],
                        stencil=c["stencil"], parts=parts)
    steps = 15
    for _ in range(steps):
        sm.step()
    box.step(steps)
    p, v, fh = box.get_particles()
    d = OC.min_image(p - sm.parts.pos, shape, False)
    assert np.abs(d).max() < 1e-6
    assert rel_l2(v, sm.parts.vel) < 1e-4
    rho, u = box.get_fields()
    assert rel_l2(u, sm.fluid_velocity()) < 1e-4


def test_many_bodies_repel_across_the_periodic_boundary():
    """More bodies than a warp has lanes (each body's warp strides over the
    others), some pairs closer than one unit across the periodic faces
    (minimum image in the float screen and the double force)."""
    require_cuda()
    shape = (24, 24, 24)
    L = 24.0
    rng = np.random.default_rng(31)
    radius, markers = 1.5, 12
    centres = [np.array([0.4, 6.0, 6.0]), np.array([L - 2.9, 6.5, 6.2]),     # across x = 0
               np.array([12.0, 0.3, 18.0]), np.array([12.4, L - 2.8, 18.3]),  # across y = 0
               np.array([18.0, 18.0, 0.2]), np.array([18.2, 18.3, L - 3.0])]  # across z = 0
    while len(centres) < 40:
        c = rng.uniform(0.0, L, 3)
        d = [np.linalg.norm(OC.min_image((c - e)[None, :], shape, False)[0]) for e in centres]
        if min(d) > 2 * radius + 0.2:
            centres.append(c)
    v = synth.fibonacci_sphere(markers)
    rest = OC.wrap_positions(np.concatenate([c + radius * v for c in centres]), shape, False)
    B = len(centres)
    first, count = np.arange(B) * markers, np.full(B, markers)
    body = OC.RigidBodies.from_positions(rest, first, count, 0.8, 0.3, radius, shape, False)
    X, _, _ = OC.rigid_frames(body, rest, shape, False)
    close = 0
    for b in range(B):
        for c2 in range(b + 1, B):
            d = OC.min_image((X[c2] - X[b])[None, :], shape, False)[0]
            close += np.linalg.norm(d) - 2 * radius < 1.0
    assert close >= 3                      # the repulsion is exercised
    M = B * markers
    parts = dict(pos=rest + 0.02 * rng.standard_normal(rest.shape),
                 vel=0.003 * rng.standard_normal((M, 3)), mass=0.7,
                 rigid=dict(first=first, count=count, radius=radius, k=0.8, repulsion_k=0.3,
                            ref=body.ref))
    fbar0 = synth.random_populations(shape, seed=5, amp=1e-3)
    box, sm = make_pair(shape, fbar0, tau=0.7, storage="f64", kind="mebf", stencil="trilinear",
                        parts=parts)
    for _ in range(3):
        sm.step()
    box.step(3)
    pos, vel, _ = box.get_particles()
    assert np.abs(OC.min_image(pos - sm.parts.pos, shape, False)).max() < 1e-11
    assert np.abs(vel - sm.parts.vel).max() < 1e-11
