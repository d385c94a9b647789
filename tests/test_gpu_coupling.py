"""GPU parity of the coupled step (all coupling kinds, orders, splittings and
stencils) against the FP64 oracle, plus invariants and determinism.

With FP64 population storage every part of the GPU path computes in FP64
(stencil weights, node velocities, spread force fields, particle update), so
particles and fluid agree with the oracle to roundoff accumulated over the
steps run here (1e-11 absolute on particle state, 1e-10 relative L2 on the
fluid velocity), and the total momentum budget holds to 1e-12.  With FP32
storage the interpolation/spreading arithmetic is FP32 (bounds stated in the
tests that use it).
"""
import numpy as np
import pytest

import synth
from oracle import coupling as OC
from tests.gpu_helpers import make_pair, rel_l2, require_cuda

pytestmark = pytest.mark.gpu


def _particles(shape, kind, seed, nchains=2, beads=5):
    nz, ny, nx = shape
    pos, bonds = synth.bead_chains(nchains, beads, (nx, ny, nz), 1.0, seed=seed)
    if kind == "ibm":
        return dict(pos=pos, bonds=bonds, bond_k=0.02, bond_r0=1.3)
    rng = np.random.default_rng(seed)
    M = len(pos)
    return dict(pos=pos, vel=0.01 * rng.standard_normal((M, 3)),
                mass=rng.uniform(0.5, 2.0, M), bonds=bonds, bond_k=0.3, bond_r0=1.0,
                ext=1e-4 * rng.standard_normal((M, 3)))


SCHEMES = [
    # kind, order, split, n, stencil
    ("fc", 2, "base", 1, "trilinear"),
    ("fc", 2, "base", 1, "peskin4"),
    ("fc", 2, "base", 1, "peskin3"),
    ("fc", 2, "inside", 2, "trilinear"),
    ("fc", 2, "outside", 2, "trilinear"),
    ("fc", 2, "outside", 1, "peskin4"),
    ("ebf", 2, "base", 1, "peskin4"),
    ("mebf", 2, "base", 1, "peskin4"),
    ("mebf", 2, "inside", 1, "trilinear"),
    ("fc", 1, "base", 1, "trilinear"),
    ("mebf", 1, "base", 1, "peskin3"),
    ("ibm", 2, "base", 1, "peskin4"),
    ("ibm", 2, "base", 1, "trilinear"),
    ("ibm", 1, "base", 1, "peskin4"),
]


@pytest.mark.parametrize("kind,order,split,n,stencil", SCHEMES)
@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("lanes", [4, 1])
def test_coupled_steps_match_oracle(kind, order, split, n, stencil, walls, lanes):
    """lanes: markers per lane group of the 4- and 3-point interpolation
    (both variants against the oracle)."""
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    if lanes == 1 and (stencil == "trilinear" or split == "inside"):
        pytest.skip("these interpolations always run one lane per marker")
    shape = (11, 10, 12)
    fbar0 = synth.random_populations(shape, seed=21, amp=1e-3)
    parts = _particles(shape, kind, seed=5)
    if walls:       # keep markers clear of the walls
        parts["pos"][:, 2] = 3.0 + np.mod(parts["pos"][:, 2], shape[0] - 6.0)
    uw = ((0.01, 0, 0), (-0.01, 0.005, 0)) if walls else ((0, 0, 0), (0, 0, 0))
    box, sm = make_pair(shape, fbar0, coll="mrt", tau=0.8, g=(1e-5, 0, -1e-5),
                        walls=walls, uw=uw, storage="f64", kind=kind, order=order,
                        stencil=stencil, gamma=1.7, split=split, n=n, parts=parts)
    box.set_option(lbc.LBC_OPT_GATHER_LANES, lanes)
    for nsteps in (1, 2, 3):
        box.step(nsteps)
        for _ in range(nsteps):
            sm.step()
        pos, vel, fh = box.get_particles()
        d = OC.min_image(pos - sm.parts.pos, shape, walls)
        assert np.abs(d).max() < 1e-11, np.abs(d).max()
        if kind != "ibm":
            assert np.abs(vel - sm.parts.vel).max() < 1e-11
            assert np.abs(fh - sm.last_Fh).max() < 1e-11
    _, u = box.get_fields()
    assert rel_l2(u, sm.fluid_velocity()) < 1e-10
    box.close()


FP32_SCHEMES = [("fc", 2, "base", 1, "trilinear"), ("fc", 2, "inside", 2, "trilinear"),
                ("fc", 2, "outside", 2, "peskin4"), ("mebf", 2, "base", 1, "peskin4"),
                ("ibm", 2, "base", 1, "peskin3"), ("fc", 1, "base", 1, "trilinear")]


@pytest.mark.parametrize("kind,order,split,n,stencil", FP32_SCHEMES)
@pytest.mark.parametrize("walls", [False, True])
def test_coupled_steps_fp32_match_oracle(kind, order, split, n, stencil, walls):
    """FP32 storage: the particle side then computes bond vectors and
    |d|^2 - r0^2 in double-float FP32 arithmetic, stencils from a float
    split of the FP64 positions, and the wrap tests on bit patterns.  The
    12 x 10 x 11 box makes the chains cross the periodic faces (minimum
    image inside the double-float bond vector).  Bounds: FP32 rounding of
    node velocities and forces (about 1e-9 per step here); a wrong image or
    stretch would show at 1e-4 or more.  The explicit first-order step
    runs at a friction where it is stable (gamma h (1/m + 1/rho) < 2), so
    rounding is not amplified from step to step."""
    require_cuda()
    shape = (11, 10, 12)
    fbar0 = synth.random_populations(shape, seed=21, amp=1e-3)
    parts = _particles(shape, kind, seed=5, nchains=3, beads=6)
    if walls:
        parts["pos"][:, 2] = 3.0 + np.mod(parts["pos"][:, 2], shape[0] - 6.0)
    else:                  # put a chain across each periodic face
        L = np.array([shape[2], shape[1], shape[0]], dtype=float)
        parts["pos"][:6] += L - parts["pos"][:6].mean(axis=0)
        parts["pos"] = np.mod(parts["pos"], L)
    uw = ((0.01, 0, 0), (-0.01, 0.005, 0)) if walls else ((0, 0, 0), (0, 0, 0))
    box, sm = make_pair(shape, fbar0, coll="mrt", tau=0.8, g=(1e-5, 0, -1e-5),
                        walls=walls, uw=uw, storage="f32", kind=kind, order=order,
                        stencil=stencil, gamma=1.7 if order == 2 else 0.4, split=split, n=n,
                        parts=parts)
    for nsteps in (1, 2, 3):
        box.step(nsteps)
        for _ in range(nsteps):
            sm.step()
        pos, vel, fh = box.get_particles()
        d = OC.min_image(pos - sm.parts.pos, shape, walls)
        assert np.abs(d).max() < 1e-7, np.abs(d).max()
        if kind != "ibm":
            assert np.abs(vel - sm.parts.vel).max() < 1e-7
            assert np.abs(fh - sm.last_Fh).max() < 1e-6 * max(1.0, np.abs(sm.last_Fh).max())
    _, u = box.get_fields()
    assert rel_l2(u, sm.fluid_velocity()) < 1e-5
    box.close()


@pytest.mark.parametrize("kind,order,split,n", [("fc", 2, "base", 1), ("fc", 2, "outside", 2),
                                                ("mebf", 2, "inside", 2), ("ibm", 2, "base", 1),
                                                ("fc", 1, "base", 1)])
def test_total_momentum_budget_on_gpu(kind, order, split, n):
    """Periodic box: fluid + particle momentum grows by exactly h g N per
    step (Sec. 5.2: the coupling conserves total momentum)."""
    require_cuda()
    shape = (12, 12, 12)
    fbar0 = synth.random_populations(shape, seed=3)
    parts = _particles(shape, kind, seed=8, nchains=4, beads=6)
    g = np.array([1e-5, -2e-5, 0.0])
    box, _ = make_pair(shape, fbar0, coll="bgk", tau=0.9, g=g, storage="f64", kind=kind,
                       order=order, stencil="peskin4", gamma=2.0, split=split, n=n,
                       parts=parts)
    m0, P0, _ = box.invariants()
    N = np.prod(shape)
    # external forces on the particles are the only other momentum source
    src = g * N + (parts["ext"].sum(axis=0) if "ext" in parts else 0.0)
    for t in (1, 3, 6):
        box.step(t if t == 1 else 2 if t == 3 else 3)
        m, P, st = box.invariants()
        assert st == 0
        assert abs(m - m0) < 1e-9
        assert np.abs(P - P0 - t * src).max() < 1e-12, (t, P - P0 - t * src)
    box.close()


def test_spreading_is_deterministic():
    """Same inputs, fresh boxes: bit-identical particles and fluid (no
    atomics: the summation order of the spreading is fixed)."""
    require_cuda()
    shape = (16, 16, 16)
    fbar0 = synth.random_populations(shape, seed=1)
    parts = _particles(shape, "fc", seed=2, nchains=6, beads=10)
    outs = []
    for _ in range(2):
        box, _ = make_pair(shape, fbar0, coll="mrt", tau=0.8, storage="f32", kind="fc",
                           stencil="peskin4", gamma=3.0, parts=parts)
        box.step(6)
        outs.append((box.get_populations(), box.get_particles()))
        box.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    for k in range(3):
        assert np.array_equal(outs[0][1][k], outs[1][1][k])


def test_point_particle_32_fp64():
    """32^3 FP64 BGK tau = 0.8, one particle with force coupling gamma = m = 1,
    trilinear, v0 = (0.01, 0, 0), the workload's full 1000 steps: second- and
    first-order schemes against the oracle, and conservation of m v0 in the
    periodic box."""
    require_cuda()
    c = synth.config("fc_point_particle_32")
    nx, ny, nz = c["box"]
    shape = (nz, ny, nx)
    from oracle import lattice as OLat
    fbar0 = OLat.equilibrium(np.ones(shape), np.zeros((3,) + shape))
    parts = dict(pos=np.array([c["particle"]]), vel=np.array([c["velocity"]]), mass=1.0)
    for order, steps in ((2, c["steps"]), (1, c["steps"])):
        box, sm = make_pair(shape, fbar0, coll="bgk", tau=c["tau"], storage="f64",
                            kind="fc", order=order, stencil="trilinear",
                            gamma=c["gamma"], parts=parts)
        for chunk in (1, steps // 2 - 1, steps - steps // 2):
            box.step(chunk)
            for _ in range(chunk):
                sm.step()
            pos, vel, _ = box.get_particles()
            assert np.abs(vel - sm.parts.vel).max() < 1e-13
            assert np.abs(pos - sm.parts.pos).max() < 1e-11
        m, P, _ = box.invariants()
        assert np.abs(P - np.array(c["velocity"])).max() < 1e-13
        box.close()


def test_reduced_mrt_bead_chains():
    """The 256^3 chain workload at 1/4 size: 64^3 MRT FP32, bead chains with
    k = 10 bonds, force coupling gamma = 5, body force 1e-6, the multiple
    time-step split of Sec. 6 (Eq. [multistep]) with n = 4 coupled sub-steps
    per half step, as in the full workload.  FP32 storage and FP32
    interpolation/spreading: 1e-6 on positions, 1e-5 relative L2 on
    velocities."""
    require_cuda()
    c = synth.config("mrt_bead_chains_256", scale=4)
    nx, ny, nz = c["box"]
    shape = (nz, ny, nx)
    pos, bonds = synth.bead_chains(c["nchains"], c["beads"], c["box"], c["bond_r0"],
                                   seed=c["seed"])
    parts = dict(pos=pos, vel=np.zeros_like(pos), mass=c["mass"], bonds=bonds,
                 bond_k=c["bond_k"], bond_r0=c["bond_r0"])
    from oracle import lattice as OLat
    fbar0 = OLat.equilibrium(np.ones(shape), np.zeros((3,) + shape))
    box, sm = make_pair(shape, fbar0, coll="mrt", tau=c["tau"], g=c["body_force"],
                        storage="f32", kind="fc", stencil="trilinear", gamma=c["gamma"],
                        split=c["mode"], n=c["substeps"], parts=parts)
    steps = 12
    box.step(steps)
    for _ in range(steps):
        sm.step()
    pos_g, vel_g, fh_g = box.get_particles()
    d = OC.min_image(pos_g - sm.parts.pos, shape, False)
    assert np.abs(d).max() < 1e-6
    assert rel_l2(vel_g, sm.parts.vel) < 1e-5
    _, u = box.get_fields()
    assert rel_l2(u, sm.fluid_velocity()) < 1e-5
    box.close()


@pytest.mark.slow
def test_bead_chains_32_tau08_1000_steps():
    """The 256^3 chain workload at 1/8 size (32^3, 4 chains of 50 beads: the
    same bead density), with a collision that relaxes: MRT at tau = 0.8 (shear
    eigenvalue 1 - 1/tau = -0.25; ghosts fully relaxed, as in the workload),
    FP32 deviations, Eq. [multistep] with n = 4, over 1000 steps.  The FP32
    accuracy bar on a coupled box: relative L2 error of the fluid velocity at
    most 1e-5 after 1000 steps; particle positions element by element within
    2e-6 (FP32 node velocities, a few 1e-7 relative, integrated over 1000
    steps of a drift of order 0.5 lattice units)."""
    require_cuda()
    c = synth.config("mrt_bead_chains_256", scale=8)
    nx, ny, nz = c["box"]
    shape = (nz, ny, nx)
    pos, bonds = synth.bead_chains(c["nchains"], c["beads"], c["box"], c["bond_r0"],
                                   seed=c["seed"])
    parts = dict(pos=pos, vel=np.zeros_like(pos), mass=c["mass"], bonds=bonds,
                 bond_k=c["bond_k"], bond_r0=c["bond_r0"])
    from oracle import lattice as OLat
    fbar0 = OLat.equilibrium(np.ones(shape), np.zeros((3,) + shape))
    box, sm = make_pair(shape, fbar0, coll="mrt", tau=0.8, g=c["body_force"],
                        storage="f32", kind="fc", stencil="trilinear", gamma=c["gamma"],
                        split=c["mode"], n=c["substeps"], parts=parts)
    steps = 1000
    box.step(steps)
    for _ in range(steps):
        sm.step()
    pos_g, vel_g, _ = box.get_particles()
    d = OC.min_image(pos_g - sm.parts.pos, shape, False)
    assert np.abs(d).max() < 2e-6, np.abs(d).max()
    assert rel_l2(vel_g, sm.parts.vel) < 1e-5
    _, u = box.get_fields()
    assert rel_l2(u, sm.fluid_velocity()) < 1e-5
    m, P, st = box.invariants()
    assert st == 0
    box.close()


def test_fast_markers_are_rebinned_in_graph_replays():
    """Markers moving 0.3 cells per step leave their 4^3 bins every few
    steps; the re-sorts then happen inside replayed graphs (device-side
    decision).  FP64 storage: trajectories equal the oracle's to roundoff."""
    require_cuda()
    shape = (16, 20, 24)
    rng = np.random.default_rng(12)
    M = 40
    pos = rng.uniform(0, 1, (M, 3)) * [24, 20, 16]
    vel = np.tile([0.3, -0.2, 0.1], (M, 1)) + 0.02 * rng.standard_normal((M, 3))
    parts = dict(pos=pos, vel=vel, mass=50.0)
    fbar0 = synth.random_populations(shape, seed=3, amp=1e-4)
    box, sm = make_pair(shape, fbar0, tau=0.9, storage="f64", kind="fc", order=2,
                        stencil="trilinear", gamma=0.05, parts=parts)
    steps = 40
    for _ in range(steps):
        sm.step()
    box.step(steps)
    p, v, _ = box.get_particles()
    assert np.abs(OC.min_image(p - sm.parts.pos, shape, False)).max() < 1e-11
    assert np.abs(v - sm.parts.vel).max() < 1e-12
    assert box.status() == 0
    disp = np.abs(OC.min_image(sm.parts.pos - OC.wrap_positions(pos, shape, False), shape, False))
    assert disp.max() > 8.0                     # markers crossed several bins


@pytest.mark.parametrize("M", [8000, 9000])
def test_single_block_and_multi_pass_sorts(M):
    """Up to 8192 markers the re-binning runs as one single-block launch,
    above it as radix passes plus the bins: both against the oracle, with
    markers fast enough to leave their bins (re-sorts in graph replays)."""
    require_cuda()
    shape = (20, 20, 24)
    rng = np.random.default_rng(M)
    pos = rng.uniform(0.0, 1.0, (M, 3)) * [24, 20, 20]
    parts = dict(pos=pos, vel=0.2 * rng.standard_normal((M, 3)), mass=2.0)
    fbar0 = synth.random_populations(shape, seed=2, amp=1e-3)
    box, sm = make_pair(shape, fbar0, tau=0.8, storage="f64", kind="fc", order=2,
                        stencil="trilinear", gamma=1.5, parts=parts)
    for nsteps in (1, 2, 4):
        box.step(nsteps)
        for _ in range(nsteps):
            sm.step()
    pos_g, vel_g, _ = box.get_particles()
    assert np.abs(OC.min_image(pos_g - sm.parts.pos, shape, False)).max() < 1e-11
    assert np.abs(vel_g - sm.parts.vel).max() < 1e-11
    assert box.status() == 0
    tile0 = np.floor(OC.wrap_positions(pos, shape, False) / 4.0)
    assert (np.floor(pos_g / 4.0) != tile0).any(axis=1).sum() > 100   # re-binned markers


@pytest.mark.parametrize("storage,stencil", [("f64", "trilinear"), ("f32", "trilinear"),
                                             ("f64", "peskin4"), ("f32", "peskin3")])
def test_long_axis_beyond_16_bit_stencil_bases(storage, stencil):
    """A 40000 x 4 x 4 box: stencil bases beyond 2^15 along x (kept as
    21-bit fields), markers on an exact node, at half-integers, around 2^15
    and across the periodic face, and bonds at their rest length at large
    coordinates (with FP32 compute the bond vector and |d|^2 - r0^2 are
    formed in double-float arithmetic from the FP64 positions; positions
    rounded to FP32, 0.004 apart at 37 000, would move the bond forces far
    beyond the 1e-7 bound), against the oracle.  The 4-cell axes fold the
    stencils onto themselves."""
    require_cuda()
    shape = (4, 4, 40000)
    fbar0 = synth.random_populations(shape, seed=3, amp=1e-3)
    pos = np.array([[0.0, 1.3, 2.2], [39999.5, 2.0, 0.5], [39999.9, 3.7, 1.1],
                    [20000.25, 0.2, 3.9], [32767.5, 1.5, 2.5], [32768.5, 2.5, 1.5],
                    [39000.0, 1.0, 1.0],
                    # a chain at its rest length far from the origin (and one
                    # bond across the periodic face): |d|^2 - r0^2 starts at 0
                    [37000.3, 2.1, 1.7], [37001.3, 2.1, 1.7], [37002.3, 2.1, 1.7],
                    [39999.6, 0.4, 3.0], [0.6, 0.4, 3.0]])
    rng = np.random.default_rng(7)
    parts = dict(pos=pos, vel=0.01 * rng.standard_normal(pos.shape), mass=np.ones(len(pos)),
                 bonds=np.array([[7, 8], [8, 9], [10, 11]]), bond_k=0.3, bond_r0=1.0)
    box, sm = make_pair(shape, fbar0, coll="mrt", tau=0.8, g=(1e-5, 0, 0), storage=storage,
                        kind="fc", stencil=stencil, gamma=1.0, parts=parts)
    tol = 1e-11 if storage == "f64" else 1e-7
    for _ in range(2):
        box.step(1)
        sm.step()
        p, v, fh = box.get_particles()
        assert np.abs(OC.min_image(p - sm.parts.pos, shape, False)).max() < tol
        assert np.abs(v - sm.parts.vel).max() < tol
        assert np.abs(fh - sm.last_Fh).max() < tol
    _, u = box.get_fields()
    assert rel_l2(u, sm.fluid_velocity()) < (1e-10 if storage == "f64" else 1e-5)
    box.close()


def test_coupled_box_without_particles_is_the_fluid_step():
    """A force-coupled box whose particle set is empty steps the fluid alone
    (second order: the body force's half steps), as the oracle without
    coupling does."""
    require_cuda()
    shape = (6, 7, 9)
    fbar0 = synth.random_populations(shape, seed=4, amp=1e-3)
    box, sm = make_pair(shape, fbar0, coll="bgk", tau=0.9, g=(2e-5, -1e-5, 0), storage="f64",
                        kind="fc", stencil="peskin4", gamma=1.0,
                        parts=dict(pos=np.zeros((0, 3)), vel=np.zeros((0, 3)), mass=np.ones(0)))
    _, ref = make_pair(shape, fbar0, coll="bgk", tau=0.9, g=(2e-5, -1e-5, 0), storage="f64")
    box.step(3)
    for _ in range(3):
        ref.step()
    assert box.nparticles == 0
    assert np.abs(box.get_populations() - ref.fbar).max() < 1e-13
    _, _, st = box.invariants()
    assert st == 0
    box.close()
