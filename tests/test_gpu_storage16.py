"""16-bit population storage (FP16 / BF16 deviations from w_i rho0, FP32
arithmetic) against the FP64 oracle.

The accuracy bar for 16-bit storage is a relative error of at most 1e-3 in
the Stokes drag and in the trajectories.  Two cases:

* a reduced immersed-shell case (the 192^3 shell workload at 1/4 size: a
  48^3 box between walls moving at -/+0.05, one icosphere shell of radius 8
  with 642 markers and 1920 springs, immersed boundary, Peskin 4-point
  stencil), started from the steady Couette profile: shell centroid and
  marker displacements;
* heavy force-coupled particles dragged through fluid at rest (Stokes drag):
  total and per-particle coupling force.

FP32 storage on the same cases is held to a much tighter bound, and 16-bit
runs are bitwise reproducible (the stochastic rounding draws its random
numbers from the stored values themselves).
"""
import numpy as np
import pytest

import synth
from oracle import lattice as OLat
from tests.gpu_helpers import make_pair, rel_l2, require_cuda

pytestmark = pytest.mark.gpu

SHELL_STEPS = 120
DRAG_STEPS = 150


def _periodic_delta(a, b, period):
    d = np.asarray(a) - np.asarray(b)
    return d - np.round(d / period) * period


def _shell_case():
    c = synth.config("ibm_shells_192", scale=4)
    nx, ny, nz = c["box"]
    shape = (nz, ny, nx)
    pos, edges, r0 = synth.shells(c["nshells"], c["radius"], c["box"], c["seed"],
                                  c["subdivisions"])
    uw = c["wall_velocity"]
    z = np.arange(nz)
    u = np.zeros((3,) + shape)
    u[0] = (uw[0][0] + (uw[1][0] - uw[0][0]) * (z + 0.5) / nz)[:, None, None]
    fbar0 = OLat.equilibrium(np.ones(shape), u)
    parts = dict(pos=pos, bonds=edges, bond_k=c["spring_k"], bond_r0=r0)
    return c, shape, fbar0, parts


@pytest.fixture(scope="module")
def shell_oracle():
    c, shape, fbar0, parts = _shell_case()
    _, sm = make_pair(shape, fbar0, coll="bgk", tau=c["tau"], walls=True,
                      uw=c["wall_velocity"], storage="f32", kind="ibm", order=2,
                      stencil="peskin4", parts=parts)
    for _ in range(SHELL_STEPS):
        sm.step()
    return sm


@pytest.mark.parametrize("storage,bound", [("f32", 1e-6), ("f16dev", 1e-3), ("bf16dev", 1e-3)])
def test_shell_trajectory(shell_oracle, storage, bound):
    require_cuda()
    c, shape, fbar0, parts = _shell_case()
    box, _ = make_pair(shape, fbar0, coll="bgk", tau=c["tau"], walls=True,
                       uw=c["wall_velocity"], storage=storage, kind="ibm", order=2,
                       stencil="peskin4", parts=parts)
    box.step(SHELL_STEPS)
    pos, _, _ = box.get_particles()
    period = np.array([shape[2], shape[1], 1e30])
    disp_o = _periodic_delta(shell_oracle.parts.pos, parts["pos"], period)
    err = _periodic_delta(pos, shell_oracle.parts.pos, period)
    assert np.linalg.norm(disp_o.mean(axis=0)) > 1.0          # the shell moved
    centroid = np.linalg.norm(err.mean(axis=0)) / np.linalg.norm(disp_o.mean(axis=0))
    markers = np.linalg.norm(err) / np.linalg.norm(disp_o)
    assert centroid <= bound, (storage, centroid)
    assert markers <= bound, (storage, markers)


def _drag_case():
    shape = (32, 32, 32)
    rng = np.random.default_rng(7)
    M = 16
    parts = dict(pos=rng.uniform(0.0, 32.0, (M, 3)), vel=np.tile([0.01, 0.0, 0.0], (M, 1)),
                 mass=1e4)
    fbar0 = OLat.equilibrium(np.ones(shape), np.zeros((3,) + shape))
    return shape, fbar0, parts


@pytest.fixture(scope="module")
def drag_oracle():
    shape, fbar0, parts = _drag_case()
    _, sm = make_pair(shape, fbar0, coll="bgk", tau=0.8, storage="f32", kind="fc",
                      order=2, stencil="trilinear", gamma=1.0, parts=parts)
    for _ in range(DRAG_STEPS):
        sm.step()
    return sm


@pytest.mark.parametrize("storage,bound", [("f32", 1e-6), ("f16dev", 1e-3), ("bf16dev", 1e-3)])
def test_stokes_drag(drag_oracle, storage, bound):
    require_cuda()
    shape, fbar0, parts = _drag_case()
    box, _ = make_pair(shape, fbar0, coll="bgk", tau=0.8, storage=storage, kind="fc",
                       order=2, stencil="trilinear", gamma=1.0, parts=parts)
    box.step(DRAG_STEPS)
    pos, _, fh = box.get_particles()
    Fo = drag_oracle.last_Fh
    total = np.linalg.norm(fh.sum(axis=0) - Fo.sum(axis=0)) / np.linalg.norm(Fo.sum(axis=0))
    assert total <= bound, (storage, total)
    assert rel_l2(fh, Fo) <= bound, storage
    disp_o = _periodic_delta(drag_oracle.parts.pos, parts["pos"], 32.0)
    traj = np.linalg.norm(_periodic_delta(pos, drag_oracle.parts.pos, 32.0)) / np.linalg.norm(disp_o)
    assert traj <= bound, (storage, traj)


@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
def test_16bit_runs_are_reproducible(storage):
    require_cuda()
    shape, fbar0, parts = _drag_case()
    out = []
    for _ in range(2):
        box, _ = make_pair(shape, fbar0, coll="bgk", tau=0.8, storage=storage, kind="fc",
                           order=2, stencil="trilinear", gamma=1.0, parts=parts)
        box.step(40)
        out.append((box.get_populations(), box.get_particles()))
    assert np.array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)


# ------------------------------------------------ two cells per thread
# Boxes whose rows are a multiple of 64 cells take the two-cells-per-thread
# kernel (packed loads and stores, paired FP32 arithmetic).  Its collision is
# the same IEEE single-precision arithmetic as the one-cell kernel with the
# multiply-adds written out, so the two agree to FP32 rounding; each stored
# value is then rounded stochastically with the same random bits, so they
# differ at most by one 16-bit spacing, where the FP32 difference crosses a
# rounding step.  Against the oracle, one step is within one 16-bit spacing
# plus the FP32 bound.
SPACING = {"f16dev": 2.0 ** -10, "bf16dev": 2.0 ** -7}


@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
@pytest.mark.parametrize("coll,lam,walls,forced", [
    ("bgk", (0, 0, 0, 0), False, True),
    ("bgk", (0, 0, 0, 0), True, False),
    ("mrt", (0, 1.3, 0, 0), False, False),        # ghosts fully relaxed
    ("mrt", (0, 0, 0, 0), True, True),
])
def test_pair_kernel_matches_one_cell_kernel_and_oracle(storage, coll, lam, walls, forced):
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    from oracle import lb as OL
    shape = (10, 12, 128)                     # nx = 128: two warps of 64 cells per row
    nz, ny, nx = shape
    rng = np.random.default_rng(31)
    Fa = 1e-4 * rng.standard_normal((3,) + shape) if forced else None
    uw = ((0.02, 0, 0), (-0.01, 0.01, 0)) if walls else ((0, 0, 0), (0, 0, 0))
    outs = {}
    for pair in (1, 0):
        lat = lbc.lattice_desc(nx, ny, nz, collision=coll, tau=0.85, mrt_lambda=lam,
                               body_force=(1e-5, 0, -2e-6), walls=walls, wall_velocity=uw,
                               storage=storage)
        box = lbc.Box(lat, lbc.coupling_desc("fc", 2, "trilinear"), max_particles=1)
        box.set_option(lbc.LBC_OPT_LB_PAIR, pair)
        assert box.get_option(lbc.LBC_OPT_LB_PAIR) == pair
        box.set_populations(synth.random_populations(shape, seed=32, amp=1e-3))
        f0 = box.get_populations()
        if forced:
            box.set_pending_force(Fa)
        box.step(1)
        outs[pair] = (f0, box.get_populations())
        box.close()
    f0, got = outs[1]
    assert np.array_equal(f0, outs[0][0])
    w0 = OLat.W.reshape(19, 1, 1, 1)
    # FP32 rounding of the two forms (contractions differ) moves a value by a
    # few 1e-9; FP16's spacing of a small deviation can be finer than that
    sp = SPACING[storage] * np.abs(outs[0][1] - w0)
    assert (np.abs(got - outs[0][1]) <= sp + 1e-7).all()
    p = OL.LBParams(collision=coll, tau=0.85, mrt_lambda=lam, body_force=(1e-5, 0, -2e-6),
                    walls=walls, u_bot=uw[0], u_top=uw[1])
    ref = OL.step_recombined(f0, Fa, None, p)
    if walls:
        # reading the state back rounds the bounced-back values of the wall
        # layers to 16 bits (the kernel uses them unrounded), and the step
        # streams them one layer inward: compare the layers beyond
        ref, got = ref[:, 2:-2], got[:, 2:-2]
    bound = 1e-7 + SPACING[storage] * np.abs(ref - w0)
    assert (np.abs(got - ref) <= bound).all(), float((np.abs(got - ref) / bound).max())
