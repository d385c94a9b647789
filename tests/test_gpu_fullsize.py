"""Parity at the full size of the 256^3 bead-chain workload, in the launch
configuration the benchmark times (MRT with fully relaxed ghosts, FP32
deviations, the force-field variant of the fused LB kernel, autotuned block
shape).

* One LB step checked on sampled cells: the step is local (a cell's new
  populations come from the collisions at its 19 upstream neighbours), so the
  oracle's recombined step applied to the 3 x 3 x 3 neighbourhood of a cell,
  taken from the GPU's own input state, gives the exact result at its centre.
  Bound: FP32 arithmetic on deviations of order 1e-3 w_i, so 1e-7 absolute
  (a dropped or mis-signed term is of order 1e-6 to 1e-4).
* The coupled step over 20 steps: total mass conserved and the fluid plus
  particle momentum growing by exactly t g N (Eq. [fc-splitting] conserves
  momentum; the body force g acts on N cells), at FP32 roundoff.
"""
import numpy as np
import pytest

import synth
from oracle import lb as OL
from tests.gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu

NAME = "mrt_bead_chains_256"


def _lattice(lbc, c):
    nx, ny, nz = c["box"]
    return lbc.lattice_desc(nx, ny, nz, collision=c["collision"], tau=c["tau"], rho0=c["rho0"],
                            body_force=c["body_force"], storage=c["storage"])


def _coupling(lbc, c):
    return lbc.coupling_desc(c["kind"], 2, c["stencil"], gamma=c["gamma"], split=c["mode"],
                             substeps=c["substeps"])


@pytest.mark.parametrize("tau,storage", [(1.0, "f32"), (0.8, "f32"), (1.0, "f16dev"),
                                         (0.8, "bf16dev")])
def test_lb_step_256_on_sampled_cells(tau, storage):
    """tau = 1 is the workload's setting, where MRT with fully relaxed ghosts
    has every non-conserved eigenvalue 1 - lambda = 0 and the step is
    f^eq(u1) (the same as BGK at tau = 1); tau = 0.8 relaxes the stress with
    eigenvalue -0.25, so the kernel's non-equilibrium path is checked too.
    The 16-bit forms run the two-cell kernel of the bench's storage forms;
    each stored value is rounded stochastically to one of its two 16-bit
    neighbours, so their bound adds one spacing (FP16: 2^-10, BF16: 2^-7 of
    the scaled deviation, twice that below it)."""
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    from oracle import lattice as OLat
    c = dict(synth.config(NAME), tau=tau, storage=storage)
    nx, ny, nz = c["box"]
    shape = (nz, ny, nx)
    # force fields allocated, no particle set: the step is the LB step with
    # the pending force F_a (h/2) and the body force (h)
    box = lbc.Box(_lattice(lbc, c), _coupling(lbc, c), max_particles=1)
    box.autotune()
    box.set_populations(synth.random_populations(shape, seed=44, amp=1e-3))
    f0 = box.get_populations()                  # the stored FP32 state, exactly
    rng = np.random.default_rng(45)
    Fa = 1e-4 * rng.standard_normal((3,) + shape)
    box.set_pending_force(Fa)
    box.step(1)
    f1 = box.get_populations()
    box.close()
    p = OL.LBParams(collision=c["collision"], tau=c["tau"], rho0=c["rho0"],
                    body_force=c["body_force"])
    cells = rng.integers(0, [nz, ny, nx], size=(400, 3))
    corners = [[z, y, x] for z in (0, nz - 1) for y in (0, ny - 1) for x in (0, nx - 1)]
    cells[:len(corners)] = corners                # periodic wrap on every face
    sp = {"f32": 0.0, "f16dev": 2.0 ** -9, "bf16dev": 2.0 ** -6}[storage]
    w0 = (OLat.W * c["rho0"]).reshape(-1)
    worst = 0.0
    for z, y, x in cells:
        iz = (z + np.arange(-1, 2)) % nz
        iy = (y + np.arange(-1, 2)) % ny
        ix = (x + np.arange(-1, 2)) % nx
        loc = f0[:, iz][:, :, iy][:, :, :, ix]
        Floc = Fa[:, iz][:, :, iy][:, :, :, ix]
        out = OL.step_recombined(loc, Floc, None, p)[:, 1, 1, 1]
        tol = 1e-7 + sp * np.abs(out - w0)
        worst = max(worst, float((np.abs(out - f1[:, z, y, x]) / tol).max()))
    assert worst <= 1.0, worst


def test_thermal_lb_step_256_on_sampled_cells():
    """The fused thermal step (Eq. [mrt-fluct]) at the full size in the
    bench's launch configuration: 400 sampled cells (the eight corners
    among them) against the oracle's fluctuating step of their 3^3
    neighbourhoods, each cell's kicks drawn from the Philox counter of its
    flat index in the full box."""
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    from oracle import fluct as OF
    c = dict(synth.config(NAME), tau=0.8)
    nx, ny, nz = c["box"]
    shape = (nz, ny, nx)
    kT, seed = 1e-5, 2014
    box = lbc.Box(_lattice(lbc, c), _coupling(lbc, c), max_particles=1)
    box.autotune()
    box.set_populations(synth.random_populations(shape, seed=46, amp=1e-3))
    f0 = box.get_populations()
    box.set_thermal(kT, seed)
    box.step(1)                                   # the first step after the seed: counter 0
    f1 = box.get_populations()
    box.close()
    p = OL.LBParams(collision=c["collision"], tau=c["tau"], rho0=c["rho0"],
                    body_force=c["body_force"])
    rng = np.random.default_rng(47)
    cells = rng.integers(0, [nz, ny, nx], size=(400, 3))
    corners = [[z, y, x] for z in (0, nz - 1) for y in (0, ny - 1) for x in (0, nx - 1)]
    cells[:len(corners)] = corners
    err = 0.0
    for z, y, x in cells:
        iz = (z + np.arange(-1, 2)) % nz
        iy = (y + np.arange(-1, 2)) % ny
        ix = (x + np.arange(-1, 2)) % nx
        loc = f0[:, iz][:, :, iy][:, :, :, ix]
        flat = (iz[:, None, None] * ny + iy[None, :, None]) * nx + ix[None, None, :]
        out = OF.step_recombined_fluct(loc, None, None, p, kT, seed, 0, cells=flat)[:, 1, 1, 1]
        err = max(err, float(np.abs(out - f1[:, z, y, x]).max()))
    # FP32 arithmetic on deviations of 1e-3 and kicks of about 1e-2 x sqrt(mu)
    assert err < 1e-7, err


def test_stress_epilogue_256_on_sampled_cells():
    """The stress epilogue (Eq. [viscstress]) at the full size in the bench's
    launch configuration (tau = 0.8, so the stress relaxes): sampled cells
    of the written sigma against oracle.lb.viscous_stress of the state the
    step collided, and the step's populations unchanged by the epilogue on
    the same sampled cells against the plain step's oracle."""
    require_cuda()
    import torch
    from paper_1406_2211_gb300 import lbc
    c = dict(synth.config(NAME), tau=0.8)
    nx, ny, nz = c["box"]
    shape = (nz, ny, nx)
    box = lbc.Box(_lattice(lbc, c), _coupling(lbc, c), max_particles=1)
    box.autotune()
    box.set_populations(synth.random_populations(shape, seed=48, amp=1e-3))
    f0 = box.get_populations()
    sig = box.stress_output()
    box.step(1)
    torch.cuda.synchronize()
    rng = np.random.default_rng(49)
    cells = rng.integers(0, [nz, ny, nx], size=(400, 3))
    got = sig.cpu().numpy()
    f1 = box.get_populations()
    box.stress_output(False)
    box.close()
    p = OL.LBParams(collision=c["collision"], tau=c["tau"], rho0=c["rho0"],
                    body_force=c["body_force"])
    comp = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2))
    worst, worst_f = 0.0, 0.0
    for z, y, x in cells:
        ref = OL.viscous_stress(f0[:, z:z + 1, y:y + 1, x:x + 1], p)[:, :, 0, 0, 0]
        for k, (a, b) in enumerate(comp):
            worst = max(worst, abs(float(got[k, z, y, x]) - ref[a, b]))
        iz = (z + np.arange(-1, 2)) % nz
        iy = (y + np.arange(-1, 2)) % ny
        ix = (x + np.arange(-1, 2)) % nx
        loc = f0[:, iz][:, :, iy][:, :, :, ix]
        out = OL.step_recombined(loc, None, None, p)[:, 1, 1, 1]
        worst_f = max(worst_f, float(np.abs(out - f1[:, z, y, x]).max()))
    # FP32 sums of 19 deviations of 1e-3
    assert worst < 1e-8, worst
    assert worst_f < 1e-7, worst_f


def test_bead_chain_workload_256_mass_and_momentum():
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    c = synth.config(NAME)
    nx, ny, nz = c["box"]
    pos, bonds = synth.bead_chains(c["nchains"], c["beads"], c["box"], c["bond_r0"],
                                   seed=c["seed"])
    box = lbc.Box(_lattice(lbc, c), _coupling(lbc, c), max_particles=len(pos),
                  max_bonds=len(bonds))
    box.autotune()
    box.init_equilibrium(c["rho0"], (0.0, 0.0, 0.0))
    box.set_particles(pos, vel=np.zeros_like(pos), mass=c["mass"], bonds=bonds,
                      bond_k=c["bond_k"], bond_r0=c["bond_r0"])
    m0, P0, st0 = box.invariants()
    steps = 20
    box.step(steps)
    m1, P1, st1 = box.invariants()
    box.close()
    assert st0 == 0 and st1 == 0
    N = nx * ny * nz
    assert abs(m1 - m0) <= 1e-9 * m0
    expect = steps * np.asarray(c["body_force"]) * N
    assert np.abs(P1 - P0 - expect).max() <= 1e-3 * np.abs(expect).max(), (P1 - P0, expect)


@pytest.mark.parametrize("storage", ["f32", "bf16dev"])
def test_lb_step_192_walls_on_sampled_cells(storage):
    """The 192^3 shell configuration's LB variant (BGK, moving walls with
    halfway bounce-back in z, force fields): sampled interior and wall cells
    against the oracle.  A wall cell's neighbourhood is the two layers next
    to the wall, streamed with the oracle's walls (the other face of that
    two-layer box is not read).  BF16 stores each scaled deviation rounded
    stochastically to one of its two neighbours in BF16, so the bound is
    one BF16 spacing (at most 2^-6 of the exact value's magnitude) plus the
    FP32 bound."""
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    from oracle import lattice as OLat
    c = synth.config("ibm_shells_192")
    nx, ny, nz = c["box"]
    shape = (nz, ny, nx)
    uw = c["wall_velocity"]
    lat = lbc.lattice_desc(nx, ny, nz, collision=c["collision"], tau=c["tau"], rho0=c["rho0"],
                           walls=True, wall_velocity=uw, storage=storage)
    box = lbc.Box(lat, lbc.coupling_desc("ibm", 2, c["stencil"]), max_particles=1)
    box.autotune()
    box.set_populations(synth.random_populations(shape, seed=46, amp=1e-3))
    f0 = box.get_populations()
    rng = np.random.default_rng(47)
    Fa = 1e-4 * rng.standard_normal((3,) + shape)
    box.set_pending_force(Fa)
    box.step(1)
    f1 = box.get_populations()
    box.close()
    cells = rng.integers(0, [nz, ny, nx], size=(300, 3))
    cells[:100, 0] = 0                             # bottom wall layer
    cells[100:200, 0] = nz - 1                     # top wall layer
    w0 = (OLat.W * c["rho0"]).reshape(-1)
    worst = 0.0
    for z, y, x in cells:
        iy = (y + np.arange(-1, 2)) % ny
        ix = (x + np.arange(-1, 2)) % nx
        if z == 0:
            iz, zc, walls = np.array([0, 1]), 0, True
        elif z == nz - 1:
            iz, zc, walls = np.array([nz - 2, nz - 1]), 1, True
        else:
            iz, zc, walls = z + np.arange(-1, 2), 1, False
        pl = OL.LBParams(collision=c["collision"], tau=c["tau"], rho0=c["rho0"], walls=walls,
                         u_bot=uw[0], u_top=uw[1]) if walls else OL.LBParams(
                             collision=c["collision"], tau=c["tau"], rho0=c["rho0"])
        loc = f0[:, iz][:, :, iy][:, :, :, ix]
        Floc = Fa[:, iz][:, :, iy][:, :, :, ix]
        out = OL.step_recombined(loc, Floc, None, pl)[:, zc, 1, 1]
        got = f1[:, z, y, x]
        # one BF16 spacing: 2^-7 of the value, 2^-6 of the value below it
        tol = 1e-7 + (2.0 ** -6 * np.abs(out - w0) if storage == "bf16dev" else 0.0)
        worst = max(worst, float((np.abs(out - got) / tol).max()))
    assert worst <= 1.0, worst
