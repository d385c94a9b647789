"""Shared helpers for the GPU parity tests: build a library box and the
matching oracle simulation from one parameter set."""
import numpy as np

from oracle import coupling as OC
from oracle import lb as OL
from oracle import sim as OS


def require_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)


def make_pair(shape, fbar0, coll="bgk", tau=0.8, lam=(0, 0, 0, 0), g=(0, 0, 0),
              walls=False, uw=((0, 0, 0), (0, 0, 0)), storage="f64", kind="none",
              order=2, stencil="trilinear", gamma=1.0, split="base", n=1,
              parts=None, rho0=1.0, graphs=True, storage_scale=0.0):
    """(library Box, oracle Sim) with identical inputs.

    parts: dict(pos, vel, mass, bonds, bond_k, bond_r0, ext) or None.
    """
    from paper_1406_2211_gb300 import lbc
    nz, ny, nx = shape
    lat = lbc.lattice_desc(nx, ny, nz, collision=coll, tau=tau, mrt_lambda=lam,
                           rho0=rho0, body_force=g, walls=walls, wall_velocity=uw,
                           storage=storage, storage_scale=storage_scale)
    cpl = lbc.coupling_desc(kind, order, stencil, gamma=gamma, split=split, substeps=n)
    M = 0 if parts is None else len(parts["pos"])
    B = 0 if parts is None or parts.get("bonds") is None else len(parts["bonds"])
    box = lbc.Box(lat, cpl, max_particles=max(M, 1) if kind != "none" else 0,
                  max_bonds=B)
    if not graphs:
        box.set_option(lbc.LBC_OPT_GRAPHS, 0)
    box.set_populations(fbar0)
    p = OL.LBParams(collision=coll, tau=tau, mrt_lambda=lam, rho0=rho0, body_force=g,
                    walls=walls, u_bot=uw[0], u_top=uw[1])
    oparts = None
    if parts is not None:
        rig = parts.get("rigid")
        box.set_particles(parts["pos"], vel=parts.get("vel"), mass=parts.get("mass"),
                          ext_force=parts.get("ext"), bonds=parts.get("bonds"),
                          bond_k=parts.get("bond_k"), bond_r0=parts.get("bond_r0"), rigid=rig)
        M = len(parts["pos"])
        mass = parts.get("mass")
        orig = None if rig is None else OC.RigidBodies(rig["first"], rig["count"], rig["ref"],
                                                        rig["k"], rig.get("repulsion_k", 0.0),
                                                        rig["radius"])
        oparts = OC.Particles(OC.wrap_positions(np.asarray(parts["pos"], float), shape, walls),
                              vel=parts.get("vel"),
                              mass=None if mass is None else np.broadcast_to(mass, (M,)),
                              bonds=parts.get("bonds"), bond_k=parts.get("bond_k"),
                              bond_r0=parts.get("bond_r0"), ext_force=parts.get("ext"),
                              rigid=orig)
    mode = {"base": "base", "inside": "inside", "outside": "outside"}[split]
    sm = OS.Sim(shape, p, OS.CouplingParams(kind, order, stencil, gamma=gamma,
                                            substeps=n, mode=mode),
                oparts, fbar=fbar0.copy())
    return box, sm


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
