"""The node-moment field (LBC_OPT_NODE_MOMENTS) on the GPU.

After each LB step of a coupled step one pass stores j and 1 / rho of the
cells near markers; the interpolations up to the next LB step read them
instead of pulling 19 populations per stencil node (Eq. [IBM-interpolation]
needs only these moments and the force fields).  Both routes run the same
arithmetic, so a run with the field must equal the run without it bit for
bit, for every coupling scheme, stencil and storage format, across setters
that replace the populations or the particles, and inside a batch.
"""
import numpy as np
import pytest

import synth
from tests.gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu

STEPS = 7


def _case(name):
    """(lattice kwargs, coupling kwargs, particle kwargs) of a small case."""
    rng = np.random.default_rng(len(name) * 7919 + ord(name[0]))
    if name.startswith("ibm"):
        walls = name.endswith("walls")
        pos, bonds = synth.bead_chains(3, 8, (20, 16, 18), 1.0, seed=4)
        if walls:
            pos[:, 2] = 4.0 + np.mod(pos[:, 2], 10.0)
        lat = dict(nx=20, ny=16, nz=18, tau=0.9, walls=walls,
                   wall_velocity=((-0.02, 0, 0), (0.02, 0, 0)) if walls else ((0, 0, 0), (0, 0, 0)))
        cpl = dict(kind="ibm", order=2 if "order1" not in name else 1, stencil="peskin4")
        parts = dict(pos=pos, bonds=bonds, bond_k=0.05, bond_r0=1.0)
        return lat, cpl, parts
    M = 60
    pos = rng.uniform(0.0, 1.0, (M, 3)) * [22, 18, 20]
    vel = 0.01 * rng.standard_normal((M, 3))
    lat = dict(nx=22, ny=18, nz=20, tau=0.8, walls=False,
               wall_velocity=((0, 0, 0), (0, 0, 0)))
    table = {
        "mebf_p4": dict(kind="mebf", order=2, stencil="peskin4"),
        "fc_tri_order1": dict(kind="fc", order=1, stencil="trilinear", gamma=2.0),
        "fc_p3_outside": dict(kind="fc", order=2, stencil="peskin3", gamma=2.0,
                              split="outside", substeps=2),
        "ebf_p4_f64": dict(kind="ebf", order=2, stencil="peskin4"),
        "fc_p4_bf16": dict(kind="fc", order=2, stencil="peskin4", gamma=1.0),
    }
    cpl = table[name]
    parts = dict(pos=pos, vel=vel, mass=2.0)
    return lat, cpl, parts


STORAGE = {"ebf_p4_f64": "f64", "fc_p4_bf16": "bf16dev"}
NAMES = ["ibm_walls", "ibm_periodic", "ibm_order1", "mebf_p4", "fc_tri_order1",
         "fc_p3_outside", "ebf_p4_f64", "fc_p4_bf16"]


def _box(name, moments):
    from paper_1406_2211_gb300 import lbc
    lat, cpl, parts = _case(name)
    storage = STORAGE.get(name, "f32")
    ld = lbc.lattice_desc(lat["nx"], lat["ny"], lat["nz"], tau=lat["tau"], walls=lat["walls"],
                          wall_velocity=lat["wall_velocity"], storage=storage,
                          body_force=(1e-5, 0.0, 0.0))
    cd = lbc.coupling_desc(cpl["kind"], cpl["order"], cpl["stencil"], gamma=cpl.get("gamma", 1.0),
                           split=cpl.get("split", "base"), substeps=cpl.get("substeps", 1))
    B = len(parts["bonds"]) if "bonds" in parts else 0
    box = lbc.Box(ld, cd, max_particles=len(parts["pos"]), max_bonds=B)
    box.set_option(lbc.LBC_OPT_NODE_MOMENTS, 1 if moments else 0)
    fbar = synth.random_populations((lat["nz"], lat["ny"], lat["nx"]), seed=21, amp=1e-3)
    box.set_populations(fbar)
    box.set_particles(parts["pos"], vel=parts.get("vel"), mass=parts.get("mass"),
                      bonds=parts.get("bonds"), bond_k=parts.get("bond_k"),
                      bond_r0=parts.get("bond_r0"))
    return box


def _state(box):
    return [box.get_populations()] + list(box.get_particles())


def _assert_same(a, b, what):
    assert len(a) == len(b)
    for k, (x, y) in enumerate(zip(a, b)):
        assert np.array_equal(x, y), (what, k, np.abs(x - y).max())


@pytest.mark.parametrize("name", NAMES)
def test_field_gives_identical_results(name):
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    on, off = _box(name, True), _box(name, False)
    assert on.get_option(lbc.LBC_OPT_NODE_MOMENTS) == 1
    assert off.get_option(lbc.LBC_OPT_NODE_MOMENTS) == 0
    on.step(STEPS)
    off.step(STEPS)
    # more launches in the (first) step counted: the pass after the LB step
    # and a brick listing after each sort (a no-op unless the markers were
    # re-binned); the split with the coupling outside sorts twice in its
    # first step
    sorts = 2 if _case(name)[1].get("split") == "outside" else 1
    assert on.launches_per_step() == off.launches_per_step() + 1 + sorts
    _assert_same(_state(on), _state(off), name)


@pytest.mark.parametrize("name", ["ibm_walls", "mebf_p4", "fc_p4_bf16"])
def test_setters_between_steps_invalidate_the_field(name):
    require_cuda()
    lat, _, parts = _case(name)
    shape = (lat["nz"], lat["ny"], lat["nx"])
    fnew = synth.random_populations(shape, seed=33, amp=2e-3)
    moved = np.asarray(parts["pos"]) + 0.3
    out = []
    for moments in (True, False):
        box = _box(name, moments)
        box.step(3)
        box.set_populations(fnew)          # the field now lags the populations
        box.step(2)
        box.set_particles(moved, vel=parts.get("vel"), mass=parts.get("mass"),
                          bonds=parts.get("bonds"), bond_k=parts.get("bond_k"),
                          bond_r0=parts.get("bond_r0"))
        box.step(3)
        out.append(_state(box))
    _assert_same(out[0], out[1], name)


def test_toggling_mid_run():
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    ref = _box("mebf_p4", False)
    ref.step(9)
    box = _box("mebf_p4", True)
    box.step(3)
    box.set_option(lbc.LBC_OPT_NODE_MOMENTS, 0)
    box.step(3)                                  # the field falls behind
    box.set_option(lbc.LBC_OPT_NODE_MOMENTS, 1)  # and must not be read stale
    box.step(3)
    _assert_same(_state(box), _state(ref), "toggle")


def test_eager_launches_match_graphs():
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    a, b = _box("ibm_walls", True), _box("ibm_walls", True)
    b.set_option(lbc.LBC_OPT_GRAPHS, 0)
    a.step(STEPS)
    b.step(STEPS)
    _assert_same(_state(a), _state(b), "graphs")


def test_default_follows_the_node_count():
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    lat = lbc.lattice_desc(64, 64, 64)
    dense = lbc.Box(lat, lbc.coupling_desc("mebf", 2, "peskin4"), max_particles=4000)
    sparse = lbc.Box(lat, lbc.coupling_desc("fc", 2, "trilinear", gamma=1.0), max_particles=100)
    multi = lbc.Box(lat, lbc.coupling_desc("fc", 2, "trilinear", gamma=1.0, split="inside",
                                           substeps=4), max_particles=100000)
    assert dense.get_option(lbc.LBC_OPT_NODE_MOMENTS) == 1
    assert sparse.get_option(lbc.LBC_OPT_NODE_MOMENTS) == 0
    assert multi.get_option(lbc.LBC_OPT_NODE_MOMENTS) == 0
    with pytest.raises(lbc.LBCError):          # the multistep split caches per marker
        multi.set_option(lbc.LBC_OPT_NODE_MOMENTS, 1)
    sparse.set_option(lbc.LBC_OPT_NODE_MOMENTS, 1)
    assert sparse.get_option(lbc.LBC_OPT_NODE_MOMENTS) == 1
    for option, bad in ((lbc.LBC_OPT_NODE_MOMENTS, 2), (lbc.LBC_OPT_GATHER_LANES, 3),
                        (lbc.LBC_OPT_GATHER_LANES, -1)):
        with pytest.raises(lbc.LBCError):
            sparse.set_option(option, bad)
    assert sparse.get_option(lbc.LBC_OPT_GATHER_LANES) == 0     # automatic by default


def test_batch_member_with_field_equals_alone():
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    import torch
    alone = _box("ibm_walls", True)
    alone.step(6)
    batch = lbc.Batch(3)
    boxes = [_box("ibm_walls", True), _box("mebf_p4", False), _box("fc_p4_bf16", True)]
    for bx in boxes:
        assert batch.add(bx, 6)
    while len(batch):
        batch.advance(4)
    torch.cuda.synchronize()
    _assert_same(_state(boxes[0]), _state(alone), "batch")
    for name, bx in zip(["mebf_p4", "fc_p4_bf16"], boxes[1:]):
        ref = _box(name, False)
        ref.step(6)
        _assert_same(_state(bx), _state(ref), name)
    batch.close()


@pytest.mark.parametrize("name", ["ibm_walls", "mebf_p4", "fc_p3_outside", "ebf_p4_f64"])
def test_one_and_four_lanes_agree(name):
    """The interpolation with one lane per marker and with four lanes differ
    only in the order of the floating-point sum over the stencil."""
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    out = []
    for lanes in (1, 4):
        box = _box(name, True)
        box.set_option(lbc.LBC_OPT_GATHER_LANES, lanes)
        assert box.get_option(lbc.LBC_OPT_GATHER_LANES) == lanes
        box.step(STEPS)
        out.append(_state(box))
    tol = 1e-12 if STORAGE.get(name) == "f64" else 2e-5
    for k, (x, y) in enumerate(zip(*out)):
        scale = max(np.abs(y).max(), 1e-30)
        assert np.abs(x - y).max() <= tol * scale, (name, k, np.abs(x - y).max() / scale)
