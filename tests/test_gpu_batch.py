"""Batched stepping (lbc_batch_*) and the serving loop on the GPU.

A box advanced inside a batch, next to members of other sizes, storage
formats, coupling kinds and step budgets, must give exactly the results of
the same box advanced alone (same kernel bodies, same per-box arguments),
whether the members' particle work runs as one launch per operation or on
a stream per member, and the same results as stepping the box on its own
with lbc_box_step.
"""
import zlib

import numpy as np
import pytest

import synth
from tests.gpu_helpers import require_cuda

pytestmark = pytest.mark.gpu


def _spec(name):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if name == "fc32":
        return dict(shape=(24, 24, 24), storage="f32", kind="fc", stencil="trilinear", gamma=2.0,
                    pos=rng.uniform(0, 24, (30, 3)), vel=0.01 * rng.standard_normal((30, 3)))
    if name == "fc16":
        return dict(shape=(16, 32, 40), storage="f16dev", kind="fc", stencil="trilinear",
                    gamma=3.0, pos=rng.uniform(0, 16, (100, 3)) * [2.5, 2.0, 1.0],
                    vel=0.01 * rng.standard_normal((100, 3)))
    if name == "fluid":
        return dict(shape=(20, 20, 20), storage="f32", kind="none", g=(1e-5, 0, 0))
    if name == "ibm_walls":
        pos, bonds = synth.bead_chains(2, 6, (16, 16, 12), 1.0, seed=3)
        pos[:, 2] = 3.0 + np.mod(pos[:, 2], 6.0)
        return dict(shape=(12, 16, 16), storage="f32", kind="ibm", stencil="peskin4",
                    walls=True, uw=((-0.02, 0, 0), (0.02, 0, 0)), pos=pos, bonds=bonds)
    if name == "mrt_bf16":
        return dict(shape=(18, 20, 22), storage="bf16dev", kind="fc", stencil="peskin4",
                    coll="mrt", tau=1.0, gamma=1.0, pos=rng.uniform(2, 16, (20, 3)),
                    vel=0.005 * rng.standard_normal((20, 3)))
    raise KeyError(name)


def _make(spec):
    from paper_1406_2211_gb300 import lbc
    nz, ny, nx = spec["shape"]
    lat = lbc.lattice_desc(nx, ny, nz, collision=spec.get("coll", "bgk"),
                           tau=spec.get("tau", 0.8), body_force=spec.get("g", (0, 0, 0)),
                           walls=spec.get("walls", False),
                           wall_velocity=spec.get("uw", ((0, 0, 0), (0, 0, 0))),
                           storage=spec["storage"])
    cpl = lbc.coupling_desc(spec["kind"], 2, spec.get("stencil", "trilinear"),
                            gamma=spec.get("gamma", 1.0))
    M = len(spec["pos"]) if "pos" in spec else 0
    B = len(spec["bonds"]) if "bonds" in spec else 0
    box = lbc.Box(lat, cpl, max_particles=M, max_bonds=B)
    fbar = synth.random_populations(spec["shape"], seed=11, amp=1e-3)
    box.set_populations(fbar)
    if M:
        if spec["kind"] == "ibm":
            box.set_particles(spec["pos"], bonds=spec["bonds"], bond_k=0.05, bond_r0=1.0)
        else:
            box.set_particles(spec["pos"], vel=spec["vel"], mass=1.0)
    return box


def _state(box):
    out = [box.get_populations()]
    if box.nparticles:
        out.extend(box.get_particles())
    return out


def _same(a, b):
    return len(a) == len(b) and all(np.array_equal(x, y) for x, y in zip(a, b))


NAMES = ["fc32", "fc16", "fluid", "ibm_walls", "mrt_bf16"]
BUDGET = {"fc32": 9, "fc16": 5, "fluid": 12, "ibm_walls": 9, "mrt_bf16": 7}


def _run_batch(names, chunk, launch="auto"):
    from paper_1406_2211_gb300 import lbc
    import torch
    batch = lbc.Batch(8)
    batch.set_launch(launch)
    boxes = {n: _make(_spec(n)) for n in names}
    for n in names:
        assert batch.add(boxes[n], BUDGET[n])
    finished = []
    while len(batch):
        _, fin = batch.advance(chunk)
        finished.extend(fin)
    torch.cuda.synchronize()
    assert len(finished) == len(names)
    states = {n: _state(boxes[n]) for n in names}
    batch.close()
    return states


@pytest.fixture(scope="module")
def alone():
    require_cuda()
    return {n: _run_batch([n], chunk=4)[n] for n in NAMES}


def test_member_alone_equals_member_in_mix(alone):
    mixed = _run_batch(NAMES, chunk=4)
    for n in NAMES:
        assert _same(mixed[n], alone[n]), n


@pytest.mark.parametrize("launch", ["streams", "batched"])
def test_both_launch_forms_give_the_same_results(alone, launch):
    """The members' particle work as one launch per operation for all
    members (recorded steps, device argument tables) or on a stream per
    member: each member's results are those of the member alone, bit for
    bit, either way."""
    mixed = _run_batch(NAMES, chunk=4, launch=launch)
    for n in NAMES:
        assert _same(mixed[n], alone[n]), (n, launch)


def test_chunking_does_not_change_results(alone):
    mixed = _run_batch(NAMES, chunk=3)
    for n in NAMES:
        assert _same(mixed[n], alone[n]), n


def test_batch_matches_box_stepping(alone):
    for n in NAMES:
        box = _make(_spec(n))
        box.step(BUDGET[n])
        st = _state(box)
        ref = alone[n]
        for x, y in zip(st, ref):
            assert np.array_equal(x, y), n


def test_batch_rules():
    from paper_1406_2211_gb300 import lbc
    require_cuda()
    batch = lbc.Batch(2)
    a, b, c = (_make(_spec("fluid")) for _ in range(3))
    assert batch.add(a, 3) and batch.add(b, 3)
    assert not batch.add(c, 3)                     # no free slot
    with pytest.raises(lbc.LBCError):              # a member is stepped by its batch
        a.step(1)
    assert batch.remaining(a) == 3
    done, fin = batch.advance(2)
    assert done == 2 and not fin and batch.remaining(b) == 1
    batch.remove(b)
    b.step(1)                                      # free again
    done, fin = batch.advance(5)
    assert done == 1 and fin == [a] and len(batch) == 0
    batch.close()


def test_serving_loop_results_equal_alone_runs():
    require_cuda()
    import torch
    from paper_1406_2211_gb300 import lbc
    from paper_1406_2211_gb300.serve import BoxFactory, Job, JobServer, summary
    jobs_spec = synth.ensemble_jobs(6, seed=5, edge_range=(16, 40), particles_range=(1, 40),
                                    steps_range=(5, 25), rate=200.0)
    jobs = []
    for i, s in enumerate(jobs_spec):
        rng = np.random.default_rng(s["seed"])
        L = s["edge"]
        spec = dict(edge=L, gamma=s["gamma"], storage=s["storage"],
                    pos=rng.uniform(0, L, (s["nparticles"], 3)),
                    vel=0.01 * rng.standard_normal((s["nparticles"], 3)))
        jobs.append(Job(i, spec, s["arrival"], s["steps"], L ** 3))
    fac = BoxFactory()
    batch = lbc.Batch(3)
    srv = JobServer(fac, batch, memory_budget=2 ** 31, max_active=3, chunk_steps=4,
                    sync=torch.cuda.synchronize)
    done = srv.run(jobs)
    assert len(done) == 6 and srv.peak_active <= 3
    s = summary(done, srv.elapsed)
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0
    for j in done:                                  # the same job alone
        box = fac.create(j)
        solo = lbc.Batch(1)
        solo.add(box, j.steps)
        while len(solo):
            solo.advance(4)
        r = fac.result(box)
        for k in ("pos", "vel", "force_h"):
            assert np.array_equal(r[k], j.result[k]), (j.id, k)
        solo.close()
        fac.release(box)
    batch.close()


# ------------------------------------------------------------ failures
def test_nonfinite_box_is_latched_by_the_step_path():
    """A NaN population set from the host: the next LB step meets a
    non-finite density, lbc_box_check latches LBC_ERR_NONFINITE (without
    lbc_box_invariants), later steps refuse, and replacing the state clears
    it."""
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    spec = _spec("fc32")
    box = _make(spec)
    assert box.check() == 0
    f = box.get_populations()
    f[3, 5, 6, 7] = np.nan
    box.set_populations(f)
    box.step(2)
    assert box.check() == lbc.LBC_ERR_NONFINITE
    assert box.status() == lbc.LBC_ERR_NONFINITE
    with pytest.raises(lbc.LBCError):
        box.step(1)
    box.set_populations(synth.random_populations(spec["shape"], seed=11, amp=1e-3))
    assert box.check() == 0
    box.step(1)
    assert box.check() == 0
    box.close()


def test_failed_member_is_retired_while_the_others_finish():
    """One member of a batch gets a NaN population injected from the host.
    The batch retires it (reported as finished, status LBC_ERR_NONFINITE)
    without stopping the others, which end with exactly the results of the
    same boxes advanced in a batch without it."""
    require_cuda()
    from paper_1406_2211_gb300 import lbc
    names = ["fc32", "fluid", "mrt_bf16"]

    def run(inject):
        batch = lbc.Batch(4)
        boxes = {n: _make(_spec(n)) for n in names}
        if inject:
            bad = _make(_spec("fc16"))
            f = bad.get_populations()
            f[0, 1, 2, 3] = np.nan
            bad.set_populations(f)
            assert batch.add(bad, 40)
        for n in names:
            assert batch.add(boxes[n], BUDGET[n])
        finished = []
        while len(batch) > 0:
            _, fin = batch.advance(2)
            finished.extend(fin)
        batch.close()
        states = {n: _state(boxes[n]) for n in names}
        for b in boxes.values():
            assert b.check() == 0
            b.close()
        if inject:
            assert bad in finished
            assert bad.status() == lbc.LBC_ERR_NONFINITE
            bad.close()
        return states

    clean, mixed = run(False), run(True)
    for n in names:
        assert _same(clean[n], mixed[n]), n


def test_serving_reports_failed_and_rejected_jobs():
    """The serving loop on the GPU: a job whose box is set up with a NaN
    population ends as "failed" with the library's reason, a job whose box
    the batch refuses (x-rows longer than the batched launch takes) as
    "rejected", and the other jobs complete."""
    require_cuda()
    import torch
    from paper_1406_2211_gb300 import lbc
    from paper_1406_2211_gb300.serve import BoxFactory, Job, JobServer, summary

    class Injecting(BoxFactory):
        def create(self, job):
            box = super().create(job)
            if job.spec.get("nan"):
                f = box.get_populations()
                f[1, 2, 3, 4] = np.nan
                box.set_populations(f)
            return box

    rng = np.random.default_rng(3)
    jobs = []
    for i, (L, nan) in enumerate([(16, False), (20, True), (12, False), (130, False),
                                  (18, False)]):
        M = 5
        spec = dict(edge=L, storage="f32", gamma=2.0, pos=rng.uniform(0, L, (M, 3)),
                    vel=np.zeros((M, 3)), nan=nan)
        jobs.append(Job(i, spec, 0.0, 30, L ** 3))
    batch = lbc.Batch(8)
    srv = JobServer(Injecting(), batch, 2 ** 34, 8, chunk_steps=10, sync=torch.cuda.synchronize)
    done = srv.run(jobs)
    batch.close()
    by = {j.id: j for j in done}
    assert sorted(by) == [0, 1, 2, 3, 4]
    assert by[1].status.startswith("failed") and "non-finite" in by[1].status
    assert by[3].status.startswith("rejected")
    for i in (0, 2, 4):
        assert by[i].status == "ok" and np.isfinite(by[i].result["pos"]).all()
    s = summary(done, srv.elapsed)
    assert (s["jobs"], s["failed"], s["rejected"]) == (3, 1, 1)
