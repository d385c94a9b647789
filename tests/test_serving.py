"""Host logic of the serving loop (admission by memory and slots, continuous
batching, completion tracking, latency statistics) with stand-ins for the
boxes and the batch: a simulated clock advances with the work the batch
does, so every run is deterministic and needs no GPU."""
import numpy as np
import pytest

from paper_1406_2211_gb300.serve import Job, JobServer, summary


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeFactory:
    def __init__(self):
        self.live = {}
        self.created = []

    def bytes(self, job):
        return job.cells * 10

    def create(self, job):
        box = {"job": job.id, "steps": 0}
        self.live[id(box)] = box
        self.created.append(job.id)
        return box

    def result(self, box):
        return box["steps"]

    def release(self, box):
        del self.live[id(box)]


class FakeBatch:
    """Advances members together; the clock moves by the cell updates done
    at a fixed rate (1e6 cell updates per simulated second)."""

    def __init__(self, slots, clock):
        self.slots = slots
        self.clock = clock
        self.members = []         # [box, remaining]
        self.sizes = []
        self.cells = {}

    def add(self, box, steps):
        if len(self.members) >= self.slots:
            return False
        self.members.append([box, steps])
        return True

    def advance(self, k):
        if not self.members:
            return 0, []
        d = min(k, min(r for _, r in self.members))
        self.sizes.append(len(self.members))
        work = 0
        for m in self.members:
            m[0]["steps"] += d
            m[1] -= d
            work += self.cells[m[0]["job"]] * d
        self.clock.t += work / 1e6
        done = [m[0] for m in self.members if m[1] == 0]
        self.members = [m for m in self.members if m[1] > 0]
        return d, done


def _jobs(n, seed, rate):
    rng = np.random.default_rng(seed)
    arr = np.cumsum(rng.exponential(1.0 / rate, n)) if rate else np.zeros(n)
    out = []
    for i in range(n):
        L = int(rng.integers(8, 24))
        out.append(Job(i, {"edge": L}, arr[i], int(rng.integers(5, 60)), L ** 3))
    return out


def _run(jobs, slots=4, budget=None, chunk=7):
    clock = Clock()
    fac = FakeFactory()
    batch = FakeBatch(slots, clock)
    batch.cells = {j.id: j.cells for j in jobs}
    if budget is None:
        budget = 10 ** 9
    srv = JobServer(fac, batch, budget, slots, chunk_steps=chunk, clock=clock, sleep=clock.sleep)
    done = srv.run(jobs)
    return srv, fac, batch, done


def test_all_jobs_complete_with_their_step_budget():
    jobs = _jobs(30, 1, rate=50.0)
    srv, fac, batch, done = _run(jobs)
    assert sorted(j.id for j in done) == list(range(30))
    for j in done:
        assert j.result == j.steps                 # exactly its budget
        assert j.arrival <= j.admitted <= j.finished
    assert not fac.live                            # every box released


def test_slots_and_memory_budget_are_respected():
    jobs = _jobs(40, 2, rate=None)                 # all arrive at once
    budget = 3 * 24 ** 3 * 10
    srv, fac, batch, done = _run(jobs, slots=5, budget=budget)
    assert len(done) == 40
    assert srv.peak_active <= 5
    assert srv.peak_bytes <= budget
    assert max(batch.sizes) <= 5


def test_admission_is_in_arrival_order():
    jobs = _jobs(25, 3, rate=20.0)
    srv, fac, batch, done = _run(jobs, slots=3)
    assert fac.created == sorted(fac.created, key=lambda i: (jobs[i].arrival, i))


def test_continuous_batching_admits_while_others_run():
    # job 1 arrives while job 0 is on the device and joins the running batch
    jobs = [Job(0, {}, 0.0, 1000, 1000), Job(1, {}, 0.05, 10, 1000)]
    srv, fac, batch, done = _run(jobs, slots=4, chunk=5)
    j0, j1 = sorted(done, key=lambda j: j.id)
    assert j1.admitted < j0.finished               # admitted before job 0 ended
    assert j1.finished < j0.finished               # and left before it
    assert max(batch.sizes) == 2                   # both were advanced together


def test_job_larger_than_budget_is_rejected():
    jobs = [Job(0, {}, 0.0, 10, 10 ** 6), Job(1, {}, 0.0, 5, 4)]
    srv, fac, batch, done = _run(jobs, budget=100)
    by = {j.id: j for j in done}
    assert by[0].status.startswith("rejected") and by[0].result is None
    assert by[1].status == "ok" and by[1].result == 5     # the other job ran
    s = summary(done, srv.elapsed)
    assert s["jobs"] == 1 and s["rejected"] == 1


class FailingFactory(FakeFactory):
    """Job ids in `bad_spec` have a description the factory cannot build;
    boxes of jobs in `blow_up` report a device failure when they finish (as
    a box whose LB steps met a non-finite density does)."""

    def __init__(self, bad_spec=(), blow_up=()):
        super().__init__()
        self.bad_spec, self.blow_up = set(bad_spec), set(blow_up)

    def create(self, job):
        if job.id in self.bad_spec:
            raise ValueError("invalid job description")
        return super().create(job)

    def status(self, box):
        return "non-finite density" if box["job"] in self.blow_up else 0


class RemovableBatch(FakeBatch):
    def remove(self, box):
        self.members = [m for m in self.members if m[0] is not box]


def test_failed_rejected_and_cancelled_jobs_leave_the_others_running():
    jobs = _jobs(12, 7, rate=None)
    clock = Clock()
    fac = FailingFactory(bad_spec={3}, blow_up={5})
    batch = RemovableBatch(4, clock)
    batch.cells = {j.id: j.cells for j in jobs}
    jobs[8].steps = 10 ** 6                     # long enough to be cancelled while running
    srv = JobServer(fac, batch, 10 ** 9, 4, chunk_steps=7, clock=clock, sleep=clock.sleep)
    srv.cancel(11)                              # cancelled while queued
    orig = batch.advance

    def advance(k):                             # cancel job 8 once it runs
        if any(m[0]["job"] == 8 for m in batch.members):
            srv.cancel(8)
        return orig(k)
    batch.advance = advance
    done = srv.run(jobs)
    by = {j.id: j for j in done}
    assert sorted(by) == list(range(12))
    assert by[3].status.startswith("rejected")
    assert by[5].status == "failed: non-finite density" and by[5].result is None
    assert by[8].status == "cancelled" and by[11].status == "cancelled"
    for i in set(range(12)) - {3, 5, 8, 11}:
        assert by[i].status == "ok" and by[i].result == jobs[i].steps
    assert not fac.live                         # every box released
    s = summary(done, srv.elapsed)
    assert (s["jobs"], s["failed"], s["rejected"], s["cancelled"]) == (8, 1, 1, 2)


def test_summary_statistics():
    jobs = _jobs(50, 4, rate=30.0)
    srv, fac, batch, done = _run(jobs)
    s = summary(done, srv.elapsed)
    lat = np.array([j.latency for j in done])
    assert s["jobs"] == 50
    assert s["p50_latency_s"] == pytest.approx(np.percentile(lat, 50))
    assert s["p99_latency_s"] == pytest.approx(np.percentile(lat, 99))
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0
    assert s["cell_updates"] == sum(j.cells * j.steps for j in jobs)


def test_box_factory_descriptors_follow_the_job_spec():
    """The library factory maps a job's coupling kind, stencil, collision,
    tau and storage into the box descriptors; its device-memory query is
    host-only."""
    from paper_1406_2211_gb300 import lbc
    from paper_1406_2211_gb300.serve import BoxFactory
    fac = BoxFactory(tau=0.9)
    pos = np.zeros((10, 3))
    plain = Job(0, dict(edge=16, storage="f32", pos=pos), 0.0, 5, 16 ** 3)
    lat, cpl, M = fac._descs(plain)
    assert (lat.collision, lat.tau, lat.storage) == (lbc.LBC_BGK, 0.9, lbc.LBC_F32)
    assert (cpl.kind, cpl.stencil, cpl.gamma, M) == (lbc.LBC_FC, lbc.LBC_TRILINEAR, 1.0, 10)
    ibm = Job(1, dict(edge=24, storage="bf16dev", pos=pos, kind="ibm", stencil="peskin4",
                      collision="mrt", tau=1.1), 0.0, 5, 24 ** 3)
    lat, cpl, M = fac._descs(ibm)
    assert (lat.collision, lat.tau, lat.storage) == (lbc.LBC_MRT, 1.1, lbc.LBC_BF16_DEV)
    assert (cpl.kind, cpl.stencil) == (lbc.LBC_IBM, lbc.LBC_PESKIN4)
    assert fac.bytes(ibm) > fac.bytes(plain) > 16 ** 3 * 2 * 19 * 4
