"""Serving loop for ensembles of independent suspension boxes.

Jobs (box edge, particle set, coupling parameters, storage, step count,
arrival time) are admitted in arrival order while a batch slot and enough
device memory are free; admitted boxes stay resident and advance together in
one lbc_batch (continuous batching: jobs that arrive while others are on
the GPU join the running batch, and a job leaves it as soon as its step
budget is spent).  Per job the loop records admission and completion times;
`summary` gives p50 / p99 latency (completion - arrival), jobs/s and the
aggregate lattice-update rate.

Failures are per job: a job whose box cannot be built or admitted is
"rejected", a job whose box fails while stepping (the library latches a
non-finite density met by an LB step, and the batch retires that member
without stopping the others) is "failed", and `cancel` removes a job
("cancelled"); the other jobs run on.  `summary` counts only completed jobs
in the rates and latencies and reports the others by kind.

The loop only schedules: every step runs in the library's kernels through
the `Batch` / `Box` bindings.  `JobServer` takes a factory (create / bytes /
result / release) and a batch object, so the host logic can be exercised
with stand-ins.
"""
import collections
import time

import numpy as np


class Job:
    """One request.  `spec` is the caller's description (edge, steps, ...);
    `arrival` is in seconds from the start of the run."""

    def __init__(self, jid, spec, arrival, steps, cells):
        self.id = jid
        self.spec = spec
        self.arrival = float(arrival)
        self.steps = int(steps)
        self.cells = int(cells)
        self.admitted = None
        self.finished = None
        self.result = None
        self.status = None          # "ok", "failed: ...", "rejected: ...", "cancelled"

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


class JobServer:
    """Admission by memory and slots, batched stepping, completion tracking.

    factory.bytes(job) -> device bytes the job's box needs
    factory.create(job) -> box (resident, initialised)
    factory.result(box) -> whatever the caller wants kept (read after the
                           batch has finished the box)
    factory.status(box) -> (optional) 0 if the box's run succeeded, else an
                           error description
    factory.release(box) -> frees the box's device memory
    batch.remove(box) -> takes a member out (for cancellation)
    batch.add(box, steps) -> bool (False: no free slot)
    batch.advance(max_steps) -> (steps done, finished boxes)
    sync() -> waits for the enqueued work
    """

    def __init__(self, factory, batch, memory_budget, max_active, chunk_steps=100,
                 sync=None, clock=time.perf_counter, sleep=time.sleep):
        self.factory = factory
        self.batch = batch
        self.memory_budget = int(memory_budget)
        self.max_active = int(max_active)
        self.chunk_steps = int(chunk_steps)
        self.sync = sync if sync is not None else (lambda: None)
        self.clock = clock
        self.sleep = sleep
        self.peak_active = 0
        self.peak_bytes = 0
        self._cancel = set()

    def cancel(self, jid):
        """Cancel job `jid`: it leaves the queue, or the batch at the next
        chunk boundary, with status "cancelled"."""
        self._cancel.add(jid)

    def run(self, jobs):
        pending = collections.deque(sorted(jobs, key=lambda j: (j.arrival, j.id)))
        queue = collections.deque()
        active = {}                # id(box) -> (job, box, bytes)
        used = 0
        done = []
        t0 = self.clock()
        def close(job, status):
            job.finished = self.clock() - t0
            job.status = status
            done.append(job)

        while pending or queue or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            # cancellations: queued jobs leave at once, running ones here
            if self._cancel:
                for job in [j for j in queue if j.id in self._cancel]:
                    queue.remove(job)
                    close(job, "cancelled")
                for key, (job, box, need) in list(active.items()):
                    if job.id in self._cancel:
                        self.batch.remove(box)
                        self.factory.release(box)
                        del active[key]
                        used -= need
                        close(job, "cancelled")
            # admit in arrival order while a slot and the memory are free
            while queue and len(active) < self.max_active:
                job = queue[0]
                try:
                    need = self.factory.bytes(job)
                except Exception as e:              # an invalid job description
                    queue.popleft()
                    close(job, "rejected: %s" % e)
                    continue
                if need > self.memory_budget:
                    queue.popleft()
                    close(job, "rejected: needs %d bytes, more than the budget" % need)
                    continue
                if used + need > self.memory_budget:
                    break
                queue.popleft()
                try:
                    box = self.factory.create(job)
                except Exception as e:
                    close(job, "rejected: %s" % e)
                    continue
                try:
                    admitted = self.batch.add(box, job.steps)
                except Exception as e:              # the batch refuses this box
                    self.factory.release(box)
                    close(job, "rejected: %s" % e)
                    continue
                if not admitted:
                    self.factory.release(box)
                    queue.appendleft(job)
                    break
                job.admitted = self.clock() - t0
                active[id(box)] = (job, box, need)
                used += need
            self.peak_active = max(self.peak_active, len(active))
            self.peak_bytes = max(self.peak_bytes, used)
            if not active:
                if pending:
                    self.sleep(max(0.0, min(pending[0].arrival - now, 0.01)))
                continue
            _, finished = self.batch.advance(self.chunk_steps)
            self.sync()
            now = self.clock() - t0
            status_of = getattr(self.factory, "status", None)
            for box in finished:
                job, b, need = active.pop(id(box))
                job.finished = now
                err = status_of(b) if status_of else 0
                if err:
                    job.status = "failed: %s" % err
                else:
                    job.status = "ok"
                    job.result = self.factory.result(b)
                self.factory.release(b)
                used -= need
                done.append(job)
        self.elapsed = self.clock() - t0
        return done


def summary(jobs, elapsed):
    """p50 / p99 latency, throughput and aggregate MLUPS of completed jobs
    (status "ok", or no status: jobs of a run without failures), and the
    number of failed, rejected and cancelled ones."""
    kinds = collections.Counter((j.status or "ok").split(":")[0] for j in jobs)
    jobs = [j for j in jobs if j.status in (None, "ok")]
    lat = np.array([j.latency for j in jobs], dtype=np.float64)
    updates = float(sum(j.cells * j.steps for j in jobs))
    return {"jobs": len(jobs), "elapsed_s": elapsed,
            "failed": kinds.get("failed", 0), "rejected": kinds.get("rejected", 0),
            "cancelled": kinds.get("cancelled", 0),
            "jobs_per_s": len(jobs) / elapsed if elapsed > 0 else None,
            "mlups": updates / elapsed / 1e6 if elapsed > 0 else None,
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "cell_updates": updates}


class BoxFactory:
    """Builds library boxes for ensemble jobs: cubic periodic box of edge
    spec["edge"] and storage spec["storage"], with particles at spec["pos"].
    Optional keys (defaults in brackets): "collision" ["bgk"], "tau" [the
    factory's], "kind" ["fc"; "ebf", "mebf", "ibm"], "stencil"
    ["trilinear"; "peskin4", "peskin3"], "gamma" [1.0], "mass" [1.0],
    "vel" [zero]; markers of an "ibm" job carry neither mass nor velocity."""

    def __init__(self, tau=0.8, rho0=1.0, stream=None):
        from . import lbc
        self.lbc = lbc
        self.tau = tau
        self.rho0 = rho0
        self.stream = stream

    def _descs(self, job):
        s = job.spec
        L = int(s["edge"])
        lat = self.lbc.lattice_desc(L, L, L, collision=s.get("collision", "bgk"),
                                    tau=float(s.get("tau", self.tau)), rho0=self.rho0,
                                    storage=s["storage"])
        cpl = self.lbc.coupling_desc(s.get("kind", "fc"), 2, s.get("stencil", "trilinear"),
                                     gamma=float(s.get("gamma", 1.0)))
        return lat, cpl, len(s["pos"])

    def bytes(self, job):
        import ctypes as C
        lat, cpl, M = self._descs(job)
        n = C.c_size_t()
        self.lbc.check(self.lbc.library().lbc_box_bytes_required(C.byref(lat), C.byref(cpl), M, 0,
                                                                C.byref(n)),
                       "lbc_box_bytes_required")
        return int(n.value)

    def create(self, job):
        lat, cpl, M = self._descs(job)
        box = self.lbc.Box(lat, cpl, max_particles=M, stream=self.stream)
        box.init_equilibrium(self.rho0, (0.0, 0.0, 0.0))
        s = job.spec
        if s.get("kind", "fc") == "ibm":
            box.set_particles(s["pos"])
        else:
            box.set_particles(s["pos"], vel=s.get("vel"), mass=float(s.get("mass", 1.0)))
        return box

    def status(self, box):
        """0 if the box ran without a device-detected failure, else the
        library's description of it (lbc_box_check)."""
        st = box.check()
        return 0 if st == 0 else self.lbc.library().lbc_status_string(st).decode()

    def result(self, box):
        pos, vel, fh = box.get_particles()
        return {"pos": pos, "vel": vel, "force_h": fh}

    def release(self, box):
        box.close()
        box.arena = None
