"""Serving loop for ensembles of independent suspension boxes.

Jobs (box edge, particle set, coupling parameters, storage, step count,
arrival time) are admitted in arrival order while a batch slot and enough
device memory are free; admitted boxes stay resident and advance together in
one lbc_batch (continuous batching: jobs that arrive while others are on
the GPU join the running batch, and a job leaves it as soon as its step
budget is spent).  Per job the loop records admission and completion times;
`summary` gives p50 / p99 latency (completion - arrival), jobs/s and the
aggregate lattice-update rate.

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

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


class JobServer:
    """Admission by memory and slots, batched stepping, completion tracking.

    factory.bytes(job) -> device bytes the job's box needs
    factory.create(job) -> box (resident, initialised)
    factory.result(box) -> whatever the caller wants kept (read after the
                           batch has finished the box)
    factory.release(box) -> frees the box's device memory
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

    def run(self, jobs):
        pending = collections.deque(sorted(jobs, key=lambda j: (j.arrival, j.id)))
        queue = collections.deque()
        active = {}                # id(box) -> (job, box, bytes)
        used = 0
        done = []
        t0 = self.clock()
        while pending or queue or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            # admit in arrival order while a slot and the memory are free
            while queue and len(active) < self.max_active:
                job = queue[0]
                need = self.factory.bytes(job)
                if need > self.memory_budget:
                    raise ValueError("job %d needs %d bytes, more than the budget" % (job.id, need))
                if used + need > self.memory_budget:
                    break
                queue.popleft()
                box = self.factory.create(job)
                if not self.batch.add(box, job.steps):
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
            for box in finished:
                job, b, need = active.pop(id(box))
                job.finished = now
                job.result = self.factory.result(b)
                self.factory.release(b)
                used -= need
                done.append(job)
        self.elapsed = self.clock() - t0
        return done


def summary(jobs, elapsed):
    """p50 / p99 latency, throughput and aggregate MLUPS of completed jobs."""
    lat = np.array([j.latency for j in jobs], dtype=np.float64)
    updates = float(sum(j.cells * j.steps for j in jobs))
    return {"jobs": len(jobs), "elapsed_s": elapsed,
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

    def result(self, box):
        pos, vel, fh = box.get_particles()
        return {"pos": pos, "vel": vel, "force_h": fh}

    def release(self, box):
        box.close()
        box.arena = None
