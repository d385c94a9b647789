"""Benchmark of the coupled D3Q19 step on the 256^3 bead-chain workload.

Workload (the single-box configuration the throughput metric is quoted on):
256^3 periodic box, MRT collision (shear rate 1/tau, tau = 1), FP32
populations stored as deviations from w_i rho0, 2000 bead chains of 50 beads
(100 000 particles, harmonic bonds k = 10, r0 = 1), viscous force coupling
gamma = 5, m = 1, trilinear interpolation and spreading, body force 1e-6
along x, the multiple-time-step split of Sec. 6 (Eq. [multistep]) with four
coupled particle sub-steps per half step.  Inputs are synthetic and seeded
(synth/).

One "step" is one full coupled time step (drift/forces, marker binning,
interpolation + coupling, spreading, fused LB step).  value = million lattice
updates per second (MLUPS) of the whole job over all ranks; the population
arrays (1.27 GB each) are larger than L2, so no flush is needed.

Printed as one JSON line (rank 0).  --impl reference times the FP64 oracle
on the host cores instead (a bounded sample of the same workload).
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled D3Q19 MLUPS & % of HBM peak; ensemble jobs/s with p50/p99 latency"
WORKLOAD = "mrt_bead_chains_256"
LB_KERNEL_SOURCES = ["paper_1406_2211_gb300/csrc/lb_kernels.cu",
                     "paper_1406_2211_gb300/csrc/lb_cell.cuh",
                     "paper_1406_2211_gb300/csrc/lb_device.cuh",
                     "paper_1406_2211_gb300/csrc/lbc_common.cuh"]
PROFILE = os.path.join(ROOT, "profiles", "lb_step_mrt_f32_256.md")


def lb_source_hash():
    h = hashlib.sha256()
    for f in LB_KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per LB launch from the committed ncu summary, if it was
    taken on the current LB kernel source."""
    if not os.path.exists(PROFILE):
        return None
    text = open(PROFILE).read()
    m_hash = re.search(r"lb_source_hash:\s*([0-9a-f]+)", text)
    m_traf = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_traf or m_hash.group(1) != lb_source_hash():
        return None
    return float(m_traf.group(1))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ workload
def workload(scale=1):
    import synth
    c = synth.config(WORKLOAD, scale=scale)
    pos, bonds = synth.bead_chains(c["nchains"], c["beads"], c["box"], c["bond_r0"],
                                   seed=c["seed"])
    return c, pos, bonds


def make_box(c, npart, nbonds, storage=None):
    from paper_1406_2211_gb300 import lbc
    nx, ny, nz = c["box"]
    lat = lbc.lattice_desc(nx, ny, nz, collision=c["collision"], tau=c["tau"],
                           rho0=c["rho0"], body_force=c["body_force"],
                           storage=storage or c["storage"])
    cpl = lbc.coupling_desc(c["kind"], 2, c["stencil"], gamma=c["gamma"], split=c["mode"],
                            substeps=c["substeps"])
    return lbc.Box(lat, cpl, max_particles=npart, max_bonds=nbonds)


# algorithmic bytes per cell update of the fused LB step: 19 reads + 19 writes
BYTES_PER_CELL = {"f32": 2 * 19 * 4, "f16dev": 2 * 19 * 2, "bf16dev": 2 * 19 * 2, "f64": 2 * 19 * 8}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "lbc_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(r["sm"] for r in rows)
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------ GPU arm
def max_over_ranks(ms, world, device):
    """The job's time: the slowest rank's, the same on every rank (replicas
    share no data; this is the only collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells, steps, world, ms):
    """Lattice updates of all ranks' replicas over the job's time."""
    return world * cells * steps / (ms * 1e-3) / 1e6


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    c, pos, bonds = workload(scale=args.scale)
    nx, ny, nz = c["box"]
    cells = nx * ny * nz
    M, B = len(pos), len(bonds)
    stream = torch.cuda.current_stream()

    def timed(storage, steps, sample_clocks, tau=None, prep=None):
        """Warm up, then time `steps` coupled steps of a fresh box (CUDA
        events on the launching stream, barrier + synchronize on both sides);
        LB kernel launches are timed by event nodes inside the graphs."""
        from paper_1406_2211_gb300 import lbc
        box = make_box(c if tau is None else dict(c, tau=tau), M, B, storage)
        box.init_equilibrium(c["rho0"], (0.0, 0.0, 0.0))
        box.set_particles(pos, vel=np.zeros_like(pos), mass=c["mass"], bonds=bonds,
                          bond_k=c["bond_k"], bond_r0=c["bond_r0"])
        shape = box.autotune()           # LB launch shape, before any timing
        keep = prep(box) if prep else None   # a variant's set-up (kept alive)
        box.step(args.warmup)
        box.set_option(lbc.LBC_OPT_TIMING, steps + 4)
        # the graphs are recaptured with timing nodes: one eager step + one
        # replay before the timed region keeps capture out of it
        box.step(3)
        box.lb_timing(reset=True)
        r = {"launches_per_step": box.launches_per_step(),
             "pop_bytes": box.population_bytes(), "lb_block": list(shape)}
        clocks = ClockSampler(local_rank) if sample_clocks else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        box.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        r["ms"] = e0.elapsed_time(e1)
        r["clocks"] = clocks.stop() if clocks else None
        r["lb_ms"], r["lb_n"] = box.lb_timing(reset=True)
        del keep
        _, _, st = box.invariants()
        if st != 0:
            raise RuntimeError("non-finite state after the timed steps (%s)" % storage)
        if r["lb_n"] == 0 or r["lb_ms"] <= 0:
            raise RuntimeError("no LB kernel launches were timed")
        box.close()
        del box
        torch.cuda.empty_cache()
        r["ms_max"] = max_over_ranks(r["ms"], world, "cuda")
        r["value"] = whole_job_mlups(cells, steps, world, r["ms_max"])
        r["lb_avg_ms"] = r["lb_ms"] / r["lb_n"]
        r["achieved"] = BYTES_PER_CELL[storage] * cells / (r["lb_avg_ms"] * 1e-3) / 1e9
        # the whole coupled step against the same roofline: algorithmic
        # population bytes per step over the step's time
        r["step_gbs"] = BYTES_PER_CELL[storage] * cells / (r["ms_max"] / steps * 1e-3) / 1e9
        return r

    main = timed(c["storage"], args.steps, True)
    ms, ms_max, value = main["ms"], main["ms_max"], main["value"]
    lb_ms, lb_n, lb_avg_ms = main["lb_ms"], main["lb_n"], main["lb_avg_ms"]
    launches_per_step, pop_bytes, clk = main["launches_per_step"], main["pop_bytes"], main["clocks"]

    # roofline of the dominant kernel (fused LB step): algorithmic bytes =
    # 2 x 19 populations x 4 bytes per cell
    alg_bytes = BYTES_PER_CELL[c["storage"]] * cells
    achieved = main["achieved"]
    peak, peak_kind = measured_peaks()
    traffic = profiled_traffic()

    # the same coupled step with 16-bit population storage (deviations from
    # w_i rho0, stochastic rounding, FP32 arithmetic)
    # and FP32 at tau = 0.8, where the MRT stress relaxes (at the workload's
    # tau = 1 every non-conserved eigenvalue is 0): the kernel time does not
    # depend on it
    forms = None
    if not args.no_forms:
        forms = {}
        nform = min(args.steps, 100)
        # thermal fluctuations (Eq. [mrt-fluct] kicks inside the fused LB
        # kernel, random force zeta on the beads) at k_B T = 1e-7, and the
        # FP32 step with the stress epilogue (Eq. [viscstress]: 6 FP32
        # values more per cell, 176 B per cell update)
        thermal = lambda box: box.set_thermal(1e-7, 2014)
        stress = lambda box: box.stress_output()
        for name, st16, tau, prep, extra in (
                ("f16dev", "f16dev", None, None, 0), ("bf16dev", "bf16dev", None, None, 0),
                ("f32_tau0.8", "f32", 0.8, None, 0), ("f32_thermal", "f32", None, thermal, 0),
                ("bf16dev_thermal", "bf16dev", None, thermal, 0),
                ("f32_stress", "f32", None, stress, 24)):
            r = timed(st16, nform, False, tau=tau, prep=prep)
            alg = BYTES_PER_CELL[st16] + extra
            lb_gbs = alg * cells / (r["lb_avg_ms"] * 1e-3) / 1e9
            forms[name] = {"value": r["value"], "unit": "MLUPS", "steps": nform,
                           "ms_per_step": r["ms_max"] / nform, "tau": tau or c["tau"],
                           "lb_avg_ms": r["lb_avg_ms"], "lb_achieved_gbs": lb_gbs,
                           "lb_frac_of_peak": lb_gbs / peak,
                           "step_frac": r["step_gbs"] / peak,
                           "alg_bytes_per_cell": alg, "lb_block": r["lb_block"]}

    # end to end through the C ABI with host buffers: upload particles,
    # step, read particles and invariants back (copies inside the timing)
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hpos, hvel = pin(pos), pin(np.zeros_like(pos))
        box2 = make_box(c, M, B)
        box2.init_equilibrium(c["rho0"], (0.0, 0.0, 0.0))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        box2.set_particles(hpos, vel=hvel, mass=c["mass"], bonds=bonds,
                           bond_k=c["bond_k"], bond_r0=c["bond_r0"])
        box2.step(args.steps)
        rpos, rvel, _ = box2.get_particles()
        _, _, st2 = box2.invariants()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        t_e2e = max_over_ranks(t_e2e, world, "cuda")
        h2d = hpos.nbytes + hvel.nbytes + M * 8 + bonds.nbytes + 2 * B * 8
        # F^h comes back in the compute type (FP32 unless the storage is FP64)
        d2h = rpos.nbytes + rvel.nbytes + M * (24 if c["storage"] == "f64" else 12) + 4 * 8
        e2e = {"value": whole_job_mlups(cells, args.steps, world, t_e2e * 1e3), "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "scope": "lbc_box_set_particles (host arrays) + lbc_box_step + "
                        "lbc_box_get_particles + lbc_box_invariants"}
        box2.close()

    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded bead chains, fluid at rest)",
        "config": {"workload": WORKLOAD if args.scale == 1 else "%s/%d" % (WORKLOAD, args.scale),
                   "box": [nx, ny, nz], "collision": "mrt",
                   "tau": c["tau"], "storage": "f32 deviations", "particles": M,
                   "bonds": B, "coupling": "force coupling, gamma=5, m=1",
                   "stencil": "trilinear", "split": "Eq. multistep, n=4 coupled sub-steps per half",
                   "body_force": list(c["body_force"]),
                   "l2": "inputs larger than L2 (2 x %.2f GB population arrays)" % (pop_bytes / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "lb_block": main["lb_block"]},
        "roofline": {"bound": "hbm", "kernel": "lb_step_kernel (fused LB step)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_kind,
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": lb_avg_ms,
                     "launches_timed": lb_n,
                     "lb_share_of_step": lb_ms / ms if ms > 0 else None,
                     # the whole coupled step: 152 B x cells / ms_per_step / peak
                     "step_achieved": main["step_gbs"], "step_frac": main["step_gbs"] / peak},
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clk,
        "e2e": e2e,
        "storage_forms": forms,
    }
    return line


# ------------------------------------------------------------------ other workloads
def other_workload_boxes(name, storage, stencil=None, kind=None, mass_scale=1.0):
    """Full-size box of the shell (IBM) or rigid-sphere (modified EBF)
    workload with its particles set.  For the spheres: another stencil, the
    IBM kind, or the markers' mass scaled (the immersion limit m -> 0)."""
    import numpy as np
    import synth
    from paper_1406_2211_gb300 import lbc
    c = synth.config(name)
    nx, ny, nz = c["box"]
    if name.startswith("ibm_shells"):
        pos, edges, r0 = synth.shells(c["nshells"], c["radius"], c["box"], c["seed"],
                                      c["subdivisions"])
        lat = lbc.lattice_desc(nx, ny, nz, collision=c["collision"], tau=c["tau"],
                               walls=True, wall_velocity=c["wall_velocity"], storage=storage)
        cpl = lbc.coupling_desc("ibm", 2, c["stencil"])
        box = lbc.Box(lat, cpl, max_particles=len(pos), max_bonds=len(edges))
        box.init_equilibrium(c["rho0"], (0.0, 0.0, 0.0))
        box.set_particles(pos, bonds=edges, bond_k=c["spring_k"], bond_r0=r0)
        desc = "%d shells x 642 IBM markers, springs k = %g, walls -/+%g, Peskin-4" % (
            c["nshells"], c["spring_k"], c["wall_velocity"][1][0])
    else:
        pos, first, count = synth.rigid_spheres(c["nspheres"], c["radius"], c["markers"],
                                                c["box"], seed=c["seed"])
        mass = mass_scale * c["rho0"] * 4.0 / 3.0 * np.pi * c["radius"] ** 3 / c["markers"]
        lat = lbc.lattice_desc(nx, ny, nz, collision=c["collision"], tau=c["tau"], storage=storage)
        st = stencil or c["stencil"]
        kd = kind or "mebf"
        cpl = lbc.coupling_desc(kd, 2, st)
        box = lbc.Box(lat, cpl, max_particles=len(pos))
        box.init_equilibrium(c["rho0"], (0.0, 0.0, 0.0))
        rng = np.random.default_rng(c["seed"])
        rigid = dict(first=first, count=count, radius=c["radius"], k=c["rigid_k"],
                     repulsion_k=c["repulsion_k"])
        if kd == "ibm":
            box.set_particles(pos, rigid=rigid)
        else:
            box.set_particles(pos, vel=0.002 * rng.standard_normal(pos.shape), mass=mass,
                              rigid=rigid)
        desc = "%d rigid spheres x %d markers (tethers k = %g), %s, %s, tau = %g" % (
            c["nspheres"], c["markers"], c["rigid_k"],
            "IBM" if kd == "ibm" else "modified EBF" + (" (m x %g)" % mass_scale if mass_scale != 1.0 else ""),
            {"peskin4": "Peskin-4", "trilinear": "trilinear", "peskin3": "3-point"}[st], c["tau"])
    return box, nx * ny * nz, desc


OTHER_WORKLOADS = (("ibm_shells_192", ("f32", "f16dev", "bf16dev")),
                   ("mebf_rigid_spheres_128", ("f32", "f32_trilinear")))


def run_other_workloads(args, peak, only=None):
    """The shell and rigid-sphere workloads at full size (or only the one
    named): coupled MLUPS over `steps` steps (CUDA events, at most 60) and the
    LB kernel's fraction of the peak."""
    import torch
    from paper_1406_2211_gb300 import lbc
    out = {}
    steps = min(args.steps, 60)
    for name, storages in OTHER_WORKLOADS:
        if only is not None and name != only:
            continue
        out[name] = {}
        for st in storages:
            box, cells, desc = other_workload_boxes(
                name, st.split("_")[0], stencil="trilinear" if st.endswith("_trilinear") else None)
            shape = box.autotune()
            box.step(args.warmup)
            box.set_option(lbc.LBC_OPT_TIMING, steps + 4)
            box.step(3)
            box.lb_timing(reset=True)
            stream = torch.cuda.current_stream()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            box.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            lb_ms, lb_n = box.lb_timing(reset=True)
            _, _, status = box.invariants()
            box.close()
            del box
            torch.cuda.empty_cache()
            if status != 0:
                raise RuntimeError("non-finite state in %s (%s)" % (name, st))
            lb_avg = lb_ms / lb_n
            out[name][st] = {"value": cells * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                             "steps": steps, "ms_per_step": ms / steps, "lb_avg_ms": lb_avg,
                             "lb_frac_of_peak": BYTES_PER_CELL[st.split("_")[0]] * cells / (lb_avg * 1e-3) / 1e9 / peak,
                             "step_frac": BYTES_PER_CELL[st.split("_")[0]] * cells / (ms / steps * 1e-3) / 1e9 / peak,
                             "lb_block": list(shape), "model": desc}
        if name.startswith("mebf_rigid"):
            out[name]["immersion_limit"] = immersion_limit_on_gpu(args)
    return out


def immersion_limit_on_gpu(args, steps=20, mass_scale=1e-6):
    """Sec. 5.3, Eq. [immersion]: the modified EBF with the markers' mass
    m -> 0 (immersion number r -> 1) becomes the immersed boundary method.
    The full 128^3 rigid-sphere workload run both ways from the same state
    for `steps` steps on the GPU: the largest difference of the sphere
    centroids (expected O(m)), and each form's time per step."""
    import numpy as np
    import torch
    import synth
    c = synth.config("mebf_rigid_spheres_128")
    L = np.array(c["box"], dtype=float)
    res = {}
    cents = {}
    for label, kind, ms in (("mebf_m0", "mebf", mass_scale), ("ibm", "ibm", 1.0)):
        box, cells, desc = other_workload_boxes("mebf_rigid_spheres_128", "f32", kind=kind,
                                                mass_scale=ms)
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        box.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        pos, _, _ = box.get_particles()
        _, _, st = box.invariants()
        box.close()
        torch.cuda.empty_cache()
        if st != 0:
            raise RuntimeError("non-finite state in the immersion-limit run (%s)" % label)
        m = c["markers"]
        P = pos.reshape(-1, m, 3)
        ref = P[:, :1, :]
        d = P - ref
        d -= L * np.round(d / L)                  # unwrapped around the first marker
        cents[label] = ref[:, 0, :] + d.mean(axis=1)
        res[label + "_ms_per_step"] = e0.elapsed_time(e1) / steps
        res[label + "_model"] = desc
    dc = cents["mebf_m0"] - cents["ibm"]
    dc -= L * np.round(dc / L)
    res.update({"steps": steps, "mass_scale": mass_scale,
                "max_centroid_difference": float(np.abs(dc).max())})
    return res


# ------------------------------------------------------------------ serving
def serving_jobs(njobs, seed, step_scale, rate=None):
    """A bounded sample of the serving ensemble: cubic periodic boxes of edge
    log-uniform in [32, 128], 1-5000 force-coupled particles (gamma uniform in
    [0.5, 10]), FP32 or FP16-deviation storage (50/50), steps uniform in
    [1000, 20000] divided by step_scale, Poisson arrivals at `rate` jobs/s
    (all at t = 0 if None)."""
    import numpy as np
    import synth
    from paper_1406_2211_gb300.serve import Job
    lo, hi = 1000 // step_scale, 20000 // step_scale
    specs = synth.ensemble_jobs(njobs, seed=seed, steps_range=(lo, hi), rate=rate)
    jobs = []
    for i, sp in enumerate(specs):
        rng = np.random.default_rng(sp["seed"])
        L, M = sp["edge"], sp["nparticles"]
        spec = dict(edge=L, gamma=sp["gamma"], storage=sp["storage"],
                    pos=rng.uniform(0.0, L, (M, 3)), vel=np.zeros((M, 3)))
        jobs.append(Job(i, spec, sp["arrival"], sp["steps"], L ** 3))
    return jobs


def run_serving(args):
    """Continuous batching of the ensemble sample: first with every job
    queued at t = 0 (capacity), then with Poisson arrivals at 0.8 x that
    capacity (latency).  Returns the serving summary."""
    import torch
    from paper_1406_2211_gb300 import lbc
    from paper_1406_2211_gb300.serve import BoxFactory, JobServer, summary
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.5 * free)
    slots = 32

    def serve(jobs):
        batch = lbc.Batch(slots)
        srv = JobServer(BoxFactory(), batch, budget, slots, chunk_steps=50,
                        sync=torch.cuda.synchronize)
        done = srv.run(jobs)
        out = summary(done, srv.elapsed)
        out["peak_active"] = srv.peak_active
        out["peak_bytes"] = srv.peak_bytes
        batch.close()
        torch.cuda.empty_cache()
        return out

    n = args.serve_jobs
    if args.serve_full:
        # the ensemble's own job sizes (steps uniform in [1000, 20000]):
        # capacity with every job queued at t = 0, then Poisson arrivals at
        # 0.5, 0.8 and 1.2 of that capacity
        n = args.serve_full
        sat = serve(serving_jobs(n, 12345, 1))
        sweep = {}
        for load in (0.5, 0.8, 1.2):
            r = serve(serving_jobs(n, 12345, 1, rate=load * sat["jobs_per_s"]))
            sweep["%.1f" % load] = {k: r[k] for k in ("jobs_per_s", "mlups", "p50_latency_s",
                                                     "p99_latency_s", "elapsed_s", "peak_active",
                                                     "failed", "rejected")}
        return {"jobs": n, "unit": "jobs/s", "capacity_jobs_per_s": sat["jobs_per_s"],
                "capacity_mlups": sat["mlups"], "capacity_elapsed_s": sat["elapsed_s"],
                "loads": sweep, "slots": slots, "memory_budget_bytes": budget,
                "sample": "%d jobs of the 2000-job ensemble (same distributions, full step "
                          "counts 1000-20000), seed 12345; capacity with all jobs queued at "
                          "t = 0, then Poisson arrivals at 0.5 / 0.8 / 1.2 x capacity" % n}
    sat = serve(serving_jobs(n, 12345, 20))
    rate = 0.8 * sat["jobs_per_s"]
    lat = serve(serving_jobs(n, 12345, 20, rate=rate))
    return {"jobs": n, "unit": "jobs/s", "value": lat["jobs_per_s"], "mlups": lat["mlups"],
            "p50_latency_s": lat["p50_latency_s"], "p99_latency_s": lat["p99_latency_s"],
            "offered_rate_jobs_per_s": rate, "offered_load": 0.8,
            "capacity_jobs_per_s": sat["jobs_per_s"], "capacity_mlups": sat["mlups"],
            "peak_active": lat["peak_active"], "slots": slots, "memory_budget_bytes": budget,
            "sample": "%d jobs of the 2000-job ensemble (same distributions), steps / 20 "
                      "(50-1000), seed 12345; arrivals Poisson at 0.8 x the capacity "
                      "measured with all jobs queued at t = 0" % n}


# ------------------------------------------------------------------ CPU arm
def oracle_sample(max_seconds, min_steps=2, max_steps=None):
    """The FP64 oracle on a bounded sample of the workload: the 256^3 box cut
    to 64^3 with 1/64 of the chains (same density), MRT, same coupling.
    Runs in this process with one BLAS thread.  Returns (MLUPS, steps, s)."""
    import numpy as np
    from oracle import coupling as OC
    from oracle import lattice as OLat
    from oracle import lb as OL
    from oracle import sim as OS
    c, pos, bonds = workload(scale=4)
    nx, ny, nz = c["box"]
    shape = (nz, ny, nx)
    p = OL.LBParams(collision=c["collision"], tau=c["tau"], rho0=c["rho0"],
                    body_force=c["body_force"])
    parts = OC.Particles(pos, vel=np.zeros_like(pos), mass=np.full(len(pos), c["mass"]),
                         bonds=bonds, bond_k=c["bond_k"], bond_r0=c["bond_r0"])
    sm = OS.Sim(shape, p, OS.CouplingParams("fc", 2, c["stencil"], gamma=c["gamma"],
                                            substeps=c["substeps"], mode=c["mode"]),
                parts, fbar=OLat.equilibrium(np.full(shape, c["rho0"]),
                                             np.zeros((3,) + shape)))
    t0 = time.perf_counter()
    n = 0
    while True:
        sm.step()
        n += 1
        el = time.perf_counter() - t0
        if max_steps is not None and n >= max_steps:
            break
        if n >= min_steps and el >= max_seconds:
            break
    cells = nx * ny * nz
    return cells * n / el / 1e6, n, el, "%dx%dx%d box, %d particles, %d steps" % (
        nx, ny, nz, len(pos), n)


def cpu_model():
    """CPU model name of the host (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline_subprocess(max_seconds):
    """The oracle on one host core, then on every core at once (one
    single-threaded oracle process per core, each on its own copy of the
    sample: the oracle has no shared-memory parallel form, so all cores are
    used as independent replicas and the rates add up).  Both are started
    before any CUDA work."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(%f)))" % (ROOT, max_seconds))

    def run(nproc):
        procs = [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                  stderr=subprocess.DEVNULL, text=True) for _ in range(nproc)]
        res = []
        for p in procs:
            out, _ = p.communicate(timeout=900)
            if p.returncode != 0:
                return None
            res.append(json.loads(out.strip().splitlines()[-1]))
        return res

    one = run(1)
    if not one:
        return None
    v1, n1, el1, sample = one[0]
    cores = os.cpu_count() or 1
    allc = run(cores) if cores > 1 else one
    out = {"value": v1, "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "cpu_model": cpu_model(),
           "sample": "FP64 NumPy oracle, " + sample + " (%.1f s)" % el1,
           "one_core": {"value": v1, "cores": 1}}
    if allc:
        vall = sum(r[0] for r in allc)
        out.update({"value": vall, "cores": cores,
                    "sample": "FP64 NumPy oracle, %d concurrent single-threaded copies of: %s "
                              "(about %.0f s each)" % (cores, sample, max_seconds),
                    "all_cores": {"value": vall, "cores": cores}})
    return out


def run_reference(args):
    """--impl reference: the oracle, timed on the host cores, K steps of a
    bounded sample of the workload (rank 0 only)."""
    env_threads = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1"}
    for k, v in env_threads.items():
        os.environ.setdefault(k, v)
    # warm-up and timed steps on the 64^3 sample; each step ~0.3 s
    oracle_sample(0.0, min_steps=args.warmup, max_steps=args.warmup)
    steps = min(args.steps, 60)
    v, n, el, sample = oracle_sample(0.0, min_steps=steps, max_steps=steps)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS",
            "n_gpus": 0, "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * el / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded bead chains, fluid at rest)",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": "FP64 NumPy oracle, " + sample +
                                       " (steps capped at 60 of the requested %d)" % args.steps},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the ensemble serving measurement")
    ap.add_argument("--serve-jobs", type=int, default=32)
    # the serving measurement at the ensemble's full job sizes (N jobs, a
    # load sweep; minutes of device time), printed as its own JSON line
    ap.add_argument("--serve-full", type=int, default=0)
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the 16-bit storage forms of the same step")
    # box edge / SCALE and particle count / SCALE^3 at the same densities: the
    # small case for multi-pass profiler captures (default: the full workload)
    ap.add_argument("--scale", type=int, default=1)
    # only the full-size shell or rigid-sphere workload (its own JSON line;
    # for launch lists of that workload)
    ap.add_argument("--workload", default=None, choices=[n for n, _ in OTHER_WORKLOADS])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return 0
    if args.serve_full:
        if rank == 0:
            print(json.dumps({"serving_full": run_serving(args)}))
        return 0
    if args.workload is not None:
        if rank == 0:
            res = run_other_workloads(args, measured_peaks()[0], only=args.workload)
            print(json.dumps({"workload": args.workload, "results": res[args.workload]}))
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the oracle process is started before any CUDA work
        cpu = cpu_baseline_subprocess(args.cpu_seconds)
    line = run_gpu(args, rank, world, local_rank)
    line["cpu_baseline"] = cpu
    if rank == 0 and world == 1 and not args.no_serving:
        line["serving"] = run_serving(args)
    if rank == 0 and world == 1 and not args.no_forms:
        line["other_workloads"] = run_other_workloads(args, line["roofline"]["peak"])
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
