"""ctypes binding of the C ABI in include/lbc.h (argument marshalling only).

Function names match the C entry points.  `Box` is a convenience wrapper that
allocates the caller-owned device arena as a torch tensor and passes torch's
current CUDA stream; every step of the computation runs in the library's
CUDA kernels.  There is no CPU fallback: importing works without a GPU, but
any call that needs the library raises if it is missing.
"""
import ctypes as C
import os

import numpy as np

from .builder import LIB

# ---- constants (mirrors include/lbc.h; checked by tests/test_abi.py) ----
LBC_OK = 0
LBC_ERR_ARG = -1
LBC_ERR_OOM = -2
LBC_ERR_CUDA = -3
LBC_ERR_NONFINITE = -4
LBC_ERR_TIMEOUT = -5
LBC_ERR_STATE = -6
LBC_ERR_UNSUPPORTED = -7
LBC_BGK, LBC_MRT = 0, 1
LBC_F64, LBC_F32, LBC_F16_DEV, LBC_BF16_DEV = 0, 1, 2, 3
LBC_NONE, LBC_IBM, LBC_FC, LBC_EBF, LBC_MEBF = 0, 1, 2, 3, 4
LBC_TRILINEAR, LBC_PESKIN4, LBC_PESKIN3 = 0, 1, 2
LBC_SPLIT_BASE, LBC_SPLIT_INSIDE, LBC_SPLIT_OUTSIDE = 0, 1, 2
LBC_OPT_GRAPHS = 1
LBC_BATCH_MAX_NX = 128
LBC_OPT_TIMING = 2
LBC_OPT_NODE_MOMENTS = 3
LBC_OPT_GATHER_LANES = 4
LBC_OPT_THERMAL_AMPLITUDE = 5
LBC_OPT_LB_PAIR = 6
LBC_BATCH_OPT_LAUNCH = 1
LBC_BATCH_LAUNCH_AUTO, LBC_BATCH_LAUNCH_STREAMS, LBC_BATCH_LAUNCH_BATCHED = 0, 1, 2
LBC_NOALLOC_MAX_PLANES = 4096

STORAGE = {"f64": LBC_F64, "f32": LBC_F32, "f16dev": LBC_F16_DEV,
           "bf16dev": LBC_BF16_DEV}
COLLISION = {"bgk": LBC_BGK, "mrt": LBC_MRT}
KIND = {"none": LBC_NONE, "ibm": LBC_IBM, "fc": LBC_FC, "ebf": LBC_EBF,
        "mebf": LBC_MEBF}
STENCIL = {"trilinear": LBC_TRILINEAR, "peskin4": LBC_PESKIN4,
           "peskin3": LBC_PESKIN3}
SPLIT = {"base": LBC_SPLIT_BASE, "inside": LBC_SPLIT_INSIDE,
         "outside": LBC_SPLIT_OUTSIDE}


class lbc_lattice_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("collision", C.c_int32), ("tau", C.c_double),
                ("mrt_lambda", C.c_double * 4), ("rho0", C.c_double),
                ("body_force", C.c_double * 3), ("z_walls", C.c_int32),
                ("wall_velocity", (C.c_double * 3) * 2), ("storage", C.c_int32),
                ("storage_scale", C.c_double)]


class lbc_coupling_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("order", C.c_int32), ("stencil", C.c_int32),
                ("gamma", C.c_double), ("split", C.c_int32), ("substeps", C.c_int32)]


class lbc_particles_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos", C.c_void_p), ("vel", C.c_void_p),
                ("mass", C.c_void_p), ("ext_force", C.c_void_p),
                ("nbonds", C.c_int64), ("bond_ij", C.c_void_p),
                ("bond_k", C.c_void_p), ("bond_r0", C.c_void_p),
                ("nrigid", C.c_int64), ("rigid_first", C.c_void_p),
                ("rigid_count", C.c_void_p), ("rigid_radius", C.c_void_p),
                ("rigid_ref", C.c_void_p), ("rigid_k", C.c_double),
                ("rigid_repulsion_k", C.c_double)]


_P = C.c_void_p
_S = C.c_int32
_PROTOS = {
    "lbc_abi_version": (C.c_int32, []),
    "lbc_desc_sizes": (None, [C.POINTER(C.c_size_t)]),
    "lbc_status_string": (C.c_char_p, [C.c_int32]),
    "lbc_box_bytes_required": (_S, [C.POINTER(lbc_lattice_desc), C.POINTER(lbc_coupling_desc),
                                    C.c_int64, C.c_int64, C.POINTER(C.c_size_t)]),
    "lbc_box_create": (_S, [C.POINTER(lbc_lattice_desc), C.POINTER(lbc_coupling_desc),
                            C.c_int64, C.c_int64, _P, C.c_size_t, _P, C.POINTER(_P)]),
    "lbc_box_destroy": (_S, [_P]),
    "lbc_box_init_equilibrium": (_S, [_P, C.c_double, C.POINTER(C.c_double), _P]),
    "lbc_box_set_fields": (_S, [_P, _P, _P, _P]),
    "lbc_box_set_populations": (_S, [_P, _P, _P]),
    "lbc_box_get_populations": (_S, [_P, _P, _P]),
    "lbc_box_set_pending_force": (_S, [_P, _P, _P]),
    "lbc_box_set_particles": (_S, [_P, C.POINTER(lbc_particles_desc), _P]),
    "lbc_box_step": (_S, [_P, C.c_int64, _P]),
    "lbc_box_get_fields": (_S, [_P, _P, _P, _P]),
    "lbc_box_get_particles": (_S, [_P, _P, _P, _P, _P]),
    "lbc_box_get_stress": (_S, [_P, _P, _P]),
    "lbc_box_autotune": (_S, [_P, _P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lbc_box_invariants": (_S, [_P, _P, _P, _P]),
    "lbc_box_status": (_S, [_P]),
    "lbc_box_check": (_S, [_P, _P]),
    "lbc_box_set_option": (_S, [_P, C.c_int32, C.c_int64]),
    "lbc_box_get_option": (_S, [_P, C.c_int32, C.POINTER(C.c_int64)]),
    "lbc_box_set_thermal": (_S, [_P, C.c_double, C.c_uint64]),
    "lbc_box_set_stress_output": (_S, [_P, _P, C.c_size_t]),
    "lbc_box_launches_per_step": (C.c_int64, [_P]),
    "lbc_box_population_bytes": (C.c_size_t, [_P]),
    "lbc_box_lb_timing": (_S, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]),
    "lbc_fbar_moments_noalloc": (_S, [_P, C.c_int32, C.c_int32, C.c_int32, _P, _P]),
    "lbc_batch_bytes_required": (C.c_size_t, [C.c_int32]),
    "lbc_batch_create": (_S, [C.c_int32, _P, C.c_size_t, C.POINTER(_P)]),
    "lbc_batch_add": (_S, [_P, _P, C.c_int64]),
    "lbc_batch_remove": (_S, [_P, _P]),
    "lbc_batch_remaining": (_S, [_P, _P, C.POINTER(C.c_int64)]),
    "lbc_batch_advance": (_S, [_P, C.c_int64, _P, C.POINTER(_P), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int64)]),
    "lbc_batch_size": (C.c_int32, [_P]),
    "lbc_batch_set_option": (_S, [_P, C.c_int32, C.c_int64]),
    "lbc_batch_launches_per_step": (C.c_int64, [_P]),
    "lbc_batch_destroy": (_S, [_P]),
}

_lib = None


def library(build_if_missing=True):
    """Load liblbc.so (building it first if needed); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB) and build_if_missing:
        from .builder import build
        build()
    if not os.path.exists(LIB):
        raise RuntimeError("liblbc.so is not built; run paper_1406_2211_gb300.build")
    lib = C.CDLL(LIB)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    sizes = (C.c_size_t * 3)()
    lib.lbc_desc_sizes(sizes)
    want = (C.sizeof(lbc_lattice_desc), C.sizeof(lbc_coupling_desc),
            C.sizeof(lbc_particles_desc))
    if tuple(sizes) != want:
        raise RuntimeError("descriptor layout mismatch: %s vs %s" % (tuple(sizes), want))
    _lib = lib
    return lib


class LBCError(RuntimeError):
    def __init__(self, status, where):
        msg = library().lbc_status_string(status).decode()
        super().__init__("%s failed: %s (%d)" % (where, msg, status))
        self.status = status


def check(status, where):
    if status != LBC_OK:
        raise LBCError(status, where)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def lattice_desc(nx, ny, nz, collision="bgk", tau=1.0, mrt_lambda=(0, 0, 0, 0),
                 rho0=1.0, body_force=(0, 0, 0), walls=False,
                 wall_velocity=((0, 0, 0), (0, 0, 0)), storage="f32",
                 storage_scale=0.0):
    d = lbc_lattice_desc()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.collision = COLLISION[collision]
    d.tau = tau
    for k in range(4):
        d.mrt_lambda[k] = mrt_lambda[k]
    d.rho0 = rho0
    for k in range(3):
        d.body_force[k] = body_force[k]
    d.z_walls = 1 if walls else 0
    for w in range(2):
        for k in range(3):
            d.wall_velocity[w][k] = wall_velocity[w][k]
    d.storage = STORAGE[storage]
    d.storage_scale = storage_scale
    return d


def coupling_desc(kind="none", order=2, stencil="trilinear", gamma=1.0,
                  split="base", substeps=1):
    d = lbc_coupling_desc()
    d.kind = KIND[kind]
    d.order = order
    d.stencil = STENCIL[stencil]
    d.gamma = gamma
    d.split = SPLIT[split]
    d.substeps = substeps
    return d


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Box:
    """One simulation box in a torch-allocated device arena."""

    def __init__(self, lattice, coupling=None, max_particles=0, max_bonds=0,
                 stream=None, device="cuda"):
        import torch
        lib = library()
        self.lib = lib
        self.lattice = lattice
        self.coupling = coupling if coupling is not None else coupling_desc()
        self.shape = (lattice.nz, lattice.ny, lattice.nx)
        self.N = lattice.nx * lattice.ny * lattice.nz
        nbytes = C.c_size_t()
        check(lib.lbc_box_bytes_required(C.byref(lattice), C.byref(self.coupling),
                                         max_particles, max_bonds, C.byref(nbytes)),
              "lbc_box_bytes_required")
        self.arena = torch.empty(int(nbytes.value), dtype=torch.uint8, device=device)
        if self.arena.data_ptr() % 256:
            raise RuntimeError("arena is not 256-byte aligned")
        self.stream = stream
        h = C.c_void_p()
        check(lib.lbc_box_create(C.byref(lattice), C.byref(self.coupling), max_particles,
                                 max_bonds, C.c_void_p(self.arena.data_ptr()),
                                 int(nbytes.value), self._s(), C.byref(h)),
              "lbc_box_create")
        self.handle = h
        self.nparticles = 0
        self.device = device
        self.storage = {0: "f64", 1: "f32", 2: "f16dev", 3: "bf16dev"}[lattice.storage]
        self._sigma = None

    def _s(self):
        return _stream_handle(self.stream)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.lbc_box_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- state setters
    def init_equilibrium(self, rho=1.0, u=(0.0, 0.0, 0.0)):
        uu = (C.c_double * 3)(*u)
        check(self.lib.lbc_box_init_equilibrium(self.handle, rho, uu, self._s()),
              "lbc_box_init_equilibrium")

    def set_fields(self, rho, u):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        check(self.lib.lbc_box_set_fields(self.handle, _ptr(rho), _ptr(u), self._s()),
              "lbc_box_set_fields")

    def set_populations(self, fbar):
        f = np.ascontiguousarray(fbar, dtype=np.float64)
        assert f.shape == (19,) + self.shape
        check(self.lib.lbc_box_set_populations(self.handle, _ptr(f), self._s()),
              "lbc_box_set_populations")

    def get_populations(self):
        f = np.empty((19,) + self.shape)
        check(self.lib.lbc_box_get_populations(self.handle, _ptr(f), self._s()),
              "lbc_box_get_populations")
        return f

    def set_pending_force(self, Fa):
        F = None if Fa is None else np.ascontiguousarray(Fa, dtype=np.float64)
        check(self.lib.lbc_box_set_pending_force(self.handle, _ptr(F), self._s()),
              "lbc_box_set_pending_force")

    def set_particles(self, pos, vel=None, mass=None, ext_force=None, bonds=None,
                      bond_k=None, bond_r0=None, rigid=None):
        """rigid: dict(first, count, radius, k, repulsion_k[, ref]) or None."""
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        n = pos.shape[0]
        arrs = dict(pos=pos)
        d = lbc_particles_desc()
        d.n = n
        d.pos = _ptr(pos)
        if vel is not None:
            arrs["vel"] = np.ascontiguousarray(vel, dtype=np.float64).reshape(n, 3)
            d.vel = _ptr(arrs["vel"])
        if mass is not None:
            arrs["mass"] = np.ascontiguousarray(
                np.broadcast_to(np.asarray(mass, dtype=np.float64), (n,)))
            d.mass = _ptr(arrs["mass"])
        if ext_force is not None:
            arrs["ext"] = np.ascontiguousarray(ext_force, dtype=np.float64).reshape(n, 3)
            d.ext_force = _ptr(arrs["ext"])
        if bonds is not None and len(bonds):
            bij = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
            nb = bij.shape[0]
            bk = np.ascontiguousarray(np.broadcast_to(np.asarray(bond_k, dtype=np.float64), (nb,)))
            br = np.ascontiguousarray(np.broadcast_to(np.asarray(bond_r0, dtype=np.float64), (nb,)))
            arrs.update(bij=bij, bk=bk, br=br)
            d.nbonds = nb
            d.bond_ij, d.bond_k, d.bond_r0 = _ptr(bij), _ptr(bk), _ptr(br)
        if rigid is not None:
            rf = np.ascontiguousarray(rigid["first"], dtype=np.int32).reshape(-1)
            rc = np.ascontiguousarray(rigid["count"], dtype=np.int32).reshape(-1)
            rr = np.ascontiguousarray(np.broadcast_to(np.asarray(rigid["radius"], dtype=np.float64),
                                                      rf.shape))
            arrs.update(rf=rf, rc=rc, rr=rr)
            d.nrigid = rf.shape[0]
            d.rigid_first, d.rigid_count, d.rigid_radius = _ptr(rf), _ptr(rc), _ptr(rr)
            if rigid.get("ref") is not None:
                arrs["rq"] = np.ascontiguousarray(rigid["ref"], dtype=np.float64).reshape(n, 3)
                d.rigid_ref = _ptr(arrs["rq"])
            d.rigid_k = float(rigid["k"])
            d.rigid_repulsion_k = float(rigid.get("repulsion_k", 0.0))
        check(self.lib.lbc_box_set_particles(self.handle, C.byref(d), self._s()),
              "lbc_box_set_particles")
        self.nparticles = n

    def set_option(self, option, value):
        check(self.lib.lbc_box_set_option(self.handle, option, value), "lbc_box_set_option")

    def set_thermal(self, kT, seed=0, printed_amplitude=None):
        """Thermal fluctuations at temperature kT (0: off): the fluid's
        moments and the random force of force-coupled particles.
        printed_amplitude: True / False selects the kick amplitude
        (LBC_OPT_THERMAL_AMPLITUDE) first; None leaves it."""
        if printed_amplitude is not None:
            self.set_option(LBC_OPT_THERMAL_AMPLITUDE, 1 if printed_amplitude else 0)
        check(self.lib.lbc_box_set_thermal(self.handle, float(kT), int(seed)),
              "lbc_box_set_thermal")

    def stress_output(self, enable=True):
        """Let every LB step write the viscous stress of the populations it
        collides into a device tensor sigma[6][nz][ny][nx] (the compute
        type: float64 for FP64 storage, else float32), returned here; the
        tensor is read after the step.  enable=False stops it."""
        import torch
        if not enable:
            check(self.lib.lbc_box_set_stress_output(self.handle, None, 0),
                  "lbc_box_set_stress_output")
            self._sigma = None
            return None
        dt = torch.float64 if self.storage == "f64" else torch.float32
        sig = torch.zeros((6,) + self.shape, dtype=dt, device=self.device)
        check(self.lib.lbc_box_set_stress_output(self.handle, C.c_void_p(sig.data_ptr()),
                                                 sig.numel() * sig.element_size()),
              "lbc_box_set_stress_output")
        self._sigma = sig           # kept alive while the library writes it
        return sig

    def get_option(self, option):
        v = C.c_int64()
        check(self.lib.lbc_box_get_option(self.handle, option, C.byref(v)), "lbc_box_get_option")
        return int(v.value)

    # --- stepping and observables
    def step(self, nsteps=1):
        check(self.lib.lbc_box_step(self.handle, nsteps, self._s()), "lbc_box_step")

    def get_fields(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        check(self.lib.lbc_box_get_fields(self.handle, _ptr(rho), _ptr(u), self._s()),
              "lbc_box_get_fields")
        return rho, u

    def autotune(self):
        """Tune the LB launch shape (lbc_box_autotune); returns (bx, by)."""
        bx, by = C.c_int32(), C.c_int32()
        check(self.lib.lbc_box_autotune(self.handle, self._s(), C.byref(bx), C.byref(by)),
              "lbc_box_autotune")
        return int(bx.value), int(by.value)

    def get_stress(self):
        """Viscous stress sigma[6][nz][ny][nx] (xx, yy, zz, xy, yz, xz)."""
        sig = np.empty((6,) + self.shape)
        check(self.lib.lbc_box_get_stress(self.handle, _ptr(sig), self._s()),
              "lbc_box_get_stress")
        return sig

    def get_particles(self):
        n = self.nparticles
        pos, vel, fh = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
        check(self.lib.lbc_box_get_particles(self.handle, _ptr(pos), _ptr(vel), _ptr(fh),
                                             self._s()), "lbc_box_get_particles")
        return pos, vel, fh

    def invariants(self):
        m = np.zeros(1)
        p = np.zeros(3)
        st = self.lib.lbc_box_invariants(self.handle, _ptr(m), _ptr(p), self._s())
        return float(m[0]), p, st

    def status(self):
        return self.lib.lbc_box_status(self.handle)

    def check(self):
        """Synchronise and latch the device flags (lbc_box_check); returns
        the box's status code (0 = ok)."""
        return int(self.lib.lbc_box_check(self.handle, self._s()))

    def launches_per_step(self):
        return int(self.lib.lbc_box_launches_per_step(self.handle))

    def lb_timing(self, reset=True):
        ms = C.c_double()
        n = C.c_int64()
        check(self.lib.lbc_box_lb_timing(self.handle, C.byref(ms), C.byref(n), 1 if reset else 0),
              "lbc_box_lb_timing")
        return float(ms.value), int(n.value)

    def population_bytes(self):
        return int(self.lib.lbc_box_population_bytes(self.handle))


class Batch:
    """A set of boxes advanced together (lbc_batch_*): continuous batching.

    The box tables live in a torch-allocated device arena.  `add` admits a
    Box with a step budget, `advance` moves every member forward and returns
    the Boxes whose budget is spent (they leave the batch)."""

    def __init__(self, max_boxes, stream=None, device="cuda"):
        import torch
        lib = library()
        self.lib = lib
        self.max_boxes = max_boxes
        nbytes = int(lib.lbc_batch_bytes_required(max_boxes))
        if nbytes == 0:
            raise LBCError(LBC_ERR_ARG, "lbc_batch_bytes_required")
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream
        h = C.c_void_p()
        check(lib.lbc_batch_create(max_boxes, C.c_void_p(self.arena.data_ptr()), nbytes,
                                   C.byref(h)), "lbc_batch_create")
        self.handle = h
        self.members = {}          # handle value -> Box

    def _s(self):
        return _stream_handle(self.stream)

    def add(self, box, steps):
        """Admit `box` for `steps` steps; returns False if no slot is free."""
        st = self.lib.lbc_batch_add(self.handle, box.handle, int(steps))
        if st == LBC_ERR_OOM:
            return False
        check(st, "lbc_batch_add")
        self.members[box.handle.value] = box
        return True

    def remove(self, box):
        check(self.lib.lbc_batch_remove(self.handle, box.handle), "lbc_batch_remove")
        self.members.pop(box.handle.value, None)

    def remaining(self, box):
        n = C.c_int64()
        check(self.lib.lbc_batch_remaining(self.handle, box.handle, C.byref(n)),
              "lbc_batch_remaining")
        return int(n.value)

    def advance(self, max_steps):
        """Advance all members by min(max_steps, smallest budget) steps;
        returns (steps done, list of finished Boxes)."""
        fin = (C.c_void_p * self.max_boxes)()
        nfin = C.c_int32()
        done = C.c_int64()
        check(self.lib.lbc_batch_advance(self.handle, int(max_steps), self._s(), fin,
                                         C.byref(nfin), C.byref(done)), "lbc_batch_advance")
        out = [self.members.pop(fin[k]) for k in range(nfin.value)]
        return int(done.value), out

    def __len__(self):
        return int(self.lib.lbc_batch_size(self.handle))

    def launches_per_step(self):
        return int(self.lib.lbc_batch_launches_per_step(self.handle))

    def set_launch(self, mode):
        """How members' particle work runs: "auto", "streams" or "batched"
        (LBC_BATCH_OPT_LAUNCH)."""
        v = {"auto": LBC_BATCH_LAUNCH_AUTO, "streams": LBC_BATCH_LAUNCH_STREAMS,
             "batched": LBC_BATCH_LAUNCH_BATCHED}[mode]
        check(self.lib.lbc_batch_set_option(self.handle, LBC_BATCH_OPT_LAUNCH, v),
              "lbc_batch_set_option")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.lbc_batch_destroy(self.handle)
            self.handle = None
            self.members = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
