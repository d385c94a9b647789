"""Seeded synthetic workloads (positions, bonds, meshes, fields, job lists).

No method arithmetic here: only geometry, random numbers and the parameter
presets of the five benchmark configurations.  Everything is NumPy and
deterministic for a given seed.

Coordinates are lattice units with cell (i, j, k) at position (i, j, k);
positions are returned as (M, 3) arrays in (x, y, z) order, fields as
(3, nz, ny, nx) / (nz, ny, nx) arrays.
"""
import math

import numpy as np

__all__ = [
    "D3Q19_WEIGHTS", "random_populations", "shear_wave", "rest_fields",
    "random_points", "bead_chains", "icosphere", "place_spheres",
    "fibonacci_sphere", "shells", "rigid_spheres", "ensemble_jobs", "CONFIGS", "config",
]

# lattice weights in the D3Q19 ordering used by both implementations: rest,
# +x, -x, +y, -y, +z, -z, then the twelve edge links in opposite pairs
D3Q19_WEIGHTS = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)


def random_populations(shape, seed, amp=1e-3, rho0=1.0):
    """Positive populations rho0 w_i (1 + amp xi_i), xi ~ U(-1, 1).

    A generic non-equilibrium state (random density, velocity and stress).
    Shape of the result: (19, nz, ny, nx).
    """
    rng = np.random.default_rng(seed)
    xi = rng.uniform(-1.0, 1.0, (19,) + tuple(shape))
    return rho0 * D3Q19_WEIGHTS.reshape(19, 1, 1, 1) * (1.0 + amp * xi)


def rest_fields(shape, rho0=1.0):
    return np.full(shape, rho0), np.zeros((3,) + tuple(shape))


def shear_wave(shape, U, comp=1, along=0, rho0=1.0):
    """u_comp = U sin(2 pi x_along / L) (a transverse shear wave)."""
    rho, u = rest_fields(shape, rho0)
    n = shape[2 - along]
    ph = np.sin(2.0 * np.pi * np.arange(n) / n)
    sl = [None, None, None]
    sl[2 - along] = slice(None)
    u[comp] = U * ph[tuple(sl)] * np.ones(shape)
    return rho, u


def random_points(n, box, seed):
    """n points uniform in [0, nx) x [0, ny) x [0, nz); box = (nx, ny, nz)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (n, 3)) * np.asarray(box, dtype=np.float64)


def bead_chains(nchains, beads, box, r0, seed):
    """Random-walk chains: heads uniform in the box, each next bead at
    distance r0 in a uniform random direction.  Returns (pos, bonds)."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    heads = rng.uniform(0.0, 1.0, (nchains, 3)) * box
    dirs = rng.standard_normal((nchains, beads - 1, 3))
    dirs /= np.linalg.norm(dirs, axis=2, keepdims=True)
    steps = np.concatenate([heads[:, None, :], r0 * dirs], axis=1)
    pos = np.cumsum(steps, axis=1).reshape(-1, 3)
    pos = np.mod(pos, box)
    pos = np.where(pos >= box, pos - box, pos)
    idx = np.arange(nchains * beads).reshape(nchains, beads)
    bonds = np.stack([idx[:, :-1].reshape(-1), idx[:, 1:].reshape(-1)], axis=1)
    return pos, bonds.astype(np.int32)


def icosphere(subdivisions):
    """Unit-sphere mesh from an icosahedron subdivided `subdivisions` times.

    Returns (vertices (V, 3), edges (E, 2)); 3 subdivisions give 642
    vertices and 1920 edges.
    """
    t = (1.0 + 5.0 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    for _ in range(subdivisions):
        cache = {}
        new_faces = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    edges = set()
    for a, b, c in faces:
        for p, q in ((a, b), (b, c), (c, a)):
            edges.add((min(p, q), max(p, q)))
    return np.array(verts), np.array(sorted(edges), dtype=np.int32)


def place_spheres(n, radius, box, seed, gap=1.0, wall_clearance=None,
                  max_tries=200000):
    """Centres of n non-overlapping spheres (centre distance >= 2R + gap).

    wall_clearance: if given, z centres keep that distance (plus R) from the
    walls at z = -1/2 and z = nz - 1/2; x and y are periodic.
    """
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    lo = np.zeros(3)
    hi = box.copy()
    if wall_clearance is not None:
        lo[2] = -0.5 + radius + wall_clearance
        hi[2] = box[2] - 0.5 - radius - wall_clearance
    centres = []
    tries = 0
    while len(centres) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place %d spheres" % n)
        c = lo + rng.uniform(0.0, 1.0, 3) * (hi - lo)
        ok = True
        for d in centres:
            dd = c - d
            dd[:2] -= box[:2] * np.rint(dd[:2] / box[:2])
            if wall_clearance is None:
                dd[2] -= box[2] * np.rint(dd[2] / box[2])
            if np.dot(dd, dd) < (2 * radius + gap) ** 2:
                ok = False
                break
        if ok:
            centres.append(c)
    return np.array(centres)


def fibonacci_sphere(n):
    """n quasi-uniform points on the unit sphere (golden-angle spiral)."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(1.0 - z * z)
    th = math.pi * (3.0 - 5.0 ** 0.5) * k
    return np.column_stack([r * np.cos(th), r * np.sin(th), z])


def shells(nshells, radius, box, seed, subdivisions=3, wall_clearance=3.0):
    """Icosphere shells of the given radius at non-overlapping positions.

    Returns (pos (nshells*V, 3), edges (nshells*E, 2), rest lengths)."""
    v, e = icosphere(subdivisions)
    centres = place_spheres(nshells, radius, box, seed, gap=2.0,
                            wall_clearance=wall_clearance)
    box = np.asarray(box, dtype=np.float64)
    pos = (centres[:, None, :] + radius * v[None, :, :]).reshape(-1, 3)
    pos[:, :2] = np.mod(pos[:, :2], box[:2])
    V = v.shape[0]
    edges = (e[None, :, :] + V * np.arange(nshells)[:, None, None]).reshape(-1, 2)
    r0 = np.tile(radius * np.linalg.norm(v[e[:, 0]] - v[e[:, 1]], axis=1), nshells)
    return pos, edges.astype(np.int32), r0


def rigid_spheres(nspheres, radius, markers, box, seed, gap=1.0):
    """Surface markers of non-overlapping spheres: Fibonacci points on each
    sphere of the given radius.  Returns (pos (n*markers, 3) wrapped into the
    periodic box, first (n,), count (n,))."""
    centres = place_spheres(nspheres, radius, box, seed, gap=gap)
    v = fibonacci_sphere(markers)
    box = np.asarray(box, dtype=np.float64)
    pos = (centres[:, None, :] + radius * v[None, :, :]).reshape(-1, 3)
    pos = np.mod(pos, box)
    pos = np.where(pos >= box, pos - box, pos)
    first = np.arange(nspheres) * markers
    count = np.full(nspheres, markers)
    return pos, first.astype(np.int32), count.astype(np.int32)


def ensemble_jobs(njobs, seed, edge_range=(32, 128), particles_range=(1, 5000),
                  gamma_range=(0.5, 10.0), steps_range=(1000, 20000),
                  rate=None):
    """Job list for the serving ensemble: per job edge L (log-uniform),
    particle count, friction, step count, storage kind, arrival time."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(edge_range[0]), math.log(edge_range[1])
    edges = np.rint(np.exp(rng.uniform(lo, hi, njobs))).astype(int)
    nparts = rng.integers(particles_range[0], particles_range[1] + 1, njobs)
    gammas = rng.uniform(gamma_range[0], gamma_range[1], njobs)
    steps = rng.integers(steps_range[0], steps_range[1] + 1, njobs)
    storage = np.where(rng.uniform(0, 1, njobs) < 0.5, "f32", "f16dev")
    if rate is None:
        arrivals = np.zeros(njobs)
    else:
        arrivals = np.cumsum(rng.exponential(1.0 / rate, njobs))
    seeds = rng.integers(0, 2 ** 31 - 1, njobs)
    return [dict(edge=int(edges[i]), nparticles=int(nparts[i]),
                 gamma=float(gammas[i]), steps=int(steps[i]),
                 storage=str(storage[i]), arrival=float(arrivals[i]),
                 seed=int(seeds[i])) for i in range(njobs)]


# Parameter presets of the five benchmark workloads.  Readings of the
# unspecified items are documented next to them.
CONFIGS = {
    "fc_point_particle_32": dict(
        box=(32, 32, 32), collision="bgk", tau=0.8, storage="f64", rho0=1.0,
        kind="fc", gamma=1.0, mass=1.0, stencil="trilinear",
        particle=(16.3, 16.7, 16.1), velocity=(0.01, 0.0, 0.0), steps=1000,
        orders=(2, 1)),
    "mrt_bead_chains_256": dict(
        box=(256, 256, 256), collision="mrt", tau=1.0, storage="f32",
        rho0=1.0, kind="fc", gamma=5.0, mass=1.0, stencil="trilinear",
        nchains=2000, beads=50, bond_k=10.0, bond_r0=1.0,
        body_force=(1e-6, 0.0, 0.0), steps=2000, seed=12345,
        # bond frequency sqrt(4k/m) ~ 6.3 needs particle sub-steps below
        # h/3; gamma = 5 is unstable with coupling-only half steps of h/2
        # once beads share stencil nodes, and with Eq. [multistep] at n = 2
        # for the full 2000 chains: Eq. [multistep] with n = 4 (dt = h/8)
        substeps=4, mode="inside"),
    "ibm_shells_192": dict(
        box=(192, 192, 192), collision="bgk", tau=1.0, storage="f32",
        rho0=1.0, kind="ibm", stencil="peskin4", nshells=64, radius=8.0,
        subdivisions=3, spring_k=0.05, walls=True,
        wall_velocity=((-0.05, 0.0, 0.0), (0.05, 0.0, 0.0)), seed=12345,
        steps=2000),
    "mebf_rigid_spheres_128": dict(
        box=(128, 128, 128), collision="bgk", tau=0.7, storage="f32",
        rho0=1.0, kind="mebf", stencil="peskin4", nspheres=500, radius=4.5,
        markers=400, seed=12345, steps=5000,
        # rigid-sphere model (not in the paper): markers of mass
        # rho0 (4/3) pi R^3 / markers tethered to the best-fit rigid frame
        # (stiffness rigid_k), soft repulsion below a one-unit gap
        rigid_k=1.0, repulsion_k=0.1),
    "serving_ensemble": dict(njobs=2000, seed=12345, collision="bgk", tau=0.8,
                          kind="fc", mass=1.0, stencil="trilinear"),
}


def config(name, scale=1):
    """A preset with the box divided by `scale` and particle counts scaled
    by scale^-3 (same densities), for reduced-size parity runs."""
    c = dict(CONFIGS[name])
    if scale != 1 and "box" in c:
        c["box"] = tuple(max(1, b // scale) for b in c["box"])
        for key in ("nchains", "nshells", "nspheres"):
            if key in c:
                c[key] = max(1, int(round(c[key] / scale ** 3)))
    return c
