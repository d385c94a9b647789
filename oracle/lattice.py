"""D3Q19 lattice, equilibrium, force term and MRT moment basis (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper keeps the velocity set generic (Sec. 2: the c_i are the abscissae of
a Gauss-Hermite quadrature).  The lattice below is D3Q19, which the paper
does not name; its weights are the standard ones (rest 1/3, six face links
1/18, twelve edge links 1/36) with c_s^2 = 1/3 in lattice units (h = a = 1).

Readings (the paper gives no explicit formulas for these):
  * f^eq is the second-order Hermite equilibrium
        f_i^eq = w_i rho [1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2)]
    whose moments are those listed after Eq. [He-trafo1] (rho, rho u and
    Pi = rho cs2 I + rho u u).
  * G_i is the second-order Hermite force term
        G_i = w_i [c.F/cs2 + (c.u)(c.F)/cs2^2 - u.F/cs2]
    which has the moments of Eq. [force-moments]:
    sum G = 0, sum c G = F, sum c c G = F u + u F.
  * The MRT basis (Sec. 3.2, Eq. [mrt-coll]; Alg. 1 uses e_ki and b_k but the
    paper lists no basis) is a w-orthogonal polynomial basis: 1; c;
    c^2-1; 3cx^2-c^2, cy^2-cz^2, cx cy, cy cz, cx cz; (3c^2-5)c;
    (cy^2-cz^2)cx, (cz^2-cx^2)cy, (cx^2-cy^2)cz; 3c^4-6c^2+1;
    (2c^2-3)(3cx^2-c^2), (2c^2-3)(cy^2-cz^2).  b_k = sum_i w_i e_ki^2 is the
    squared length named in Sec. 3.2.  Relaxation groups: bulk {4},
    shear {5..9}, odd ghosts {10..15}, even ghosts {16..18}.
"""
import numpy as np

CS2 = 1.0 / 3.0
Q = 19

# velocity set; index order: rest, 6 faces (+x,-x,+y,-y,+z,-z), 12 edges in
# opposite pairs
C = np.array([
    [0, 0, 0],
    [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
    [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
    [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1],
], dtype=np.int64)
CF = C.astype(np.float64)
W = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)


def opposite():
    """Index of -c_i for every i (found by search, not by table)."""
    opp = np.empty(Q, dtype=np.int64)
    for i in range(Q):
        opp[i] = [j for j in range(Q) if np.all(C[j] == -C[i])][0]
    return opp


OPP = opposite()


def density(f):
    """rho = sum_i f_i  (Sec. 2, moments after Eq. [He-trafo1])."""
    return f.sum(axis=0)


def momentum(f):
    """rho u = sum_i f_i c_i; returns shape (3, ...)."""
    return np.tensordot(CF.T, f, axes=([1], [0]))


def equilibrium(rho, u):
    """Second-order equilibrium f_i^eq(rho, u); rho (...), u (3, ...)."""
    cu = np.tensordot(CF, u, axes=([1], [0]))          # (19, ...)
    uu = (u * u).sum(axis=0)
    return W.reshape((Q,) + (1,) * rho.ndim) * rho * (
        1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2))


def force_term(u, F):
    """Hermite force term G_i(u, F) with the moments of Eq. [force-moments]."""
    cu = np.tensordot(CF, u, axes=([1], [0]))
    cF = np.tensordot(CF, F, axes=([1], [0]))
    uF = (u * F).sum(axis=0)
    return W.reshape((Q,) + (1,) * uF.ndim) * (
        cF / CS2 + cu * cF / (CS2 * CS2) - uF / CS2)


def mrt_basis():
    """Rows e_k (k = 0..18) of the w-orthogonal moment basis, and b_k."""
    cx, cy, cz = CF.T
    c2 = cx * cx + cy * cy + cz * cz
    E = np.array([
        np.ones(Q), cx, cy, cz,
        c2 - 1.0,
        3.0 * cx * cx - c2, cy * cy - cz * cz, cx * cy, cy * cz, cx * cz,
        (3.0 * c2 - 5.0) * cx, (3.0 * c2 - 5.0) * cy, (3.0 * c2 - 5.0) * cz,
        (cy * cy - cz * cz) * cx, (cz * cz - cx * cx) * cy,
        (cx * cx - cy * cy) * cz,
        3.0 * c2 * c2 - 6.0 * c2 + 1.0,
        (2.0 * c2 - 3.0) * (3.0 * cx * cx - c2),
        (2.0 * c2 - 3.0) * (cy * cy - cz * cz),
    ])
    b = (E * E * W).sum(axis=1)
    return E, b


MRT_E, MRT_B = mrt_basis()
# group of each moment: 0 conserved, 1 bulk, 2 shear, 3 odd ghost, 4 even ghost
MRT_GROUP = np.array([0, 0, 0, 0, 1, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 4, 4, 4])


def mrt_rates(tau, mrt_lambda):
    """Full-step eigenvalues lambda_k of the discrete collision matrix.

    mrt_lambda = (shear, bulk, odd ghost, even ghost); a zero entry takes the
    default: shear = 1/tau, bulk = shear, ghosts = 1 (fully relaxed).
    Conserved moments get lambda = 0.
    """
    lam_s = mrt_lambda[0] if mrt_lambda[0] != 0 else 1.0 / tau
    lam_b = mrt_lambda[1] if mrt_lambda[1] != 0 else lam_s
    lam_go = mrt_lambda[2] if mrt_lambda[2] != 0 else 1.0
    lam_ge = mrt_lambda[3] if mrt_lambda[3] != 0 else 1.0
    by_group = np.array([0.0, lam_b, lam_s, lam_go, lam_ge])
    return by_group[MRT_GROUP]
