"""Pins for oracle/delta.py: the conditions of App. A and their consequences.

  Eq. [delta1]  sum_j phi(r - j) = 1
  Eq. [delta2]  sum_j j phi(r - j) = r
  Eq. [delta3]  sum_j phi(r - j)^2 = C  (1/2 for the three-point function;
                3/8 for Peskin's four-point function)
  total force and torque on the grid equal the Lagrangian totals (App. A);
  spreading is the adjoint of interpolation (Sec. 5.1, Eq. [IBM-spreading]).
"""
import numpy as np
import pytest

from oracle import delta


@pytest.mark.parametrize("kind", ["trilinear", "peskin3", "peskin4"])
def test_partition_of_unity_and_first_moment(kind, rng):
    phi = delta.PHI[kind]
    r = rng.uniform(-3, 3, size=200)
    j = np.arange(-6, 7)
    vals = phi(r[:, None] - j[None, :])
    assert np.abs(vals.sum(axis=1) - 1.0).max() < 1e-14
    assert np.abs((vals * j).sum(axis=1) - r).max() < 1e-13


@pytest.mark.parametrize("kind,C", [("peskin3", 0.5), ("peskin4", 3.0 / 8.0)])
def test_sum_of_squares_constant(kind, C, rng):
    phi = delta.PHI[kind]
    r = rng.uniform(-3, 3, size=200)
    j = np.arange(-6, 7)
    vals = phi(r[:, None] - j[None, :])
    assert np.abs((vals ** 2).sum(axis=1) - C).max() < 1e-14


def test_trilinear_sum_of_squares_not_constant():
    phi = delta.PHI["trilinear"]
    j = np.arange(-3, 4)
    s0 = (phi(0.0 - j) ** 2).sum()
    s5 = (phi(0.5 - j) ** 2).sum()
    assert abs(s0 - 1.0) < 1e-15 and abs(s5 - 0.5) < 1e-15


@pytest.mark.parametrize("kind,edges", [("peskin3", (0.5, 1.5)),
                                        ("peskin4", (1.0, 2.0))])
def test_continuity_at_piece_boundaries(kind, edges):
    phi = delta.PHI[kind]
    for e in edges:
        lo = phi(np.array([e - 1e-12]))[0]
        hi = phi(np.array([e + 1e-12]))[0]
        assert abs(lo - hi) < 1e-5
    assert phi(np.array([edges[1] + 1e-9]))[0] == 0.0


def test_peskin3_center_value():
    # phi_3(0) = (1 + 1)/3 from the closed form in App. A
    assert abs(delta.phi_peskin3(np.array([0.0]))[0] - 2.0 / 3.0) < 1e-15


@pytest.mark.parametrize("kind", ["trilinear", "peskin3", "peskin4"])
def test_spread_conserves_force_and_torque(kind, rng):
    shape = (16, 14, 12)
    nz, ny, nx = shape
    M = 11
    # keep markers away from the periodic seams so torques need no image
    pos = np.column_stack([rng.uniform(3, nx - 4, M), rng.uniform(3, ny - 4, M),
                           rng.uniform(3, nz - 4, M)])
    F = rng.standard_normal((M, 3))
    grid = delta.spread(F, pos, shape, kind)
    assert np.abs(grid.reshape(3, -1).sum(axis=1) - F.sum(axis=0)).max() < 1e-13
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                          indexing="ij")
    xyz = np.stack([x, y, z]).reshape(3, -1).astype(float)
    tq_grid = np.cross(xyz.T, grid.reshape(3, -1).T).sum(axis=0)
    tq_lag = np.cross(pos, F).sum(axis=0)
    assert np.abs(tq_grid - tq_lag).max() < 1e-12


@pytest.mark.parametrize("kind", ["trilinear", "peskin3", "peskin4"])
@pytest.mark.parametrize("walls", [False, True])
def test_spread_is_adjoint_of_interpolation(kind, walls, rng):
    shape = (7, 5, 6)
    M = 9
    pos = rng.uniform(0, 1, (M, 3)) * np.array([6, 5, 7])
    F = rng.standard_normal((M, 3))
    u = rng.standard_normal((3,) + shape)
    lhs = (delta.spread(F, pos, shape, kind, walls) * u).sum()
    rhs = (F * delta.interpolate(u, pos, kind, walls)).sum()
    assert abs(lhs - rhs) < 1e-12


@pytest.mark.parametrize("kind", ["trilinear", "peskin3", "peskin4"])
def test_interpolation_exact_for_linear_fields(kind, rng):
    """Eqs. [delta1]-[delta2] make linear fields interpolate exactly."""
    shape = (20, 20, 20)
    z, y, x = np.meshgrid(*(np.arange(20.0),) * 3, indexing="ij")
    a = rng.standard_normal((3, 4))
    u = np.stack([a[c, 0] + a[c, 1] * x + a[c, 2] * y + a[c, 3] * z
                  for c in range(3)])
    pos = rng.uniform(4, 15, (13, 3))
    got = delta.interpolate(u, pos, kind)
    expect = (a[:, 0][None, :] + pos @ a[:, 1:].T)
    assert np.abs(got - expect).max() < 1e-12


def test_tiny_periodic_box_folds_the_stencil():
    """On a one-cell periodic axis every stencil node is the same node."""
    shape = (1, 1, 1)
    pos = np.array([[0.3, 0.7, 0.1]])
    for kind in ("trilinear", "peskin3", "peskin4"):
        g = delta.spread(np.array([[1.0, 2.0, 3.0]]), pos, shape, kind)
        assert np.allclose(g[:, 0, 0, 0], [1.0, 2.0, 3.0], atol=1e-15)


def _golden_phi3():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "phi3_printed_values.txt")
    pts, C = [], None
    for line in open(path):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "C":
            C = int(line[1]) / int(line[2])
        else:
            rn, rd, pn, pd = (int(v) for v in line)
            pts.append((rn / rd, pn / pd))
    return pts, C


def test_phi3_matches_printed_values():
    """phi_3 at the points where the appendix's printed closed form is
    rational (tests/golden/phi3_printed_values.txt), and its Eq. [delta3]
    constant from those values."""
    from oracle import delta as OD
    pts, C = _golden_phi3()
    r = np.array([p[0] for p in pts])
    assert np.allclose(OD.phi_peskin3(r), [p[1] for p in pts], rtol=0, atol=1e-15)
    for x in np.linspace(-0.5, 0.5, 11):
        j = np.arange(-3, 4)
        assert abs((OD.phi_peskin3(x - j) ** 2).sum() - C) < 1e-15
