"""Discrete delta functions, interpolation and spreading (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  delta_a(x) = phi(x/a) phi(y/a) phi(z/a)                       (App. A)
  u(X)  = sum_x u(x) delta_a(X - x)            Eq. [IBM-interpolation]
  F(x)  = a^-3 sum_i F_i delta_a(X_i - x)      Eq. [IBM-spreading]

with a = 1.  Kernels phi:
  trilinear  phi(r) = max(0, 1 - |r|)   (the linear interpolation App. A
             attributes to Ahlrichs & Duenweg)
  peskin3    the three-point function printed in App. A
  peskin4    Peskin's four-point function (not printed in the paper, which
             cites Peskin 2002 for the construction):
               (3 - 2|r| + sqrt(1 + 4|r| - 4 r^2)) / 8     |r| <= 1
               (5 - 2|r| - sqrt(-7 + 12|r| - 4 r^2)) / 8   1 <= |r| <= 2
The sums below run over every node whose weight can be non-zero (a window of
five nodes per axis around floor(X)); nodes are wrapped periodically, and on
an axis closed by walls, nodes outside [0, n) are dropped.
"""
import numpy as np


def phi_trilinear(r):
    return np.maximum(0.0, 1.0 - np.abs(r))


def phi_peskin3(r):
    a = np.abs(r)
    out = np.zeros_like(a)
    m1 = a <= 0.5
    m2 = (a > 0.5) & (a <= 1.5)
    out[m1] = (1.0 + np.sqrt(1.0 - 3.0 * a[m1] ** 2)) / 3.0
    out[m2] = (5.0 - 3.0 * a[m2]
               - np.sqrt(np.maximum(0.0, 6.0 * a[m2] - 2.0 - 3.0 * a[m2] ** 2))
               ) / 6.0
    return out


def phi_peskin4(r):
    a = np.abs(r)
    out = np.zeros_like(a)
    m1 = a <= 1.0
    m2 = (a > 1.0) & (a <= 2.0)
    out[m1] = (3.0 - 2.0 * a[m1] + np.sqrt(1.0 + 4.0 * a[m1] - 4.0 * a[m1] ** 2)) / 8.0
    out[m2] = (5.0 - 2.0 * a[m2]
               - np.sqrt(np.maximum(0.0, -7.0 + 12.0 * a[m2] - 4.0 * a[m2] ** 2))
               ) / 8.0
    return out


PHI = {'trilinear': phi_trilinear, 'peskin3': phi_peskin3,
       'peskin4': phi_peskin4}

WINDOW = np.arange(-2, 3)      # node offsets from floor(X) that may carry weight


def axis_weights(X, n, phi, closed=False):
    """Node indices (M, 5) and weights phi(X - node) (M, 5) along one axis."""
    base = np.floor(X).astype(np.int64)
    nodes = base[:, None] + WINDOW[None, :]
    wts = phi(X[:, None] - nodes.astype(np.float64))
    if closed:
        outside = (nodes < 0) | (nodes >= n)
        wts = np.where(outside, 0.0, wts)
        nodes = np.clip(nodes, 0, n - 1)
    else:
        nodes = np.mod(nodes, n)
    return nodes, wts


def stencil(pos, shape, kind, walls=False):
    """Flat node indices (M, 125) and weights delta(X - x) (M, 125).

    pos: (M, 3) positions (x, y, z); shape: (nz, ny, nx).
    """
    nz, ny, nx = shape
    phi = PHI[kind]
    ix, wx = axis_weights(pos[:, 0], nx, phi)
    iy, wy = axis_weights(pos[:, 1], ny, phi)
    iz, wz = axis_weights(pos[:, 2], nz, phi, closed=walls)
    flat = (iz[:, :, None, None] * ny + iy[:, None, :, None]) * nx + ix[:, None, None, :]
    wt = wz[:, :, None, None] * wy[:, None, :, None] * wx[:, None, None, :]
    M = pos.shape[0]
    nn = WINDOW.size ** 3
    return flat.reshape(M, nn), wt.reshape(M, nn)


def interpolate(field, pos, kind, walls=False):
    """u(X_i) = sum_x field(x) delta(X_i - x); field (3, nz, ny, nx) -> (M, 3)."""
    flat, wt = stencil(pos, field.shape[1:], kind, walls)
    out = np.empty((pos.shape[0], 3))
    for a in range(3):
        comp = field[a].reshape(-1)
        out[:, a] = (comp[flat] * wt).sum(axis=1)
    return out


def spread(forces, pos, shape, kind, walls=False):
    """F(x) = sum_i F_i delta(X_i - x) (a = 1); forces (M, 3) -> (3, nz, ny, nx)."""
    flat, wt = stencil(pos, shape, kind, walls)
    out = np.zeros((3, int(np.prod(shape))))
    for a in range(3):
        np.add.at(out[a], flat.reshape(-1), (wt * forces[:, a:a + 1]).reshape(-1))
    return out.reshape((3,) + tuple(shape))
