"""Oracle: composite rigid bodies and quaternion algebra (numpy FP64).

TEST INFRASTRUCTURE (see the package docstring).

A composite rigid body is a fixed set of beads in its body frame plus the
centre-of-mass position p and the unit orientation quaternion q = (s, i, j, k)
(paper, Methods and SI Sec. 1, which lists p and q as the raw pair
configuration).  The paper does not fix the quaternion convention; the reading
used here is scalar first, Hamilton product, active rotation v' = q v q*.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- templates

def cube_template(n_side: int = 5, spacing: float = 1.0) -> np.ndarray:
    """Simple-cubic n_side^3 bead lattice centred on the origin (5x5x5 = 125
    beads at spacing 1 sigma for the workload's cubes)."""
    ax = (np.arange(n_side) - (n_side - 1) / 2.0) * spacing
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    return np.ascontiguousarray(g, dtype=np.float64)


def hex_disc(radius: float = 2.0, spacing: float = 1.0) -> np.ndarray:
    """All points of a triangular (hexagonal-packed) lattice of the given
    spacing within `radius` of the origin, in the xy plane."""
    n = int(np.ceil(radius / spacing)) + 2
    pts = []
    for a in range(-n, n + 1):
        for b in range(-n, n + 1):
            x = (a + 0.5 * b) * spacing
            y = b * np.sqrt(3.0) / 2.0 * spacing
            if x * x + y * y <= radius * radius + 1e-9:
                pts.append((x, y))
    return np.array(pts, dtype=np.float64)


def cylinder_template(n_layers: int = 8, radius: float = 2.0, spacing: float = 1.0,
                      length: float = 8.0) -> np.ndarray:
    """Stacked hexagonally packed discs (19 beads of radius 2 sigma per layer,
    8 layers spanning a bead-centre length of 8 sigma: aspect ratio 2, 152
    beads), centred on the origin with the axis along z."""
    disc = hex_disc(radius, spacing)
    zs = (np.arange(n_layers) - (n_layers - 1) / 2.0) * (length / (n_layers - 1))
    out = [np.column_stack([disc, np.full(len(disc), z)]) for z in zs]
    return np.ascontiguousarray(np.concatenate(out), dtype=np.float64)


def mass_and_inertia(tmpl: np.ndarray, bead_mass: float = 1.0):
    """Total mass and the inertia tensor I = sum m (|d|^2 1 - d d^T) of the
    bead template about its centre of mass (the templates are centred)."""
    d = np.asarray(tmpl, dtype=np.float64)
    M = bead_mass * len(d)
    I = np.zeros((3, 3))
    for v in d:
        I += bead_mass * (np.dot(v, v) * np.eye(3) - np.outer(v, v))
    return M, I


def circumradius(tmpl: np.ndarray) -> float:
    """Largest bead-centre distance from the centre of mass."""
    return float(np.max(np.linalg.norm(np.asarray(tmpl, dtype=np.float64), axis=1)))


def pair_cutoff(tmpl: np.ndarray, rc: float = 2.5) -> float:
    """Body-pair cutoff Rc = 2 r_circ + r_c: no bead pair of two bodies whose
    centres are farther apart can lie within r_c of each other."""
    return 2.0 * circumradius(tmpl) + rc


# ---------------------------------------------------------------- quaternions

def qmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton product of quaternions (scalar first), broadcasting over rows."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    aw, ax, ay, az = np.moveaxis(a, -1, 0)
    bw, bx, by, bz = np.moveaxis(b, -1, 0)
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def qconj(q: np.ndarray) -> np.ndarray:
    q = np.asarray(q, dtype=np.float64)
    return q * np.array([1.0, -1.0, -1.0, -1.0])


def qrotate(q: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Active rotation v' = q v q* (computed with the quaternion product)."""
    v = np.asarray(v, dtype=np.float64)
    vq = np.concatenate([np.zeros(v.shape[:-1] + (1,)), v], axis=-1)
    return qmul(qmul(q, vq), qconj(q))[..., 1:]


def qmatrix(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of a unit quaternion, built column by column from qrotate
    so that it does not restate the closed-form matrix used elsewhere."""
    q = np.asarray(q, dtype=np.float64)
    cols = [qrotate(q, np.broadcast_to(e, q.shape[:-1] + (3,))) for e in np.eye(3)]
    return np.stack(cols, axis=-1)


def qexp(omega: np.ndarray) -> np.ndarray:
    """Unit quaternion of the rotation vector omega (angle |omega| about
    omega/|omega|)."""
    omega = np.asarray(omega, dtype=np.float64)
    th = np.linalg.norm(omega, axis=-1, keepdims=True)
    s = np.where(th > 0, np.sin(th / 2) / np.where(th > 0, th, 1.0), 0.5)
    return np.concatenate([np.cos(th / 2), s * omega], axis=-1)


def min_image(d: np.ndarray, box) -> np.ndarray:
    """d - L * round-half-even(d / L), per axis."""
    box = np.asarray(box, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    return d - box * np.rint(d / box)
