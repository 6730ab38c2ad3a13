"""Oracle: training-pair sampler and its bead-sum labels (FP64).

TEST INFRASTRUCTURE (see the package docstring).

The paper samples pair configurations from HOOMD trajectories and expresses
each in the frame of body 1 (Methods; SI Sec. 1).  Those trajectories are not
available, so the workload instead draws configurations directly: body i at
the origin with identity orientation, body j along a uniformly random unit
direction u at a separation rho uniform between contact and the body-pair
cutoff, with a uniformly random orientation q_j.  The random numbers are
inputs (six uniforms in [0, 1) per sample), so both this oracle and the GPU
sampler consume the same draws:

  u0, u1 -> direction: z = 2 u0 - 1, phi = 2 pi u1, u = (sqrt(1-z^2) cos phi,
            sqrt(1-z^2) sin phi, z)
  u2, u3, u4 -> q_j by Shoemake's uniform-rotation construction
            (sqrt(1-u2) sin 2pi u3, sqrt(1-u2) cos 2pi u3,
             sqrt(u2) sin 2pi u4, sqrt(u2) cos 2pi u4) taken as (s, i, j, k)
  u5 -> rho = rho_c + u5 (Rc - rho_c)

Contact rho_c (unstated in the paper and the workload; reading used): the
separation along u at which the smallest bead-bead distance equals sigma,
found by N_BISECT bisection steps on [0, Rc] that keep
min_dist(lo) < sigma <= min_dist(hi) and return the midpoint of the final
interval.
"""
from __future__ import annotations

import numpy as np

from . import bead_pair, min_bead_distance

N_BISECT = 40


def draws_to_config(u):
    """Direction and orientation from the first five uniforms of each sample."""
    u = np.asarray(u, dtype=np.float64)
    z = 2.0 * u[:, 0] - 1.0
    phi = 2.0 * np.pi * u[:, 1]
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    d = np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)
    a, b = np.sqrt(1.0 - u[:, 2]), np.sqrt(u[:, 2])
    q = np.stack([a * np.sin(2 * np.pi * u[:, 3]), a * np.cos(2 * np.pi * u[:, 3]),
                  b * np.sin(2 * np.pi * u[:, 4]), b * np.cos(2 * np.pi * u[:, 4])], axis=1)
    return d, q


def contact_distance(direction, q_j, tmpl, Rc, sigma=1.0, n_iter=N_BISECT):
    """Bisection for the separation along `direction` where the minimum bead
    distance between the two bodies (i at the origin, identity orientation)
    equals sigma."""
    zero = np.zeros(3)
    one = np.array([1.0, 0.0, 0.0, 0.0])
    nobox = np.zeros(3)
    lo, hi = 0.0, float(Rc)
    for _ in range(n_iter):
        mid = 0.5 * (lo + hi)
        if min_bead_distance(zero, one, mid * np.asarray(direction), q_j, nobox, tmpl) < sigma:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def sample_pairs(u, tmpl, Rc, eps=1.0, sigma=1.0, rc=2.5, contact=None):
    """Pair configurations (B, 7) = (s, q_rel) and bead-sum labels (B, 10) =
    (E, F_j, tau_i, tau_j), all in the frame of body i; also rho_c (B,).
    `contact` (default sigma) is the smallest bead-bead distance that defines
    contact: below sigma the draws reach into the repulsive wall."""
    contact = sigma if contact is None else contact
    u = np.asarray(u, dtype=np.float64)
    d, q = draws_to_config(u)
    B = len(u)
    cfg = np.zeros((B, 7))
    lab = np.zeros((B, 10))
    rho_c = np.zeros(B)
    zero = np.zeros(3)
    one = np.array([1.0, 0.0, 0.0, 0.0])
    for b in range(B):
        rho_c[b] = contact_distance(d[b], q[b], tmpl, Rc, contact)
        rho = rho_c[b] + u[b, 5] * (Rc - rho_c[b])
        s = rho * d[b]
        r = bead_pair(zero, one, s, q[b], np.zeros(3), tmpl, tmpl, eps, sigma, rc)
        cfg[b, :3] = s
        cfg[b, 3:] = q[b]
        lab[b] = np.concatenate([[r["E"]], r["F_j"], r["tau_i"], r["tau_j"]])
    return cfg, lab, rho_c


def label_pairs(cfg, tmpl, eps=1.0, sigma=1.0, rc=2.5):
    """Bead-sum labels (B, 10) for given pair configurations (s, q_rel)."""
    cfg = np.asarray(cfg, dtype=np.float64)
    zero = np.zeros(3)
    one = np.array([1.0, 0.0, 0.0, 0.0])
    out = np.zeros((len(cfg), 10))
    for b in range(len(cfg)):
        r = bead_pair(zero, one, cfg[b, :3], cfg[b, 3:7], np.zeros(3), tmpl, tmpl, eps, sigma, rc)
        out[b] = np.concatenate([[r["E"]], r["F_j"], r["tau_i"], r["tau_j"]])
    return out


def swap_reference(cfg, labels):
    """The same pairs described from the other body.  A pair configuration
    is given in the frame of its first body (SI Sec. 1): separation s and
    relative orientation q of the second body, the first at the origin with
    the identity orientation.  Taking the second body as the reference puts
    the first at s' = R(q)^T (-s) with orientation q' = q^*, and the labels
    (E, F on the second body, tau on the first, tau on the second) become
    E' = E, F' = R(q)^T (-F), tau'_1 = R(q)^T tau_2, tau'_2 = R(q)^T tau_1.
    cfg (B, 7) = (s, q); labels (B, 10) = (E, F_j, tau_i, tau_j)."""
    from . import bodies

    cfg = np.asarray(cfg, dtype=np.float64)
    lab = np.asarray(labels, dtype=np.float64)
    s, q = cfg[:, :3], cfg[:, 3:7]
    qc = bodies.qconj(q)
    out_cfg = np.concatenate([bodies.qrotate(qc, -s), qc], axis=1)
    out_lab = np.concatenate([lab[:, :1], bodies.qrotate(qc, -lab[:, 1:4]),
                              bodies.qrotate(qc, lab[:, 7:10]), bodies.qrotate(qc, lab[:, 4:7])], axis=1)
    return out_cfg, out_lab
