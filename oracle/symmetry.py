"""Oracle: symmetry-reduced pair configurations (FP64).

TEST INFRASTRUCTURE (see the package docstring).

The paper reduces a cube-cube pair configuration to a canonical one before it
reaches the network (SI Sec. 1): body 1's frame is chosen among the cube's
equivalent face frames so that body 2's centre lies in one octant with
ordered coordinates (including a reflection across y = z), and body 2's
orientation is then described relative to the face closest to body 1.  Two
configurations related by a symmetry of either body have the same energy,
and the network sees only one of them.

Reading used here (the paper's angle parametrisation is not reproduced; it has
an unbounded derivative where two faces align, which the exact gradients below
cannot use):

  * G is the point group of the bead template: the proper rotations Q_k that
    map the template onto itself, plus the inversion d -> -d when the template
    is centrosymmetric.  For a bead potential that depends only on distances,
    E(s, q) = E(sigma R_k s, Q_k (x) q) for every Q_k in G and sigma = +-1 when
    the inversion is in G (rotating or inverting the whole pair about body 1's
    centre leaves body 1 in place), and E(s, q) = E(s, q (x) Q_j) (relabelling
    body 2's own axes).
  * Canonical choice: k maximises sigma (R_k s) . u_ref over the group (with
    the inversion: |(R_k s) . u_ref|, sigma its sign), u_ref = (3, 2, 1)/sqrt(14);
    then j maximises |scalar part of (Q_k (x) q (x) Q_j)|.  Ties go to the first
    element in the group order below.
  * The canonical configuration is (sigma R_k s, Q_k (x) q (x) Q_j); the usual
    features follow.  Within a choice the map is linear and orthogonal, so
    forces and torques transform back as F_j = sigma R_k^T F_j',
    tau = R_k^T tau'.
  * Group order: each element as a unit quaternion with its first non-zero
    component positive, sorted in decreasing lexicographic order of
    (w, x, y, z) rounded to 1e-9.

Candidate rotations for the point group are the closures of the cube's group
(generated by quarter turns about x and y) and of the hexagonal prism's group
(a sixth turn about z and a half turn about x); the templates built here
(cube, hexagonal-disc cylinder, rectangular boxes) have their symmetry axes
along the coordinate axes.
"""
from __future__ import annotations

import numpy as np
import torch

from . import bodies

U_REF = np.array([3.0, 2.0, 1.0]) / np.sqrt(14.0)


def _normalise_sign(q):
    q = np.asarray(q, dtype=np.float64)
    for c in range(4):
        if abs(q[c]) > 1e-12:
            return q if q[c] > 0 else -q
    return q


def _closure(generators):
    """All products of the generators (unit quaternions, q and -q identified)."""
    found = [np.array([1.0, 0.0, 0.0, 0.0])]
    frontier = list(found)
    while frontier:
        nxt = []
        for a in frontier:
            for g in generators:
                c = _normalise_sign(bodies.qmul(g, a))
                if not any(np.allclose(c, f, atol=1e-9) for f in found):
                    found.append(c)
                    nxt.append(c)
        frontier = nxt
    return found


def _sorted(quats):
    key = lambda q: tuple(-np.round(q, 9))
    return sorted((_normalise_sign(q) for q in quats), key=key)


def candidate_rotations():
    cube = _closure([bodies.qexp(np.array([np.pi / 2, 0.0, 0.0])),
                     bodies.qexp(np.array([0.0, np.pi / 2, 0.0]))])
    hexa = _closure([bodies.qexp(np.array([0.0, 0.0, np.pi / 3])),
                     bodies.qexp(np.array([np.pi, 0.0, 0.0]))])
    out = list(cube)
    for q in hexa:
        if not any(np.allclose(q, f, atol=1e-9) for f in out):
            out.append(q)
    return out


def _maps_onto(tmpl, moved, tol):
    d = np.linalg.norm(moved[:, None, :] - tmpl[None, :, :], axis=-1)
    return bool(np.all(d.min(axis=1) < tol))


def point_group(tmpl, tol: float = 1e-6):
    """(quats (n, 4) in group order, inversion) of the template's point group
    among the candidate rotations."""
    tmpl = np.asarray(tmpl, dtype=np.float64)
    keep = [q for q in candidate_rotations() if _maps_onto(tmpl, bodies.qrotate(
        np.broadcast_to(q, (len(tmpl), 4)), tmpl), tol)]
    inversion = _maps_onto(tmpl, -tmpl, tol)
    return np.array(_sorted(keep)), inversion


def choose(s, q, group):
    """Per pair: (k, sigma, j, margin_k, margin_j) of the canonical choice;
    the margins are the gaps between the best and second-best scores."""
    quats, inversion = group
    s = np.asarray(s, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1, 4)
    R = bodies.qmatrix(quats)                       # (G, 3, 3)
    score = np.einsum("kij,bj,i->bk", R, s, U_REF)  # (B, G): (R_k s) . u_ref
    a = np.abs(score) if inversion else score
    k = np.argmax(a, axis=1)
    srt = np.sort(a, axis=1)
    mk = srt[:, -1] - srt[:, -2] if a.shape[1] > 1 else np.full(len(s), np.inf)
    sc = score[np.arange(len(s)), k]
    sigma = np.where(inversion & (sc < 0), -1.0, 1.0)
    q1 = bodies.qmul(quats[k], q)                                       # (B, 4)
    sj = np.abs(bodies.qmul(q1[:, None, :], quats[None, :, :])[..., 0])  # (B, G)
    j = np.argmax(sj, axis=1)
    srt = np.sort(sj, axis=1)
    mj = srt[:, -1] - srt[:, -2] if sj.shape[1] > 1 else np.full(len(s), np.inf)
    return k, sigma, j, mk, mj


def canonical(s, q, group):
    """Canonical configuration (s', q') as FP64 numpy arrays."""
    quats, _ = group
    k, sigma, j, _, _ = choose(s, q, group)
    s = np.asarray(s, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1, 4)
    s2 = sigma[:, None] * np.einsum("bij,bj->bi", bodies.qmatrix(quats[k]), s)
    q2 = bodies.qmul(bodies.qmul(quats[k], q), quats[j])
    return s2, q2


def canonical_torch(s, q, group):
    """The same map on torch tensors, differentiable in s and q: the choice
    is made on the detached values, and the map for that choice is linear."""
    quats, _ = group
    k, sigma, j, _, _ = choose(s.detach().numpy(), q.detach().numpy(), group)
    Qk = torch.as_tensor(quats[k], dtype=s.dtype)
    Qj = torch.as_tensor(quats[j], dtype=s.dtype)
    Rk = torch.as_tensor(bodies.qmatrix(quats[k]), dtype=s.dtype)
    sg = torch.as_tensor(sigma, dtype=s.dtype)
    s2 = sg.unsqueeze(-1) * torch.einsum("bij,bj->bi", Rk, s.reshape(-1, 3))
    q2 = _tqmul(_tqmul(Qk, q.reshape(-1, 4)), Qj)
    return s2.reshape(s.shape), q2.reshape(q.shape)


def _tqmul(a, b):
    aw, ax, ay, az = a.unbind(-1)
    bw, bx, by, bz = b.unbind(-1)
    return torch.stack([aw * bw - ax * bx - ay * by - az * bz,
                        aw * bx + ax * bw + ay * bz - az * by,
                        aw * by - ax * bz + ay * bw + az * bx,
                        aw * bz + ax * by - ay * bx + az * bw], dim=-1)


def apply(s, q, group, k, sigma=1.0, j=0):
    """The configuration (sigma R_k s, Q_k (x) q (x) Q_j) for one group choice
    (the map whose invariance the tests check)."""
    quats, _ = group
    s = np.asarray(s, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    s2 = sigma * bodies.qrotate(np.broadcast_to(quats[k], q.shape), s)
    q2 = bodies.qmul(bodies.qmul(np.broadcast_to(quats[k], q.shape), q),
                     np.broadcast_to(quats[j], q.shape))
    return s2, q2
