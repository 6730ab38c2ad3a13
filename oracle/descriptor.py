"""Oracle: the paper's six-number description of a cube pair (SI Sec. 1).

TEST INFRASTRUCTURE (see the package docstring).  PyTorch CPU, FP64.

A cube pair is given by cube 2's centre s and orientation q in the body frame
of cube 1 (14 numbers reduced to 7 by putting cube 1 at the origin with the
identity orientation).  SI Sec. 1 reduces it to six numbers, in these steps:

1. Frame of cube 1.  Of the 24 ways to take cube 1's face normals as the
   axes (i, j, k), the one that puts cube 2's centre in the non-negative
   octant; cube 1's face towards cube 2 is always (1, 0, 0), so x is the
   largest coordinate.  If then p_z > p_y, the pair is reflected across the
   y = z plane (a reflected cube pair has the same energy).  Together this is
   the signed axis permutation M (proper or not) with p = M s and
   p_x >= p_y >= p_z >= 0; ties go to the first M in a fixed order.
2. Cube 2's orientation in that frame, R' = M R(q) M^T (for an improper M
   this is the reflected cube, again a proper rotation of the template).
3. w: of cube 2's six face normals +-R' e_a, the one opposite its face
   closest to cube 1's centre, i.e. the one with the largest w . p.
4. alpha_1 = arccos(w_x) and alpha_2 = atan2(w_z, w_y): the rotation by
   -alpha_2 about x and then by -alpha_1 about z turns w onto (1, 0, 0).
5. alpha_3: after those two rotations cube 2's other face normals lie in the
   y-z plane; alpha_3 is the rotation about x that makes cube 2 coincide with
   cube 1, taken in [0, pi/2) (a quarter turn about x maps the cube onto
   itself): alpha_3 = atan2(u_z, u_y) mod pi/2 for u the rotated image of one
   of the two other face normals (any of the four gives the same value).

The six numbers are (p_x, p_y, p_z, alpha_1, alpha_2, alpha_3).  They are
differentiable in (s, q) except where a choice switches (ties in steps 1 and
3, the wrap of alpha_3) and at alpha_1 = 0, where alpha_2 is undefined (the
interacting faces are parallel): there alpha_2 and alpha_3 are coordinates of
a singular chart, and only alpha_2 + alpha_3 is fixed by the configuration.

margins() reports how far a configuration is from every such place, so that
comparisons in two precisions can leave the ambiguous ones out.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import torch

DT = torch.float64


def _signed_permutations() -> np.ndarray:
    """The 48 signed axis permutations (rows: new axes), in a fixed order."""
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            M = np.zeros((3, 3))
            for r in range(3):
                M[r, perm[r]] = signs[r]
            out.append(M)
    return np.array(out)


M48 = _signed_permutations()


def frame_choice(s) -> np.ndarray:
    """Index into M48 of the first M with M s sorted and non-negative."""
    s = np.asarray(s, dtype=np.float64).reshape(-1, 3)
    p = np.einsum("kij,bj->bki", M48, s)
    ok = (p[..., 0] >= p[..., 1]) & (p[..., 1] >= p[..., 2]) & (p[..., 2] >= 0.0)
    assert ok.any(axis=1).all()
    return np.argmax(ok, axis=1)


def qmatrix(q):
    """R(q) of unit quaternions (s, i, j, k), torch, (..., 3, 3)."""
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def _rot_x(a):
    c, s = torch.cos(a), torch.sin(a)
    o, z = torch.ones_like(a), torch.zeros_like(a)
    return torch.stack([torch.stack([o, z, z], -1), torch.stack([z, c, -s], -1),
                        torch.stack([z, s, c], -1)], -2)


def _rot_z(a):
    c, s = torch.cos(a), torch.sin(a)
    o, z = torch.ones_like(a), torch.zeros_like(a)
    return torch.stack([torch.stack([c, -s, z], -1), torch.stack([s, c, z], -1),
                        torch.stack([z, z, o], -1)], -2)


def _steps(s, q):
    """Steps 1-3: p, R', the face index a and its sign (choices detached)."""
    s = s.reshape(-1, 3)
    q = q.reshape(-1, 4)
    q = q / torch.sqrt((q * q).sum(-1, keepdim=True))  # the description is of unit quaternions
    k = frame_choice(s.detach().numpy())
    M = torch.as_tensor(M48[k], dtype=s.dtype)
    p = torch.einsum("bij,bj->bi", M, s)
    Rp = M @ qmatrix(q) @ M.transpose(1, 2)
    proj = torch.einsum("bia,bi->ba", Rp, p).detach()  # (R' e_a) . p
    a = torch.argmax(proj.abs(), dim=1)
    sigma = torch.sign(proj[torch.arange(len(a)), a])
    return p, Rp, a, sigma


def describe(s, q):
    """(B, 6) = (p_x, p_y, p_z, alpha_1, alpha_2, alpha_3) of cube 2 at s
    with orientation q in cube 1's frame; torch FP64, differentiable in s and
    q with the discrete choices held."""
    p, Rp, a, sigma = _steps(s, q)
    idx = torch.arange(len(a))
    w = sigma.unsqueeze(-1) * Rp[idx, :, a]
    a1 = torch.arccos(torch.clamp(w[:, 0], -1.0, 1.0))
    a2 = torch.atan2(w[:, 2], w[:, 1])
    align = _rot_z(-a1) @ _rot_x(-a2)
    b = (a + 1) % 3
    u = torch.einsum("bij,bj->bi", align, Rp[idx, :, b])
    a3 = torch.remainder(torch.atan2(u[:, 2], u[:, 1]), 0.5 * math.pi)
    return torch.cat([p, a1[:, None], a2[:, None], a3[:, None]], -1)


def describe_np(s, q) -> np.ndarray:
    with torch.no_grad():
        return describe(torch.as_tensor(np.asarray(s, dtype=np.float64)),
                        torch.as_tensor(np.asarray(q, dtype=np.float64))).numpy()


def reconstruct(d) -> tuple[np.ndarray, np.ndarray]:
    """A configuration (s, R) with the six numbers d: s = p and
    R = Rx(alpha_2) Rz(alpha_1) Rx(alpha_3) (the inverse of steps 4 and 5)."""
    d = torch.as_tensor(np.asarray(d, dtype=np.float64)).reshape(-1, 6)
    R = _rot_x(d[:, 4]) @ _rot_z(d[:, 3]) @ _rot_x(d[:, 5])
    return d[:, :3].numpy(), R.numpy()


def angle_gap(a, b, period: float) -> np.ndarray:
    """Distance of two angles on a circle of the given period."""
    d = np.remainder(np.asarray(a) - np.asarray(b), period)
    return np.minimum(d, period - d)


def margins(s, q) -> np.ndarray:
    """Per configuration, the smallest distance (in coordinate or radian
    units of the choice concerned) to a switch of the description: a tie of
    the frame's sort (p_x - p_y, p_y - p_z, p_z), a tie of the face choice
    (gap of the two largest |(R' e_a) . p| / |p|), the wrap of alpha_3, and
    sin(alpha_1) (alpha_2 undefined at 0)."""
    with torch.no_grad():
        st = torch.as_tensor(np.asarray(s, dtype=np.float64)).reshape(-1, 3)
        qt = torch.as_tensor(np.asarray(q, dtype=np.float64)).reshape(-1, 4)
        p, Rp, a, sigma = _steps(st, qt)
        d = describe(st, qt).numpy()
    p = p.numpy()
    m_frame = np.minimum(np.minimum(p[:, 0] - p[:, 1], p[:, 1] - p[:, 2]), p[:, 2])
    proj = np.sort(np.abs(np.einsum("bia,bi->ba", Rp.numpy(), p)), axis=1)
    m_face = (proj[:, 2] - proj[:, 1]) / np.linalg.norm(p, axis=1)
    m_wrap = angle_gap(d[:, 5], 0.0, 0.5 * math.pi)
    m_a1 = np.sin(d[:, 3])
    return np.minimum(np.minimum(m_frame, m_face), np.minimum(m_wrap, m_a1))
