"""Oracle: per-component force/torque networks for cylinders (numpy / PyTorch
CPU, FP64).

TEST INFRASTRUCTURE (see the package docstring).

Paper (Methods; SI Sec. 2): for cylinders, five separate networks predict the
force components f_1, f_2, f_3 and the torque components tau_1, tau_2
directly (tau_3, about the cylinder's own axis, is not needed), from a pair
description of four numbers that uses the cylinders' axial symmetry:

  * a frame at cylinder 1's centre with z along cylinder 1's axis, the
    direction of z chosen so that cylinder 2's centre has p_z >= 0;
  * x chosen so that p_y = 0 and p_x > 0: (p_r, p_z) place cylinder 2;
  * cylinder 2's axis, a unit vector u in this frame, in spherical
    angles: theta = arccos(u_z), phi = atan2(u_y, u_x).

Readings (the paper is silent): the cylinder's axis is its body z axis;
cylinder 2's axis direction is taken with u_z >= 0 (a cylinder is unchanged
by turning it end over end; for u_z = 0 the first non-zero of u_x, u_y is made
positive); for p_r = 0 the frame's x is the body x axis (any choice is
equivalent by the axial symmetry).  The networks' outputs are the force on
cylinder 2 and the torque on cylinder 1 in this frame; the other body's force
is the opposite and its torque follows from angular-momentum balance,
tau_2 = -tau_1 - R x F_2 (R = p_2 - p_1).

Each network: 4 normalised inputs (x - mu) * inv_sd, D SiLU layers of width
W, a scalar output y = y_scale (w_o . h_D + b_o) + y_shift.  Flat layout of
one network: mu (4), inv_sd (4), W_1 [W][4], b_1, {W_l [W][W], b_l} for
l = 2..D, w_o (W), b_o, y_scale, y_shift; the five networks (f_1, f_2, f_3,
tau_1, tau_2) follow each other.  Training: regression of the five
components, L = mean_b sum_c (y_c - t_c)^2 (the paper names no loss).
"""
from __future__ import annotations

import numpy as np
import torch

from . import bodies

N_IN = 4
N_NETS = 5


def net_size(width: int, depth: int) -> int:
    return 8 + width * N_IN + width + (depth - 1) * (width * width + width) + width + 3


def unpack(flat, width: int, depth: int):
    """List of five dicts of tensors (views into `flat`, which may require grad)."""
    flat = torch.as_tensor(flat)
    n = net_size(width, depth)
    nets = []
    for c in range(N_NETS):
        o = c * n
        p = {}

        def take(k):
            nonlocal o
            t = flat[o:o + k]
            o += k
            return t

        p["mu"] = take(4)
        p["inv_sd"] = take(4)
        p["W"] = [take(width * N_IN).reshape(width, N_IN)]
        p["b"] = [take(width)]
        for _ in range(depth - 1):
            p["W"].append(take(width * width).reshape(width, width))
            p["b"].append(take(width))
        p["wo"] = take(width)
        p["bo"] = take(1)[0]
        p["y_scale"] = take(1)[0]
        p["y_shift"] = take(1)[0]
        nets.append(p)
    return nets


def frame(s, q_rel):
    """Descriptor frame and the four numbers for a batch, in the frame of
    cylinder 1 (body i): s = R(q_i)^T R_ij, q_rel = q_i^* q_j.
    Returns x_hat, y_hat, z_hat (n x 3 each) and d = (p_r, p_z, theta, phi)."""
    s = np.atleast_2d(np.asarray(s, dtype=np.float64))
    q_rel = np.atleast_2d(np.asarray(q_rel, dtype=np.float64))
    n = len(s)
    ez = np.array([0.0, 0.0, 1.0])
    pz = s[:, 2]
    sz = np.where(pz < 0, -1.0, 1.0)
    z_hat = sz[:, None] * ez[None, :]
    r = s - pz[:, None] * ez[None, :]
    p_r = np.linalg.norm(r, axis=1)
    x_hat = np.where(p_r[:, None] > 0, r / np.where(p_r > 0, p_r, 1.0)[:, None],
                     np.broadcast_to([1.0, 0.0, 0.0], (n, 3)))
    y_hat = np.cross(z_hat, x_hat)
    a2 = bodies.qrotate(q_rel, np.broadcast_to(ez, (n, 3)))
    u = np.stack([(a2 * x_hat).sum(1), (a2 * y_hat).sum(1), (a2 * z_hat).sum(1)], 1)
    flip = (u[:, 2] < 0) | ((u[:, 2] == 0) & ((u[:, 0] < 0) | ((u[:, 0] == 0) & (u[:, 1] < 0))))
    u = np.where(flip[:, None], -u, u)
    theta = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    phi = np.arctan2(u[:, 1], u[:, 0])
    return x_hat, y_hat, z_hat, np.stack([p_r, np.abs(pz), theta, phi], 1)


def net_forward(p, d):
    """One network on descriptors d (n x 4, tensor): the scalar output."""
    h = (d - p["mu"]) * p["inv_sd"]
    for W, b in zip(p["W"], p["b"]):
        z = h @ W.T + b
        h = z * torch.sigmoid(z)
    return p["y_scale"] * (h @ p["wo"] + p["bo"]) + p["y_shift"]


def predict(nets, s, q_rel):
    """Forces and torques of the per-component networks, in the frame of
    body i: (F_j, tau_i, tau_j) as n x 3 arrays, and the five raw outputs."""
    s = np.atleast_2d(np.asarray(s, dtype=np.float64))
    xh, yh, zh, d = frame(s, q_rel)
    dt = torch.as_tensor(d)
    with torch.no_grad():
        y = torch.stack([net_forward(p, dt) for p in nets], 1).numpy()
    Fj = y[:, 0:1] * xh + y[:, 1:2] * yh + y[:, 2:3] * zh
    ti = y[:, 3:4] * xh + y[:, 4:5] * yh
    tj = -ti - np.cross(s, Fj)
    return Fj, ti, tj, y


def targets(s, q_rel, F_j, tau_i, cap=None):
    """Training targets: the bead-sum force on body j and torque on body i
    (frame of body i) in the descriptor frame, (f_1, f_2, f_3, tau_1, tau_2),
    optionally clamped to [-cap, cap] (the paper caps the wide range of its
    force and torque training values, SI Sec. 6)."""
    xh, yh, zh, d = frame(s, q_rel)
    F_j = np.atleast_2d(F_j)
    tau_i = np.atleast_2d(tau_i)
    t = np.stack([(F_j * xh).sum(1), (F_j * yh).sum(1), (F_j * zh).sum(1),
                  (tau_i * xh).sum(1), (tau_i * yh).sum(1)], 1)
    if cap:
        t = np.clip(t, -cap, cap)
    return d, t


def loss_and_grad(flat, width, depth, d, t, f_scale=None):
    """L = mean_b w_b sum_c (y_c(d_b) - t_bc)^2 and dL/dflat (FP64 autograd),
    w_b = 1 / (1 + |t_b|^2 / f_scale^2) when f_scale is given, else 1; mu,
    inv_sd, y_scale and y_shift are held fixed (zero gradient)."""
    ft = torch.as_tensor(np.asarray(flat, dtype=np.float64)).clone().requires_grad_(True)
    nets = unpack(ft, width, depth)
    dt = torch.as_tensor(np.asarray(d, dtype=np.float64))
    tt = torch.as_tensor(np.asarray(t, dtype=np.float64))
    y = torch.stack([net_forward(p, dt) for p in nets], 1)
    w = 1.0 / (1.0 + (tt ** 2).sum(1) / f_scale ** 2) if f_scale else torch.ones(len(tt), dtype=tt.dtype)
    L = (w * ((y - tt) ** 2).sum(1)).mean()
    (g,) = torch.autograd.grad(L, [ft])
    g = g.numpy().copy()
    n = net_size(width, depth)
    for c in range(N_NETS):
        g[c * n:c * n + 8] = 0.0
        g[(c + 1) * n - 2:(c + 1) * n] = 0.0
    return float(L.detach()), g


def forces_fnet(nets, pos, quat, box, pairs):
    """Whole-system forces and torques (space frame) of the per-component
    networks over the listed pairs (i < j, i taken as cylinder 1)."""
    pos = np.asarray(pos, dtype=np.float64)
    quat = np.asarray(quat, dtype=np.float64)
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    N = len(pos)
    F = np.zeros((N, 3))
    T = np.zeros((N, 3))
    if len(pairs) == 0:
        return F, T
    i, j = pairs[:, 0], pairs[:, 1]
    R = bodies.min_image(pos[j] - pos[i], box)
    s = bodies.qrotate(bodies.qconj(quat[i]), R)
    qr = bodies.qmul(bodies.qconj(quat[i]), quat[j])
    Fj, ti, tj, _ = predict(nets, s, qr)
    Fj_s = bodies.qrotate(quat[i], Fj)
    ti_s = bodies.qrotate(quat[i], ti)
    tj_s = bodies.qrotate(quat[i], tj)
    np.add.at(F, j, Fj_s)
    np.add.at(F, i, -Fj_s)
    np.add.at(T, i, ti_s)
    np.add.at(T, j, tj_s)
    return F, T
