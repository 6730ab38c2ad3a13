"""Pins of the oracle's six-number cube-pair description (oracle/descriptor.py,
paper SI Sec. 1) against facts the paper and geometry fix:

- worked configurations with hand-derived numbers: faces aligned along x
  (all angles 0), cube 2 turned about x (alpha_3 = the turn), about z
  (alpha_1 = the turn), about y (alpha_1 = the turn, alpha_2 = -pi/2); a
  centre with p_z > p_y reflected across y = z; the frame from any octant;
- completeness: the bead-sum energy of every configuration equals that of the
  configuration rebuilt from its six numbers (a wrong frame, face, sign or
  angle anywhere changes the energy);
- invariance: all 48 x 24 descriptions of the same pair (cube 1's symmetry
  operations, proper and improper, applied to the whole pair, and cube 2
  relabelled by its 24 rotations) give the same six numbers;
- the derivatives of the six numbers under small rotations of cube 2 (what
  torques are made of) equal central differences;
- a network on the six numbers: forces and torques are central differences
  of its energy, and Newton 3 and angular-momentum balance hold.
No GPU."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import bodies, descriptor, nn
from paper_2402_12199_gb300 import inputs

CUBE = bodies.cube_template()


def q_axis(axis, angle):
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    return np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * a])


def desc(s, q):
    return descriptor.describe_np(np.asarray(s, float)[None], np.asarray(q, float)[None])[0]


def close_angle(a, b, period=2 * math.pi, tol=1e-12):
    return descriptor.angle_gap(a, b, period) < tol


def test_worked_configurations():
    ident = [1.0, 0, 0, 0]
    np.testing.assert_allclose(desc([6.0, 0, 0], ident), [6, 0, 0, 0, 0, 0], atol=1e-15)
    # the frame from the -z face: centre along -z is the same aligned pair
    np.testing.assert_allclose(desc([0, 0, -6.0], ident), [6, 0, 0, 0, 0, 0], atol=1e-15)
    # turned about x by 0.3: faces still aligned, the roll is alpha_3
    d = desc([6.0, 0, 0], q_axis([1, 0, 0], 0.3))
    np.testing.assert_allclose(d[:4], [6, 0, 0, 0], atol=1e-15)
    assert abs(d[5] - 0.3) < 1e-14
    # turned about x by 1.9 (beyond a quarter turn): alpha_3 = 1.9 - pi/2
    d = desc([6.0, 0, 0], q_axis([1, 0, 0], 1.9))
    assert abs(d[5] - (1.9 - math.pi / 2)) < 1e-14
    # turned about z by 0.3: w = (cos .3, sin .3, 0): alpha_1 = 0.3, alpha_2 = 0
    d = desc([6.0, 0, 0], q_axis([0, 0, 1], 0.3))
    np.testing.assert_allclose(d, [6, 0, 0, 0.3, 0, 0], atol=1e-14)
    # turned about y by 0.3: w = (cos .3, 0, -sin .3): alpha_1 = 0.3, alpha_2 = -pi/2,
    # and the rest of the cube is square to the axes after the two rotations
    d = desc([6.0, 0, 0], q_axis([0, 1, 0], 0.3))
    np.testing.assert_allclose(d[:5], [6, 0, 0, 0.3, -math.pi / 2], atol=1e-14)
    assert close_angle(d[5], 0.0, math.pi / 2, 1e-12)


def test_frame_sorts_and_reflects():
    rng = np.random.default_rng(3)
    q = inputs.random_quaternions(1, rng)[0].astype(np.float64)
    q /= np.linalg.norm(q)
    # p_z > p_y: the frame reflects across y = z
    d1 = desc([6.0, 1.0, 2.0], q)
    np.testing.assert_allclose(d1[:3], [6.0, 2.0, 1.0], atol=1e-15)
    # every octant and axis order of the same centre lands on the same p
    for sx in (1, -1):
        for sz in (1, -1):
            for perm in ((0, 1, 2), (2, 0, 1), (1, 2, 0)):
                s = np.array([6.0 * sx, 1.0, 2.0 * sz])[list(perm)]
                np.testing.assert_allclose(desc(s, q)[:3], [6.0, 2.0, 1.0], atol=1e-15)


def _configs(n, seed, rho=(5.2, 9.0), margin=1e-3):
    c = inputs.pair_configs(4 * n, seed, *rho).astype(np.float64)
    s, q = c[:, :3], c[:, 3:] / np.linalg.norm(c[:, 3:], axis=1, keepdims=True)
    ok = descriptor.margins(s, q) > margin
    return s[ok][:n], q[ok][:n]


def _mat_to_quat(R):
    """Unit quaternion of a rotation matrix (largest-component branch)."""
    t = np.trace(R)
    if t > 0:
        w = math.sqrt(1 + t) / 2
        return np.array([w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w),
                         (R[1, 0] - R[0, 1]) / (4 * w)])
    i = int(np.argmax(np.diag(R)))
    j, k = (i + 1) % 3, (i + 2) % 3
    r = math.sqrt(1 + R[i, i] - R[j, j] - R[k, k])
    q = np.zeros(4)
    q[0] = (R[k, j] - R[j, k]) / (2 * r)
    q[1 + i] = r / 2
    q[1 + j] = (R[j, i] + R[i, j]) / (2 * r)
    q[1 + k] = (R[k, i] + R[i, k]) / (2 * r)
    return q


def test_six_numbers_fix_the_bead_energy():
    s, q = _configs(40, 11, rho=(4.8, 7.0))
    d = descriptor.describe_np(s, q)
    p_rec, R_rec = descriptor.reconstruct(d)
    box = np.array([100.0] * 3)
    zero = np.zeros(3)
    ident = np.array([1.0, 0, 0, 0])
    n_nonzero = 0
    for b in range(len(s)):
        E0 = oracle.bead_pair(zero, ident, s[b], q[b], box, CUBE)["E"]
        E1 = oracle.bead_pair(zero, ident, p_rec[b], _mat_to_quat(R_rec[b]), box, CUBE)["E"]
        n_nonzero += E0 != 0.0
        assert abs(E1 - E0) <= 1e-11 * max(1.0, abs(E0)), (b, E0, E1)
    assert n_nonzero >= 30
    # ranges: sorted non-negative centre, alpha_1 in [0, pi), alpha_3 in [0, pi/2)
    assert np.all(d[:, 0] >= d[:, 1]) and np.all(d[:, 1] >= d[:, 2]) and np.all(d[:, 2] >= 0)
    assert np.all((d[:, 3] >= 0) & (d[:, 3] < math.pi))
    assert np.all((d[:, 5] >= 0) & (d[:, 5] < math.pi / 2))


def test_description_is_invariant_under_the_cube_symmetries():
    from oracle import symmetry

    group, inversion = symmetry.point_group(CUBE)
    assert len(group) == 24 and inversion
    s, q = _configs(12, 12)
    d0 = descriptor.describe_np(s, q)
    for k in range(24):
        Rk = bodies.qmatrix(group[k])
        for sg in (1.0, -1.0):  # the improper operations: rotation times inversion
            s2 = sg * s @ Rk.T
            q1 = bodies.qmul(np.broadcast_to(group[k], q.shape), q)
            for j in range(0, 24, 5):
                q2 = bodies.qmul(q1, np.broadcast_to(group[j], q.shape))
                d = descriptor.describe_np(s2, q2)
                np.testing.assert_allclose(d[:, :5], d0[:, :5], atol=1e-11)
                assert np.all(close_angle(d[:, 5], d0[:, 5], math.pi / 2, 1e-11))


def test_angle_derivatives_under_rotations_of_cube_2():
    """d alpha / d theta (rotation of cube 2 about the frame's axes) by autograd
    equals central differences; the centre does not depend on the rotation."""
    s, q = _configs(20, 13, margin=2e-2)
    h = 1e-6
    st = torch.as_tensor(s)
    qt = torch.as_tensor(q)
    th = torch.zeros(len(s), 3, dtype=torch.float64, requires_grad=True)
    half = torch.cat([torch.zeros(len(s), 1, dtype=torch.float64), 0.5 * th], -1)
    d = descriptor.describe(st, qt + nn._qmul(half, qt))
    for c in range(3, 6):
        (g,) = torch.autograd.grad(d[:, c].sum(), [th], retain_graph=True)
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1.0
            qp = bodies.qmul(np.broadcast_to(q_axis(e, h), q.shape), q)
            qm = bodies.qmul(np.broadcast_to(q_axis(e, -h), q.shape), q)
            fd = (descriptor.describe_np(s, qp)[:, c] - descriptor.describe_np(s, qm)[:, c]) / (2 * h)
            np.testing.assert_allclose(g[:, k].numpy(), fd, rtol=1e-6, atol=1e-6)


def _paper6_net(seed=4, width=16):
    flat = inputs.mlp_params(width, 3, seed).astype(np.float64)
    flat[:10] = [6.5, 3.0, 1.5, 1.5, 0.0, 0.8, 0, 0, 0, 0]       # mu
    flat[10:20] = [0.6, 0.6, 0.8, 0.7, 0.5, 1.8, 0, 0, 0, 0]      # inv_sd
    return flat, nn.unpack(flat, width, 3, desc="paper6")


def test_network_on_six_numbers_forces_are_energy_gradients():
    flat, p = _paper6_net()
    s, q = _configs(15, 14, margin=2e-2)
    qi = inputs.random_quaternions(len(s), np.random.default_rng(5)).astype(np.float64)
    qi /= np.linalg.norm(qi, axis=1, keepdims=True)
    # space-frame pair: body i at the origin with orientation qi
    R_ij = bodies.qrotate(qi, s)
    qj = bodies.qmul(qi, q)
    r = nn.pair_forces(p, R_ij, qi, qj)
    assert np.allclose(r["F_i"] + r["F_j"], 0.0)
    np.testing.assert_allclose(r["tau_i"] + r["tau_j"] + np.cross(R_ij, r["F_j"]), 0.0, atol=1e-11)

    def energy(R, a, b):
        with torch.no_grad():
            return nn.config_energy(p, nn._to_body(torch.as_tensor(a), torch.as_tensor(R)),
                                    nn._qmul(nn._qconj(torch.as_tensor(a)),
                                             torch.as_tensor(b))).numpy()

    h = 1e-5
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (energy(R_ij + e, qi, qj) - energy(R_ij - e, qi, qj)) / (2 * h)
        np.testing.assert_allclose(-r["F_j"][:, k], fd, rtol=1e-6, atol=1e-7)
        rp = np.broadcast_to(q_axis(np.eye(3)[k], h), qj.shape)
        rm = np.broadcast_to(q_axis(np.eye(3)[k], -h), qj.shape)
        fd_j = (energy(R_ij, qi, bodies.qmul(rp, qj)) - energy(R_ij, qi, bodies.qmul(rm, qj))) / (2 * h)
        np.testing.assert_allclose(-r["tau_j"][:, k], fd_j, rtol=1e-6, atol=1e-7)
        fd_i = (energy(R_ij, bodies.qmul(rp, qi), qj) - energy(R_ij, bodies.qmul(rm, qi), qj)) / (2 * h)
        np.testing.assert_allclose(-r["tau_i"][:, k], fd_i, rtol=1e-6, atol=1e-7)
