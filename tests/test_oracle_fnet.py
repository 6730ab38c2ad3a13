"""Pins of the oracle's per-component cylinder networks (oracle/fnet.py):

  * the four-number description of simple pair configurations (side by side,
    stacked, T-shaped, crossed, cylinder 2 below cylinder 1) has closed forms;
  * it is unchanged by the symmetries it assumes: turning either cylinder
    about its own axis, turning either cylinder end over end;
  * the frame is orthonormal and right-handed with z along cylinder 1's axis
    and cylinder 2's centre in its x-z half plane;
  * the networks' five outputs map to forces and torques that obey Newton's
    third law and angular-momentum balance, give no torque on cylinder 1
    about its axis, and map back to the same five numbers;
  * a width-1 network is the hand-written scalar composition;
  * the regression loss gradient (plain and force-scale weighted) equals
    central differences.
No GPU.
"""
import math

import numpy as np
import pytest
import torch

from oracle import bodies, fnet

ID = np.array([1.0, 0, 0, 0])


def qaxis(axis, ang):
    return bodies.qexp(np.asarray(axis, dtype=np.float64) * ang)


def test_descriptor_closed_forms():
    # side by side, parallel
    _, _, _, d = fnet.frame([3.0, 0, 0], ID)
    np.testing.assert_allclose(d[0], [3.0, 0, 0, 0], atol=1e-15)
    # stacked along the axis (p_r = 0)
    _, _, _, d = fnet.frame([0, 0, 6.5], ID)
    np.testing.assert_allclose(d[0], [0, 6.5, 0, 0], atol=1e-15)
    # near T-shape: centre along body y, so x_hat = body y and y_hat = -body x;
    # cylinder 2 turned by pi/2 - 0.1 about body x: axis (0, -cos 0.1, sin 0.1)
    # in the body frame = (-cos 0.1, 0, sin 0.1) in the descriptor frame
    _, _, _, d = fnet.frame([0, 4.0, 0], qaxis([1, 0, 0], math.pi / 2 - 0.1))
    np.testing.assert_allclose(d[0], [4.0, 0, math.pi / 2 - 0.1, math.pi], atol=1e-12)
    # near cross: centre along body x; the same turn gives (0, -cos 0.1, sin 0.1)
    _, _, _, d = fnet.frame([5.0, 0, 0], qaxis([1, 0, 0], math.pi / 2 - 0.1))
    np.testing.assert_allclose(d[0], [5.0, 0, math.pi / 2 - 0.1, -math.pi / 2], atol=1e-12)
    # turned past the perpendicular: the axis is taken end over end (u_z >= 0)
    _, _, _, d = fnet.frame([5.0, 0, 0], qaxis([1, 0, 0], math.pi / 2 + 0.1))
    np.testing.assert_allclose(d[0], [5.0, 0, math.pi / 2 - 0.1, math.pi / 2], atol=1e-12)
    # below cylinder 1: p_z is |s_z|, and z_hat points down
    xh, yh, zh, d = fnet.frame([1.0, 2.0, -3.0], ID)
    np.testing.assert_allclose(d[0, :2], [math.sqrt(5.0), 3.0], atol=1e-14)
    np.testing.assert_allclose(zh[0], [0, 0, -1], atol=1e-15)
    # a tilt of 30 degrees of cylinder 2 towards cylinder 1's centre direction
    _, _, _, d = fnet.frame([4.0, 0, 1.0], qaxis([0, 1, 0], math.pi / 6))
    np.testing.assert_allclose(d[0], [4.0, 1.0, math.pi / 6, 0], atol=1e-12)


def _random_configs(n, seed):
    rng = np.random.default_rng(seed)
    s = rng.standard_normal((n, 3)) * 4
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return s, q, rng


def test_descriptor_symmetries():
    s, q, rng = _random_configs(50, 1)
    _, _, _, d0 = fnet.frame(s, q)
    n = len(s)
    for _ in range(4):
        a = rng.uniform(0, 2 * math.pi)
        # cylinder 1 turned by a about its own axis (body i's z): in its frame
        # the other body is turned by -a
        qa = np.broadcast_to(qaxis([0, 0, 1], -a), (n, 4))
        _, _, _, d = fnet.frame(bodies.qrotate(qa, s), bodies.qmul(qa, q))
        np.testing.assert_allclose(d, d0, atol=1e-12)
        # cylinder 2 turned about its own axis
        _, _, _, d = fnet.frame(s, bodies.qmul(q, np.broadcast_to(qaxis([0, 0, 1], a), (n, 4))))
        np.testing.assert_allclose(d, d0, atol=1e-12)
    # cylinder 2 end over end; cylinder 1 end over end
    flip = np.broadcast_to(qaxis([1, 0, 0], math.pi), (n, 4))
    _, _, _, d = fnet.frame(s, bodies.qmul(q, flip))
    np.testing.assert_allclose(d, d0, atol=1e-12)
    _, _, _, d = fnet.frame(bodies.qrotate(flip, s), bodies.qmul(flip, q))
    np.testing.assert_allclose(d, d0, atol=1e-12)


def test_frame_is_orthonormal_and_places_cylinder_2():
    s, q, _ = _random_configs(40, 2)
    xh, yh, zh, d = fnet.frame(s, q)
    M = np.stack([xh, yh, zh], 2)
    np.testing.assert_allclose(np.einsum("nai,naj->nij", M, M), np.broadcast_to(np.eye(3), (40, 3, 3)),
                               atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(M), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.abs(zh[:, 2]), 1.0)
    np.testing.assert_allclose((s * yh).sum(1), 0.0, atol=1e-13)
    np.testing.assert_allclose((s * xh).sum(1), d[:, 0], atol=1e-13)
    np.testing.assert_allclose((s * zh).sum(1), d[:, 1], atol=1e-13)
    assert np.all(d[:, 2] <= math.pi / 2 + 1e-15) and np.all(np.abs(d[:, 3]) <= math.pi)


def _rand_flat(width, depth, seed):
    rng = np.random.default_rng(seed)
    n = fnet.net_size(width, depth)
    flat = rng.standard_normal(5 * n) * 0.4
    for c in range(5):
        o = c * n
        flat[o:o + 4] = [4.0, 2.0, 0.8, 0.0]        # mu
        flat[o + 4:o + 8] = [0.3, 0.3, 1.2, 0.5]    # inv_sd
        flat[o + n - 2] = 1.5                       # y_scale
        flat[o + n - 1] = 0.1 * c                   # y_shift
    return flat


def test_outputs_map_to_balanced_forces_and_back():
    width, depth = 8, 3
    nets = fnet.unpack(torch.as_tensor(_rand_flat(width, depth, 3)), width, depth)
    s, q, _ = _random_configs(30, 4)
    Fj, ti, tj, y = fnet.predict(nets, s, q)
    _, _, zh, _ = fnet.frame(s, q)
    np.testing.assert_allclose((ti * zh).sum(1), 0.0, atol=1e-14)     # no tau_3
    np.testing.assert_allclose(ti + tj + np.cross(s, Fj), 0.0, atol=1e-12)
    _, t = fnet.targets(s, q, Fj, ti)
    np.testing.assert_allclose(t, y, atol=1e-12)


def test_width_one_network_closed_form():
    width, depth = 1, 2
    flat = _rand_flat(width, depth, 5)
    nets = fnet.unpack(torch.as_tensor(flat), width, depth)
    d = np.array([[3.1, 0.7, 0.4, -1.2]])
    sig = lambda z: 1.0 / (1.0 + math.exp(-z))
    n = fnet.net_size(width, depth)
    for c in range(5):
        p = flat[c * n:(c + 1) * n]
        mu, isd = p[0:4], p[4:8]
        w1, b1, w2, b2, wo, bo, ys, yt = p[8:12], p[12], p[13], p[14], p[15], p[16], p[17], p[18]
        x = (d[0] - mu) * isd
        z1 = float(w1 @ x + b1)
        h1 = z1 * sig(z1)
        z2 = w2 * h1 + b2
        h2 = z2 * sig(z2)
        expect = ys * (wo * h2 + bo) + yt
        got = float(fnet.net_forward(nets[c], torch.as_tensor(d))[0])
        assert got == pytest.approx(expect, rel=1e-14)


@pytest.mark.parametrize("f_scale", [None, 1.5])
def test_regression_gradient_matches_central_differences(f_scale):
    width, depth = 6, 2
    flat = _rand_flat(width, depth, 6)
    rng = np.random.default_rng(7)
    d = np.column_stack([rng.uniform(2, 8, 20), rng.uniform(0, 5, 20), rng.uniform(0, 1.5, 20),
                         rng.uniform(-3, 3, 20)])
    t = rng.standard_normal((20, 5))
    L, g = fnet.loss_and_grad(flat, width, depth, d, t, f_scale=f_scale)
    n = fnet.net_size(width, depth)
    h = 1e-6
    for k in rng.choice(len(flat), 40, replace=False):
        e = np.zeros_like(flat)
        e[k] = h
        fd = (fnet.loss_and_grad(flat + e, width, depth, d, t, f_scale=f_scale)[0]
              - fnet.loss_and_grad(flat - e, width, depth, d, t, f_scale=f_scale)[0]) / (2 * h)
        if k % n < 8 or k % n >= n - 2:
            assert g[k] == 0.0  # held fixed
        else:
            assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9)
