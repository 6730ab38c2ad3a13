"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed
form, an invariant, central finite differences, a structurally different
brute-force sum, or a special case that reduces to a textbook result.  No GPU.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import bodies, md, nn, sampler
from paper_2402_12199_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CUBE = bodies.cube_template()
CYL = bodies.cylinder_template()
RC = 2.5
NOBOX = np.zeros(3)
ID = np.array([1.0, 0, 0, 0])


def rand_q(rng):
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


def u_lj(r, eps=1.0, sig=1.0, rc=RC):
    return 4 * eps * ((sig / r) ** 12 - (sig / r) ** 6) - 4 * eps * ((sig / rc) ** 12 - (sig / rc) ** 6)


# ------------------------------------------------------------------ potential

def test_lj_special_points():
    """LJ minimum at r = 2^(1/6) sigma with depth -eps (before the shift), zero
    crossing at sigma, nothing at and beyond r_c (golden values)."""
    g = json.load(open(os.path.join(GOLD, "lj_points.json")))
    shift = g["shift_at_rc_2.5"]
    u, f = oracle.lj(2 ** (1 / 6))
    assert u == pytest.approx(-1.0 - shift, abs=1e-14)
    assert abs(f) < 1e-13
    u, _ = oracle.lj(1.0)
    assert u == pytest.approx(-shift, abs=1e-14)
    assert oracle.lj(2.5) == (0.0, 0.0)
    assert oracle.lj(3.0) == (0.0, 0.0)
    u, _ = oracle.lj(2.5 - 1e-12)
    assert abs(u) < 1e-12


def test_lj_force_is_minus_derivative():
    for r in [0.95, 1.0, 1.12, 1.5, 2.0, 2.4]:
        h = 1e-6
        fd = -(oracle.lj(r + h)[0] - oracle.lj(r - h)[0]) / (2 * h)
        assert oracle.lj(r)[1] * r == pytest.approx(fd, rel=1e-7, abs=1e-9)


# ------------------------------------------------------------------ bead sum

def test_one_bead_bodies_reduce_to_lj():
    """Single-bead bodies: the double sum is one LJ term, torques vanish."""
    one = np.zeros((1, 3))
    rng = np.random.default_rng(0)
    for r in [0.97, 1.1, 1.7, 2.3]:
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        res = oracle.bead_pair(np.zeros(3), rand_q(rng), r * d, rand_q(rng), NOBOX, one)
        fmag = 24 * (2 * r ** -13 - r ** -7)
        assert res["E"] == pytest.approx(u_lj(r), abs=1e-13)
        np.testing.assert_allclose(res["F_j"], fmag * d, atol=1e-12)
        np.testing.assert_allclose(res["tau_i"], 0, atol=1e-14)
        np.testing.assert_allclose(res["tau_j"], 0, atol=1e-14)


def lattice_face_sum(D):
    """Two aligned 5x5x5 cubes separated by D along x: the 15625-term double
    sum collapses to 729 offset classes with multiplicities (5-|dx|)(5-|dy|)(5-|dz|)."""
    E = 0.0
    Fx = 0.0
    for dx in range(-4, 5):
        for dy in range(-4, 5):
            for dz in range(-4, 5):
                m = (5 - abs(dx)) * (5 - abs(dy)) * (5 - abs(dz))
                x = D + dx
                r = math.sqrt(x * x + dy * dy + dz * dz)
                if r < RC:
                    E += m * u_lj(r)
                    Fx += m * 24 * (2 * r ** -14 - r ** -8) * x
    return E, Fx


@pytest.mark.parametrize("D", [5.9, 6.0, 6.3, 7.0, 7.4])
def test_face_to_face_cubes_lattice_sum(D):
    res = oracle.bead_pair(np.zeros(3), ID, np.array([D, 0, 0]), ID, NOBOX, CUBE)
    E, Fx = lattice_face_sum(D)
    assert res["E"] == pytest.approx(E, rel=1e-12, abs=1e-12)
    assert res["F_j"][0] == pytest.approx(Fx, rel=1e-11, abs=1e-12)
    np.testing.assert_allclose(res["F_j"][1:], 0, atol=1e-11)


def numpy_bead_sum(p_i, q_i, p_j, q_j, tmpl):
    """Vectorised all-pairs sum written independently of the C oracle."""
    a = bodies.qrotate(np.broadcast_to(q_i, (len(tmpl), 4)), tmpl)
    bl = bodies.qrotate(np.broadcast_to(q_j, (len(tmpl), 4)), tmpl)
    b = bl + (np.asarray(p_j) - np.asarray(p_i))
    r = b[None, :, :] - a[:, None, :]
    r2 = (r ** 2).sum(-1)
    m = r2 < RC ** 2
    rr = np.sqrt(np.where(m, r2, 1.0))
    u = np.where(m, u_lj(rr), 0.0)
    fr = np.where(m, 24 * (2 * rr ** -14 - rr ** -8), 0.0)
    f = fr[..., None] * r
    fl = f.sum(0)
    fk = f.sum(1)
    return {"E": u.sum(), "F_j": fl.sum(0), "tau_j": np.cross(bl, fl).sum(0),
            "tau_i": np.cross(a, -fk).sum(0)}


@pytest.mark.parametrize("shape", ["cube", "cylinder"])
def test_bead_sum_matches_independent_bruteforce(shape):
    tmpl = CUBE if shape == "cube" else CYL
    rng = np.random.default_rng(1 if shape == "cube" else 2)
    n_checked = 0
    for _ in range(6):
        q_i, q_j = rand_q(rng), rand_q(rng)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        rho = sampler.contact_distance(d, bodies.qmul(bodies.qconj(q_i), q_j), tmpl, 12.0)
        p_i = rng.uniform(0, 5, 3)
        p_j = p_i + bodies.qrotate(q_i, (rho + rng.uniform(0.05, 2.0)) * d)
        ref = numpy_bead_sum(p_i, q_i, p_j, q_j, tmpl)
        res = oracle.bead_pair(p_i, q_i, p_j, q_j, NOBOX, tmpl)
        for k in ("E", "F_j", "tau_i", "tau_j"):
            np.testing.assert_allclose(res[k], ref[k], rtol=1e-10, atol=1e-10)
        n_checked += res["n_in"] > 0
    assert n_checked >= 4


def test_newton3_and_angular_momentum_balance():
    rng = np.random.default_rng(3)
    for tmpl in (CUBE, CYL):
        for _ in range(4):
            q_i, q_j = rand_q(rng), rand_q(rng)
            R = rng.standard_normal(3)
            R *= (bodies.circumradius(tmpl) * 2 - 0.5) / np.linalg.norm(R)
            res = oracle.bead_pair(np.zeros(3), q_i, R, q_j, NOBOX, tmpl)
            scale = np.abs(res["F_j"]).max() + 1.0
            np.testing.assert_allclose(res["F_i"] + res["F_j"], 0, atol=1e-12 * scale)
            L = res["tau_i"] + res["tau_j"] + np.cross(R, res["F_j"])
            np.testing.assert_allclose(L, 0, atol=1e-11 * scale)


def test_bead_sum_rotation_translation_invariance():
    rng = np.random.default_rng(4)
    q_i, q_j = rand_q(rng), rand_q(rng)
    R = np.array([4.2, 3.1, -2.5])
    base = oracle.bead_pair(np.zeros(3), q_i, R, q_j, NOBOX, CUBE)
    assert base["n_in"] > 0
    for _ in range(3):
        Q = rand_q(rng)
        t = rng.uniform(-10, 10, 3)
        res = oracle.bead_pair(t, bodies.qmul(Q, q_i), t + bodies.qrotate(Q, R),
                               bodies.qmul(Q, q_j), NOBOX, CUBE)
        assert res["E"] == pytest.approx(base["E"], rel=1e-12, abs=1e-12)
        for k in ("F_j", "tau_i", "tau_j"):
            np.testing.assert_allclose(res[k], bodies.qrotate(Q, base[k]), atol=1e-10)


@pytest.mark.parametrize("shape", ["cube", "cylinder"])
def test_bead_forces_torques_are_energy_gradients(shape):
    """F_j = -dE/dp_j and tau_k = -dE/dtheta_k (rotation about space axis k),
    central differences with h = 1e-4 (SI Sec. 6 definitions)."""
    tmpl = CUBE if shape == "cube" else CYL
    rng = np.random.default_rng(5)
    q_i, q_j = rand_q(rng), rand_q(rng)
    d = np.array([0.6, -0.5, 0.62])
    d /= np.linalg.norm(d)
    rho = sampler.contact_distance(d, bodies.qmul(bodies.qconj(q_i), q_j), tmpl, 12.0)
    R = bodies.qrotate(q_i, (rho + 0.4) * d)
    E = lambda pi, qi, pj, qj: oracle.bead_pair(pi, qi, pj, qj, NOBOX, tmpl)["E"]
    res = oracle.bead_pair(np.zeros(3), q_i, R, q_j, NOBOX, tmpl)
    h = 1e-4
    scale = max(1.0, np.abs(res["F_j"]).max(), np.abs(res["tau_j"]).max())
    for k in range(3):
        e = np.eye(3)[k]
        fd = -(E(np.zeros(3), q_i, R + h * e, q_j) - E(np.zeros(3), q_i, R - h * e, q_j)) / (2 * h)
        assert res["F_j"][k] == pytest.approx(fd, abs=2e-6 * scale)
        rp, rm = bodies.qexp(h * e), bodies.qexp(-h * e)
        fd_j = -(E(np.zeros(3), q_i, R, bodies.qmul(rp, q_j))
                 - E(np.zeros(3), q_i, R, bodies.qmul(rm, q_j))) / (2 * h)
        fd_i = -(E(np.zeros(3), bodies.qmul(rp, q_i), R, q_j)
                 - E(np.zeros(3), bodies.qmul(rm, q_i), R, q_j)) / (2 * h)
        assert res["tau_j"][k] == pytest.approx(fd_j, abs=2e-6 * scale)
        assert res["tau_i"][k] == pytest.approx(fd_i, abs=2e-6 * scale)


def test_pair_cutoff_is_tight_superset():
    """Rc = 2 r_circ + r_c: corner beads facing each other along the body
    diagonal interact just inside Rc and not at or beyond it."""
    Rc = bodies.pair_cutoff(CUBE)
    assert Rc == pytest.approx(4 * math.sqrt(3) + 2.5)
    diag = np.ones(3) / math.sqrt(3)
    inside = oracle.bead_pair(np.zeros(3), ID, (Rc - 1e-9) * diag, ID, NOBOX, CUBE)
    assert inside["n_in"] == 1
    for r in [Rc, Rc + 1e-9, Rc + 3.0]:
        out = oracle.bead_pair(np.zeros(3), ID, r * diag, ID, NOBOX, CUBE)
        assert out["E"] == 0.0 and out["n_in"] == 0
    rng = np.random.default_rng(6)
    for _ in range(20):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        out = oracle.bead_pair(np.zeros(3), rand_q(rng), Rc * d, rand_q(rng), NOBOX, CUBE)
        assert out["n_in"] == 0


def test_periodic_minimum_image():
    box = np.array([30.0, 30.0, 30.0])
    rng = np.random.default_rng(7)
    q_i, q_j = rand_q(rng), rand_q(rng)
    p_i = np.array([1.0, 15.0, 29.0])
    R = np.array([-4.0, 3.0, 3.5])
    p_j = np.mod(p_i + R, box)
    a = oracle.bead_pair(p_i, q_i, p_j, q_j, box, CUBE)
    b = oracle.bead_pair(np.zeros(3), q_i, R, q_j, NOBOX, CUBE)
    assert a["n_in"] > 0
    assert a["E"] == pytest.approx(b["E"], rel=1e-12)
    np.testing.assert_allclose(a["F_j"], b["F_j"], rtol=1e-10, atol=1e-12)


def test_pair_search_matches_all_pairs():
    st, L = inputs.system_state(64, 0.10, 1.0, 1, 125.0, [500.0] * 3)
    pos = st["pos"][:, :3].astype(np.float64)
    Rc = bodies.pair_cutoff(CUBE)
    got = {tuple(p) for p in oracle.pairs_bruteforce(pos, [L] * 3, Rc)}
    d = pos[None, :, :] - pos[:, None, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    ref = {(i, j) for i in range(64) for j in range(i + 1, 64) if r[i, j] < Rc}
    assert got == ref and len(ref) > 20


# ------------------------------------------------------------------ bodies

def test_inertia_closed_forms():
    M, I = bodies.mass_and_inertia(CUBE)
    assert M == 125 and len(CUBE) == 125
    np.testing.assert_allclose(I, 500 * np.eye(3), atol=1e-12)  # 2 * 25 * (4+1+0+1+4)
    M, I = bodies.mass_and_inertia(CYL)
    assert M == 152 and len(CYL) == 152
    ixx = 8 * 24 + 19 * 42 * (8 / 7) ** 2  # disc sum y^2 = 24; sum over layers of (l-3.5)^2 = 42
    np.testing.assert_allclose(I, np.diag([ixx, ixx, 384.0]), atol=1e-9)
    assert bodies.circumradius(CUBE) == pytest.approx(2 * math.sqrt(3))
    assert bodies.circumradius(CYL) == pytest.approx(math.sqrt(20))


def test_quaternion_matrix_is_rotation():
    rng = np.random.default_rng(8)
    for _ in range(5):
        q = rand_q(rng)
        R = bodies.qmatrix(q)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0)
    # 90 degrees about z maps x to y
    q = np.array([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)])
    np.testing.assert_allclose(bodies.qrotate(q, [1.0, 0, 0]), [0, 1, 0], atol=1e-15)


# ------------------------------------------------------------------ network

W_SMALL = 16


def rand_params(width=W_SMALL, seed=0):
    mu, isd = inputs.feature_normalisation(5.0, 9.4)
    return nn.unpack(inputs.mlp_params(width, 3, seed, mu=mu, inv_sd=isd, e_scale=2.0,
                                       e_shift=-0.3).astype(np.float64), width)


def rand_pairs(n, seed):
    rng = np.random.default_rng(seed)
    R = rng.standard_normal((n, 3))
    R *= rng.uniform(5.5, 9.0, (n, 1)) / np.linalg.norm(R, axis=1, keepdims=True)
    qi = rng.standard_normal((n, 4))
    qj = rng.standard_normal((n, 4))
    return R, qi / np.linalg.norm(qi, axis=1, keepdims=True), qj / np.linalg.norm(qj, axis=1, keepdims=True)


def energy_np(p, R, qi, qj):
    t = lambda a: torch.as_tensor(np.atleast_2d(a))
    s = nn._to_body(t(qi), t(R))
    return nn.config_energy(p, s, nn._qmul(nn._qconj(t(qi)), t(qj))).detach().numpy()


def test_nn_forces_torques_match_finite_differences():
    p = rand_params()
    R, qi, qj = rand_pairs(6, 9)
    res = nn.pair_forces(p, R, qi, qj)
    h = 1e-5
    for b in range(6):
        for k in range(3):
            e = np.eye(3)[k]
            fd = -(energy_np(p, R[b] + h * e, qi[b], qj[b]) - energy_np(p, R[b] - h * e, qi[b], qj[b])) / (2 * h)
            assert res["F_j"][b, k] == pytest.approx(fd[0], rel=1e-6, abs=1e-8)
            rp, rm = bodies.qexp(h * e), bodies.qexp(-h * e)
            fdj = -(energy_np(p, R[b], qi[b], bodies.qmul(rp, qj[b]))
                    - energy_np(p, R[b], qi[b], bodies.qmul(rm, qj[b]))) / (2 * h)
            fdi = -(energy_np(p, R[b], bodies.qmul(rp, qi[b]), qj[b])
                    - energy_np(p, R[b], bodies.qmul(rm, qi[b]), qj[b])) / (2 * h)
            assert res["tau_j"][b, k] == pytest.approx(fdj[0], rel=1e-6, abs=1e-8)
            assert res["tau_i"][b, k] == pytest.approx(fdi[0], rel=1e-6, abs=1e-8)


def test_nn_newton3_angular_momentum_and_invariance():
    p = rand_params(seed=1)
    R, qi, qj = rand_pairs(8, 10)
    res = nn.pair_forces(p, R, qi, qj)
    np.testing.assert_allclose(res["F_i"] + res["F_j"], 0, atol=1e-14)
    np.testing.assert_allclose(res["tau_i"] + res["tau_j"] + np.cross(R, res["F_j"]), 0, atol=1e-11)
    rng = np.random.default_rng(11)
    Q = rand_q(rng)
    QQ = np.broadcast_to(Q, qi.shape)
    rot = nn.pair_forces(p, bodies.qrotate(QQ, R), bodies.qmul(QQ, qi), bodies.qmul(QQ, qj))
    np.testing.assert_allclose(rot["E"], res["E"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(rot["F_j"], bodies.qrotate(QQ, res["F_j"]), atol=1e-11)
    # the quaternion double cover: -q_j is the same orientation
    neg = nn.pair_forces(p, R, qi, -qj)
    np.testing.assert_allclose(neg["E"], res["E"], rtol=1e-13)
    np.testing.assert_allclose(neg["tau_j"], res["tau_j"], atol=1e-12)


def test_width_one_network_closed_form():
    """A width-1 net is a scalar composition that can be written by hand."""
    p = rand_params(width=1, seed=2)
    R, qi, qj = rand_pairs(3, 12)
    E = energy_np(p, R, qi, qj)
    silu = lambda z: z / (1 + math.exp(-z))
    for b in range(3):
        s = bodies.qrotate(bodies.qconj(qi[b]), R[b])
        qr = bodies.qmul(bodies.qconj(qi[b]), qj[b])
        qr = qr if qr[0] >= 0 else -qr
        rho = math.sqrt(s @ s)
        x = np.concatenate([s, qr, [rho, 1 / rho, rho * rho]])
        xh = (x - p["mu"].numpy()) * p["inv_sd"].numpy()
        h = silu(float(p["W"][0].numpy()[0] @ xh + p["b"][0].item()))
        h = silu(float(p["W"][1].item() * h + p["b"][1].item()))
        h = silu(float(p["W"][2].item() * h + p["b"][2].item()))
        e = p["e_scale"].item() * (p["w_o"].item() * h + p["b_o"].item()) + p["e_shift"].item()
        assert E[b] == pytest.approx(e, rel=1e-13)


def test_flat_layout_size():
    assert nn.n_params(128) == 2 * 10 + 128 * 10 + 128 + 2 * (128 * 128 + 128) + 128 + 3
    assert len(inputs.mlp_params(128)) == nn.n_params(128)


# ------------------------------------------------------------------ training

@pytest.mark.parametrize("fs", [None, 0.7])
def test_force_matching_gradient_matches_finite_differences(fs):
    w = 8
    mu, isd = inputs.feature_normalisation(5.0, 9.4)
    flat = inputs.mlp_params(w, 3, 3, mu=mu, inv_sd=isd).astype(np.float64)
    cfg = inputs.pair_configs(5, 13, 5.5, 9.0).astype(np.float64)
    rng = np.random.default_rng(14)
    lab = rng.standard_normal((5, 10))
    L0, g = nn.force_matching_loss(flat, w, 3, cfg, lab, 0.5, 0.1, fs)
    idx = rng.choice(np.arange(20, len(flat) - 2), 20, replace=False)
    h = 1e-6
    for k in idx:
        fp = flat.copy(); fp[k] += h
        fm = flat.copy(); fm[k] -= h
        fd = (nn.force_matching_loss(fp, w, 3, cfg, lab, 0.5, 0.1, fs)[0]
              - nn.force_matching_loss(fm, w, 3, cfg, lab, 0.5, 0.1, fs)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-8)
    if fs:
        # the weight divides each sample's loss by 1 + |label|^2 / fs^2
        L1, _ = nn.force_matching_loss(flat, w, 3, cfg, lab, 0.5, 0.1, None)
        assert L0 < L1
        # Boltzmann weight: samples with E* <= 0 are untouched, E* > 0 damped by exp(-E*/kT)
        lab2 = lab.copy()
        lab2[:, 0] = -np.abs(lab2[:, 0])
        La, _ = nn.force_matching_loss(flat, w, 3, cfg, lab2, 0.5, 0.1, None, 0.3)
        Lb, _ = nn.force_matching_loss(flat, w, 3, cfg, lab2, 0.5, 0.1, None, None)
        assert La == pytest.approx(Lb, rel=1e-14)


def test_teacher_equals_student_has_zero_gradient():
    w = 8
    flat = inputs.mlp_params(w, 3, 4).astype(np.float64)
    cfg = inputs.pair_configs(6, 15, 5.5, 9.0).astype(np.float64)
    p = nn.unpack(flat, w)
    E, Fj, ti, tj = nn.predict_labels(p, torch.as_tensor(cfg[:, :3]), torch.as_tensor(cfg[:, 3:]))
    lab = np.concatenate([E.detach().numpy()[:, None], Fj.numpy(), ti.numpy(), tj.numpy()], 1)
    L, g = nn.force_matching_loss(flat, w, 3, cfg, lab, 1.0, 1.0)
    assert L < 1e-28
    np.testing.assert_allclose(g, 0, atol=1e-14)


# ------------------------------------------------------------------ integrator

def test_spherical_top_free_rotation_is_exact():
    """Cube: I = 500 1, so the NO_SQUISH split is exact: q(t) = q0 (x) exp(w_b t / 2)."""
    rng = np.random.default_rng(16)
    q0 = np.array([rand_q(rng) for _ in range(4)])
    Lb = rng.standard_normal((4, 3)) * 20
    q, L = q0, Lb
    dt, n = 0.002, 50
    for _ in range(n):
        q, L = md.rotate_free(q, L, [500.0] * 3, dt)
    q_ref = bodies.qmul(q0, bodies.qexp(Lb / 500.0 * dt * n))
    np.testing.assert_allclose(q, q_ref, atol=1e-12)
    # space-frame angular momentum is conserved
    np.testing.assert_allclose(np.einsum("nab,nb->na", bodies.qmatrix(q), L),
                               np.einsum("nab,nb->na", bodies.qmatrix(q0), Lb), atol=1e-10)


def test_symmetric_top_free_rotation_conserves_invariants():
    """Cylinder (I1 = I2 != I3): L_b3 constant, |L_b| constant, space-frame L
    constant, and the body axis precesses about L at rate |L|/I1."""
    _, I = bodies.mass_and_inertia(CYL)
    I = np.diag(I)
    rng = np.random.default_rng(17)
    q0 = rand_q(rng)[None]
    Lb0 = np.array([[30.0, -10.0, 25.0]])
    q, L = q0, Lb0
    dt, n = 0.001, 400
    for _ in range(n):
        q, L = md.rotate_free(q, L, I, dt)
    assert L[0, 2] == pytest.approx(Lb0[0, 2], abs=1e-8)  # O(dt^3) splitting error per step
    assert np.linalg.norm(L) == pytest.approx(np.linalg.norm(Lb0), rel=1e-13)
    Ls0 = bodies.qmatrix(q0[0]) @ Lb0[0]
    np.testing.assert_allclose(bodies.qmatrix(q[0]) @ L[0], Ls0, atol=1e-9)
    # analytic: symmetry axis precesses about L_space with angular rate |L|/I1
    ax0 = bodies.qmatrix(q0[0])[:, 2]
    Lhat = Ls0 / np.linalg.norm(Ls0)
    ang = np.linalg.norm(Ls0) / I[0] * dt * n
    Rp = bodies.qmatrix(bodies.qexp(Lhat * ang))
    ax_t = bodies.qmatrix(q[0])[:, 2]
    np.testing.assert_allclose(ax_t, Rp @ ax0, atol=5e-6)


def _cube_system(n=8, seed=3):
    tmpl = CUBE
    M, I = bodies.mass_and_inertia(tmpl)
    st, L = inputs.system_state(n, 0.12, 1.0, seed, M, np.diag(I))
    box = np.array([L] * 3)
    Rc = bodies.pair_cutoff(tmpl)

    def force_fn(pos, quat):
        pairs = oracle.pairs_bruteforce(pos, box, Rc)
        F, tau, E, _ = oracle.forces_beads(pos, quat, box, tmpl, pairs)
        return F, tau, E

    state = {"pos": st["pos"][:, :3].astype(np.float64), "quat": st["quat"].astype(np.float64),
             "vel": st["vel"][:, :3].astype(np.float64), "angmom": st["angmom"][:, :3].astype(np.float64)}
    return state, force_fn, M, np.diag(I), box


def test_time_reversibility():
    state, force_fn, M, I, box = _cube_system()
    st, _ = md.run(state, force_fn, M, I, box, 0.002, 10)
    back = dict(st, vel=-st["vel"], angmom=-st["angmom"])
    st2, _ = md.run(back, force_fn, M, I, box, 0.002, 10)
    np.testing.assert_allclose(st2["pos"], state["pos"], atol=1e-10)
    np.testing.assert_allclose(np.abs((st2["quat"] * state["quat"]).sum(1)), 1.0, atol=1e-12)


def test_nve_energy_drift_small():
    """Bead forces: the total-energy excursion over a short NVE run stays far
    below N kT (the force jump at the bead cutoff makes it O(dt), not O(dt^2))."""
    state, force_fn, M, I, box = _cube_system(n=27, seed=5)
    _, e = md.run(state, force_fn, M, I, box, 0.002, 40)
    assert np.abs(e - e[0]).max() < 1e-4 * 27


def test_velocity_verlet_is_second_order():
    """With a smooth pair energy (the network with random weights) the energy
    error of the integrator shrinks as dt^2."""
    p = rand_params(seed=7)
    state, _, M, I, box = _cube_system(n=8, seed=6)
    Rc = bodies.pair_cutoff(CUBE)

    def force_fn(pos, quat):
        pairs = oracle.pairs_bruteforce(pos, box, Rc)
        F, tau, E, _ = nn.forces_nn(p, pos, quat, box, pairs)
        return F, tau, E

    state = dict(state, vel=state["vel"] * 20, angmom=state["angmom"] * 20)
    _, e1 = md.run(state, force_fn, M, I, box, 0.004, 10)
    _, e2 = md.run(state, force_fn, M, I, box, 0.002, 20)
    d1 = np.abs(e1 - e1[0]).max()
    d2 = np.abs(e2 - e2[0]).max()
    assert d1 > 1e-12
    assert 2.5 < d1 / d2 < 6.0, (d1, d2)


# ------------------------------------------------------------------ sampler

def test_contact_bisection_finds_sigma():
    u = inputs.sampler_uniforms(5, 18).astype(np.float64)
    d, q = sampler.draws_to_config(u)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-15)
    Rc = bodies.pair_cutoff(CUBE)
    for b in range(5):
        rc = sampler.contact_distance(d[b], q[b], CUBE, Rc)
        md_ = oracle.min_bead_distance(np.zeros(3), ID, rc * d[b], q[b], NOBOX, CUBE)
        assert md_ == pytest.approx(1.0, abs=1e-9)
        assert 4.0 < rc < Rc
    # aligned cubes along a face normal touch when the face planes are 1 sigma apart
    rc = sampler.contact_distance(np.array([1.0, 0, 0]), ID, CUBE, Rc)
    assert rc == pytest.approx(5.0, abs=1e-9)


def test_contact_bisection_at_a_smaller_distance():
    """Contact defined at 0.85 sigma: the bisection lands on that smallest bead
    distance, and aligned cubes touch at 4 + 0.85 sigma."""
    u = inputs.sampler_uniforms(4, 19).astype(np.float64)
    d, q = sampler.draws_to_config(u)
    Rc = bodies.pair_cutoff(CUBE)
    for b in range(4):
        rc = sampler.contact_distance(d[b], q[b], CUBE, Rc, 0.85)
        md_ = oracle.min_bead_distance(np.zeros(3), ID, rc * d[b], q[b], NOBOX, CUBE)
        assert md_ == pytest.approx(0.85, abs=1e-9)
    rc = sampler.contact_distance(np.array([1.0, 0, 0]), ID, CUBE, Rc, 0.85)
    assert rc == pytest.approx(4.85, abs=1e-9)
