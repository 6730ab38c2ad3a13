"""Pins of the oracle's pair-symmetrised network energy,
E_s(i, j) = (E(x_ij) + E(x_ji)) / 2 (the network evaluated with each body of
the pair as the reference, averaged), against facts that do not come from
the oracle: invariance under relabelling the bodies (which the plain network
lacks), Newton's third law and angular-momentum balance, and forces and
torques as central finite differences of the symmetrised energy."""
import numpy as np
import pytest

import oracle
from oracle import bodies, nn
from paper_2402_12199_gb300 import inputs

W = 16
BIG = np.array([1000.0] * 3)  # a box far larger than any pair: no periodic image


def params(seed):
    mu, isd = inputs.feature_normalisation(5.0, 9.4)
    return nn.unpack(inputs.mlp_params(W, 3, seed, mu=mu, inv_sd=isd, e_scale=2.0,
                                       e_shift=-0.3).astype(np.float64), W)


def small_system(n, seed, L=40.0):
    rng = np.random.default_rng(seed)
    # a loose lattice keeps every pair well inside the network's range
    g = int(np.ceil(n ** (1 / 3)))
    sites = np.stack(np.meshgrid(*[np.arange(g)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n]
    pos = sites * (L / g) + rng.uniform(-0.5, 0.5, (n, 3))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return pos, q, np.array([L] * 3)


def pairs_within(pos, box, rc):
    return oracle.pairs_bruteforce(pos, box, rc)


def test_relabelling_the_bodies_leaves_the_symmetrised_energy_unchanged():
    p = params(3)
    pos, q, box = small_system(27, 4)
    pairs = pairs_within(pos, box, 14.0)
    assert len(pairs) > 20
    F, T, E, _ = nn.forces_nn_symmetrised(p, pos, q, box, pairs)
    perm = np.random.default_rng(5).permutation(len(pos))
    inv = np.argsort(perm)
    pos2, q2 = pos[perm], q[perm]
    # the same physical pairs under the new labels, each listed i < j as the
    # library lists them: about half change their reference body
    pairs2 = np.sort(inv[pairs], axis=1)
    assert np.any(inv[pairs][:, 0] > inv[pairs][:, 1])
    F2, T2, E2, _ = nn.forces_nn_symmetrised(p, pos2, q2, box, pairs2)
    assert E2 == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(F2, F[perm], atol=1e-11)
    np.testing.assert_allclose(T2, T[perm], atol=1e-11)
    # the plain network is not invariant (so this pin has teeth)
    _, _, Ep, _ = nn.forces_nn(p, pos, q, box, pairs)
    _, _, Ep2, _ = nn.forces_nn(p, pos2, q2, box, pairs2)
    assert abs(Ep2 - Ep) > 1e-6 * abs(Ep)


def test_swapping_every_pair_leaves_it_unchanged():
    p = params(6)
    pos, q, box = small_system(8, 7, L=20.0)
    pairs = pairs_within(pos, box, 11.0)
    a = nn.forces_nn_symmetrised(p, pos, q, box, pairs)
    b = nn.forces_nn_symmetrised(p, pos, q, box, pairs[:, ::-1])
    assert a[2] == pytest.approx(b[2], rel=1e-13)
    np.testing.assert_allclose(a[0], b[0], atol=1e-12)
    np.testing.assert_allclose(a[1], b[1], atol=1e-12)


def test_newton3_and_angular_momentum_balance():
    p = params(8)
    rng = np.random.default_rng(9)
    for _ in range(5):
        d = rng.standard_normal(3)
        d *= rng.uniform(5.5, 9.0) / np.linalg.norm(d)
        pos = np.array([[0.0, 0, 0], d])
        q = rng.standard_normal((2, 4))
        q /= np.linalg.norm(q, axis=1, keepdims=True)
        F, T, _, _ = nn.forces_nn_symmetrised(p, pos, q, BIG, np.array([[0, 1]]))
        np.testing.assert_allclose(F[0] + F[1], 0, atol=1e-13)
        np.testing.assert_allclose(T[0] + T[1] + np.cross(d, F[1]), 0, atol=1e-11)


def test_forces_and_torques_are_finite_differences_of_the_symmetrised_energy():
    p = params(10)
    rng = np.random.default_rng(11)
    d = rng.standard_normal(3)
    d *= 7.0 / np.linalg.norm(d)
    pos = np.array([[0.0, 0, 0], d])
    q = rng.standard_normal((2, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    pr = np.array([[0, 1]])

    def energy(pp, qq):
        return nn.forces_nn_symmetrised(p, pp, qq, BIG, pr)[2]

    F, T, _, _ = nn.forces_nn_symmetrised(p, pos, q, BIG, pr)
    h = 1e-5
    for b in range(2):
        for k in range(3):
            e = np.eye(3)[k]
            pp, pm = pos.copy(), pos.copy()
            pp[b] += h * e
            pm[b] -= h * e
            assert F[b, k] == pytest.approx(-(energy(pp, q) - energy(pm, q)) / (2 * h), rel=1e-6,
                                            abs=1e-9)
            qp, qm = q.copy(), q.copy()
            qp[b] = bodies.qmul(bodies.qexp(h * e), q[b])
            qm[b] = bodies.qmul(bodies.qexp(-h * e), q[b])
            assert T[b, k] == pytest.approx(-(energy(pos, qp) - energy(pos, qm)) / (2 * h), rel=1e-6,
                                            abs=1e-9)


# ------------------------------------------------- swapped reference body

def _sampled(n, seed, tmpl):
    from oracle import sampler

    u = inputs.sampler_uniforms(n, seed)
    cfg, lab, _ = sampler.sample_pairs(u, tmpl, bodies.pair_cutoff(tmpl))
    return cfg, lab


def test_swapping_the_reference_twice_is_the_identity():
    from oracle import sampler

    cfg, lab = _sampled(6, 51, bodies.cube_template())
    c2, l2 = sampler.swap_reference(*sampler.swap_reference(cfg, lab))
    np.testing.assert_allclose(c2, cfg, atol=1e-13)
    np.testing.assert_allclose(l2, lab, atol=1e-12)


@pytest.mark.parametrize("shape", ["cube", "cylinder"])
def test_swapped_labels_are_the_bead_sum_of_the_swapped_configuration(shape):
    """The bead sum is symmetric in its two identical bodies, so the labels
    computed afresh at the swapped configuration must equal the swapped
    labels: pins the rotation of every component."""
    from oracle import sampler

    tmpl = bodies.cube_template() if shape == "cube" else bodies.cylinder_template()
    cfg, lab = _sampled(5, 52, tmpl)
    sc, sl = sampler.swap_reference(cfg, lab)
    fresh = sampler.label_pairs(sc, tmpl)
    scale = np.abs(lab).max()
    np.testing.assert_allclose(fresh, sl, atol=1e-10 * scale, rtol=1e-10)
