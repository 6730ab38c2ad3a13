"""Pins of the oracle's symmetry-reduced configurations (oracle/symmetry.py)
against the physics and the mathematics, not against itself:

  * the point groups have the orders geometry fixes (cube: the 24 rotations
    of the octahedral group plus inversion; hexagonal-disc cylinder: the 12 of
    the hexagonal prism plus inversion; a 3 x 4 x 6 box: 4 plus inversion; a
    cube missing one corner bead: the 3 rotations about that body diagonal,
    no inversion);
  * the bead double sum (the C oracle) gives the same energy for every
    group-related configuration, and its forces and torques transform as the
    canonical map claims (F_j -> sigma R F_j, tau -> R tau);
  * the canonical configuration is the same for every group-related
    configuration;
  * a network on canonical configurations is exactly invariant, and its
    forces and torques are still central differences of its energy.
"""
import numpy as np
import pytest
import torch

from oracle import bodies, nn, sampler, symmetry
from paper_2402_12199_gb300 import inputs

CUBE = bodies.cube_template()
CYL = bodies.cylinder_template()
BOX = np.stack(np.meshgrid(np.arange(3) - 1.0, np.arange(4) - 1.5, np.arange(6) - 2.5,
                           indexing="ij"), -1).reshape(-1, 3)


def test_point_group_orders():
    g = symmetry.point_group(CUBE)
    assert len(g[0]) == 24 and g[1]
    g = symmetry.point_group(CYL)
    assert len(g[0]) == 12 and g[1]
    g = symmetry.point_group(BOX)
    assert len(g[0]) == 4 and g[1]
    corner = CUBE[~np.all(CUBE == 2.0, axis=1)]
    assert len(corner) == 124
    g = symmetry.point_group(corner)
    assert len(g[0]) == 3 and not g[1]
    # the rotations of the cut cube keep the missing corner's diagonal
    for q in g[0]:
        np.testing.assert_allclose(bodies.qrotate(q, np.array([1.0, 1, 1])), [1, 1, 1], atol=1e-12)


def test_group_is_closed_and_contains_identity():
    quats, _ = symmetry.point_group(CUBE)
    np.testing.assert_allclose(quats[0], [1, 0, 0, 0])
    for a in quats:
        for b in quats:
            c = bodies.qmul(a, b)
            assert min(min(np.abs(c - q).max(), np.abs(c + q).max()) for q in quats) < 1e-12


def _configs(tmpl, n, seed):
    rng = np.random.default_rng(seed)
    Rc = bodies.pair_cutoff(tmpl)
    u = rng.random((n, 6))
    u[:, 5] *= 0.5  # keep near contact so the forces are large
    cfg, lab, _ = sampler.sample_pairs(u, tmpl, Rc)
    return cfg, lab


@pytest.mark.parametrize("tmpl", [CUBE, CYL], ids=["cube", "cylinder"])
def test_bead_sum_is_invariant_under_the_point_group(tmpl):
    group = symmetry.point_group(tmpl)
    quats, inversion = group
    cfg, lab = _configs(tmpl, 3, 1)
    assert np.abs(lab[:, 1:4]).max() > 1e-2
    combos = [(k, sg, 0) for k in range(len(quats)) for sg in ((1.0, -1.0) if inversion else (1.0,))]
    combos += [(0, 1.0, j) for j in range(len(quats))]
    for b in range(len(cfg)):
        s, q = cfg[b, :3], cfg[b, 3:]
        for k, sg, j in combos:
            s2, q2 = symmetry.apply(s, q, group, k, sg, j)
            lab2 = sampler.label_pairs(np.concatenate([s2, q2])[None], tmpl)[0]
            R = bodies.qmatrix(quats[k])
            scale = np.abs(lab[b]).max()
            assert lab2[0] == pytest.approx(lab[b, 0], abs=1e-11 * scale)
            np.testing.assert_allclose(lab2[1:4], sg * R @ lab[b, 1:4], atol=1e-11 * scale)
            np.testing.assert_allclose(lab2[4:7], R @ lab[b, 4:7], atol=1e-11 * scale)
            np.testing.assert_allclose(lab2[7:10], R @ lab[b, 7:10], atol=1e-11 * scale)


@pytest.mark.parametrize("tmpl", [CUBE, CYL], ids=["cube", "cylinder"])
def test_canonical_configuration_is_group_invariant(tmpl):
    group = symmetry.point_group(tmpl)
    quats, inversion = group
    rng = np.random.default_rng(2)
    c7 = inputs.pair_configs(200, 3, 5.0, 11.0).astype(np.float64)
    s, q = c7[:, :3], c7[:, 3:]
    _, _, _, mk, mj = symmetry.choose(s, q, group)
    ok = (mk > 1e-6) & (mj > 1e-6)
    assert ok.mean() > 0.95
    s, q = s[ok], q[ok]
    cs, cq = symmetry.canonical(s, q, group)
    # the canonical orientation is the representative closest to the identity
    assert np.all(np.abs(cq[:, 0]) >= np.abs(bodies.qmul(cq[:, None, :], quats[None])[..., 0]).max(1) - 1e-12)
    for _ in range(6):
        k = rng.integers(len(quats))
        j = rng.integers(len(quats))
        sg = rng.choice([1.0, -1.0]) if inversion else 1.0
        s2, q2 = symmetry.apply(s, q, group, k, sg, j)
        ts, tq = symmetry.canonical(s2, q2, group)
        np.testing.assert_allclose(ts, cs, atol=1e-10)
        # q and -q are the same rotation
        d = np.minimum(np.abs(tq - cq).max(1), np.abs(tq + cq).max(1))
        assert d.max() < 1e-10


def test_symmetric_network_is_invariant_and_differentiable():
    group = symmetry.point_group(CUBE)
    mu, isd = inputs.feature_normalisation(5.0, 9.4)
    flat = inputs.mlp_params(16, 3, 4, mu=mu, inv_sd=isd, e_scale=2.0, e_shift=-0.3)
    p = nn.unpack(flat.astype(np.float64), 16, sym=group)
    c7 = inputs.pair_configs(40, 5, 5.5, 9.0).astype(np.float64)
    s, q = c7[:, :3], c7[:, 3:]
    _, _, _, mk, mj = symmetry.choose(s, q, group)
    keep = (mk > 1e-3) & (mj > 1e-3) & (np.abs(symmetry.canonical(s, q, group)[1][:, 0]) > 1e-3)
    s, q = s[keep], q[keep]
    E, Fj, ti, tj = nn.predict_labels(p, torch.as_tensor(s), torch.as_tensor(q))
    E = E.detach().numpy()
    rng = np.random.default_rng(6)
    quats, _ = group
    for _ in range(5):
        k, j, sg = rng.integers(24), rng.integers(24), rng.choice([1.0, -1.0])
        s2, q2 = symmetry.apply(s, q, group, k, sg, j)
        E2, F2, ti2, tj2 = nn.predict_labels(p, torch.as_tensor(s2), torch.as_tensor(q2))
        np.testing.assert_allclose(E2.detach().numpy(), E, atol=1e-12)
        R = bodies.qmatrix(quats[k])
        np.testing.assert_allclose(F2.numpy(), sg * Fj.numpy() @ R.T, atol=1e-10)
        np.testing.assert_allclose(tj2.numpy(), tj.numpy() @ R.T, atol=1e-10)
        np.testing.assert_allclose(ti2.numpy(), ti.numpy() @ R.T, atol=1e-10)

    def energy(s_, q_):
        return nn.config_energy(p, torch.as_tensor(s_), torch.as_tensor(q_)).detach().numpy()

    h = 1e-5
    for a in range(3):
        e = np.eye(3)[a] * h
        fd = -(energy(s + e, q) - energy(s - e, q)) / (2 * h)
        np.testing.assert_allclose(Fj.numpy()[:, a], fd, rtol=1e-6, atol=1e-8)
        rp = np.broadcast_to(bodies.qexp(e), q.shape)
        rm = np.broadcast_to(bodies.qexp(-e), q.shape)
        fdj = -(energy(s, bodies.qmul(rp, q)) - energy(s, bodies.qmul(rm, q))) / (2 * h)
        np.testing.assert_allclose(tj.numpy()[:, a], fdj, rtol=1e-6, atol=1e-8)
        # rotating body i turns s and q the other way
        fdi = -(energy(bodies.qrotate(rm, s), bodies.qmul(rm, q))
                - energy(bodies.qrotate(rp, s), bodies.qmul(rp, q))) / (2 * h)
        np.testing.assert_allclose(ti.numpy()[:, a], fdi, rtol=1e-6, atol=1e-8)


def test_cutoff_switch_is_smooth_and_exact_at_its_ends():
    """The network's cutoff factor: 1 up to r_on, 0 from r_off, continuous
    with its first two derivatives (central differences), and a network with
    it has forces and torques that are central differences of its energy in
    the switching region, and exactly zero energy beyond r_off."""
    r_on, r_off = 8.4, 9.4
    rho = torch.linspace(7.0, 10.0, 3001, dtype=torch.float64)
    S = nn.switch(rho, r_on, r_off).numpy()
    r = rho.numpy()
    assert np.all(S[r <= r_on] == 1.0) and np.all(S[r >= r_off] == 0.0)
    assert np.all(np.diff(S) <= 1e-15)
    h = 1e-4
    for x in (r_on, r_off):
        for side in (-1, 1):
            xs = torch.tensor([x + side * 2 * h, x + side * h, x], dtype=torch.float64)
            v = nn.switch(xs, r_on, r_off).numpy()
            # first derivative 0 at the end; second derivative 0 at the end,
            # so the one-sided second difference (centred one step in) is O(h)
            assert abs(v[1] - v[2]) / h < 1e-6
            assert abs(v[0] - 2 * v[1] + v[2]) / h ** 2 < 100 * h
    mid = nn.switch(torch.tensor([0.5 * (r_on + r_off)], dtype=torch.float64), r_on, r_off)
    assert float(mid[0]) == pytest.approx(0.5)

    group = symmetry.point_group(CUBE)
    mu, isd = inputs.feature_normalisation(5.0, 9.4)
    flat = inputs.mlp_params(16, 3, 7, mu=mu, inv_sd=isd, e_scale=2.0, e_shift=-0.3)
    p = nn.unpack(flat.astype(np.float64), 16, sym=group, cutoff=(r_on, r_off))
    c7 = inputs.pair_configs(40, 8, 8.3, 9.6).astype(np.float64)
    s, q = c7[:, :3], c7[:, 3:]
    _, _, _, mk, mj = symmetry.choose(s, q, group)
    keep = (mk > 1e-3) & (mj > 1e-3) & (np.abs(symmetry.canonical(s, q, group)[1][:, 0]) > 1e-3)
    s, q = s[keep], q[keep]
    E, Fj, ti, tj = nn.predict_labels(p, torch.as_tensor(s), torch.as_tensor(q))
    rho = np.linalg.norm(s, axis=1)
    assert np.all(E.detach().numpy()[rho >= r_off] == 0.0)
    assert np.all(Fj.numpy()[rho >= r_off] == 0.0)

    def energy(s_, q_):
        return nn.config_energy(p, torch.as_tensor(s_), torch.as_tensor(q_)).detach().numpy()

    for a in range(3):
        e = np.eye(3)[a] * h
        fd = -(energy(s + e, q) - energy(s - e, q)) / (2 * h)
        np.testing.assert_allclose(Fj.numpy()[:, a], fd, rtol=1e-6, atol=1e-8)
        rp = np.broadcast_to(bodies.qexp(e), q.shape)
        rm = np.broadcast_to(bodies.qexp(-e), q.shape)
        fdj = -(energy(s, bodies.qmul(rp, q)) - energy(s, bodies.qmul(rm, q))) / (2 * h)
        np.testing.assert_allclose(tj.numpy()[:, a], fdj, rtol=1e-6, atol=1e-8)
