"""GPU parity of the symmetry-reduced network path against the FP64 oracle
(oracle/symmetry.py): the canonical representatives themselves, the network's
pair outputs at both precisions and widths, whole-system forces, the training
gradient and the second-order weight product, all with the cube's point group
attached to the network.

Configurations within 1e-4 of a boundary of the canonical choice (where FP32
and FP64 may legitimately pick different, equally valid representatives) are
left out of the comparisons; in the system test, so are the bodies of pairs
that close to one."""
import numpy as np
import pytest

from oracle import bodies, nn, symmetry
from paper_2402_12199_gb300 import inputs
from tests.helpers import TOL_BF16, TOL_F32, assert_parity, gpu_system, make_state, rel_err

pytestmark = pytest.mark.gpu
MARGIN = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _group(shape="cube"):
    return symmetry.point_group(bodies.cube_template() if shape == "cube" else bodies.cylinder_template())


def _mlp(width, seed, group, depth=3):
    from paper_2402_12199_gb300 import api

    mu, isd = inputs.feature_normalisation(5.0, 9.43)
    flat = inputs.mlp_params(width, depth, seed, mu=mu, inv_sd=isd, e_scale=1.4, e_shift=-0.1)
    m = api.MLP(width, depth)
    m.set_params(flat)
    m.set_symmetry(group[0].astype(np.float32), group[1])
    return flat, m


def _safe_configs(n, seed, group, rho=(5.0, 9.4)):
    """Seeded configurations away from the canonical choice's boundaries and
    from the scalar-part sign switch of the canonical orientation."""
    c7 = inputs.pair_configs(n, seed, *rho).astype(np.float64)
    _, _, _, mk, mj = symmetry.choose(c7[:, :3], c7[:, 3:], group)
    _, cq = symmetry.canonical(c7[:, :3], c7[:, 3:], group)
    ok = (mk > MARGIN) & (mj > MARGIN) & (np.abs(cq[:, 0]) > MARGIN)
    assert ok.mean() > 0.95
    c7 = c7[ok].astype(np.float32)
    c8 = np.zeros((len(c7), 8), np.float32)
    c8[:, :3] = c7[:, :3]
    c8[:, 4:] = c7[:, 3:]
    return c7, c8


@pytest.mark.parametrize("shape", ["cube", "cylinder", "cube rotations only"])
def test_canonical_matches_oracle(shape):
    """The cube's full group takes the library's closed-form choice; the
    cylinder's group and the cube's rotations without the inversion take the
    scan over the group's table."""
    import torch

    from paper_2402_12199_gb300 import api

    group = _group("cylinder" if shape == "cylinder" else "cube")
    if shape == "cube rotations only":
        group = (group[0], False)
    m = api.MLP(64, 3)
    m.set_params(inputs.mlp_params(64, 3, 1))
    m.set_symmetry(group[0].astype(np.float32), group[1])
    c7, c8 = _safe_configs(3000, 11, group, (5.0, 11.4))
    # the oracle maps what the GPU sees: the FP32 configurations
    s64, q64 = c8[:, :3].astype(np.float64), c8[:, 4:].astype(np.float64)
    rng = np.random.default_rng(12)
    lab = rng.standard_normal((len(c8), 12)).astype(np.float32)
    lab[:, 7] = lab[:, 11] = 0.0
    cfg_t, lab_t = torch.from_numpy(c8.copy()).cuda(), torch.from_numpy(lab.copy()).cuda()
    m.canonical(cfg_t, lab_t)
    cfg_g, lab_g = cfg_t.double().cpu().numpy(), lab_t.double().cpu().numpy()
    k, sg, j, _, _ = symmetry.choose(s64, q64, group)
    cs, cq = symmetry.canonical(s64, q64, group)
    np.testing.assert_allclose(cfg_g[:, :3], cs, atol=2e-5)
    np.testing.assert_allclose(cfg_g[:, 4:], cq, atol=2e-6)
    R = bodies.qmatrix(group[0][k])
    lab64 = lab.astype(np.float64)
    np.testing.assert_allclose(lab_g[:, 0:3], sg[:, None] * np.einsum("bij,bj->bi", R, lab64[:, 0:3]), atol=2e-6)
    np.testing.assert_allclose(lab_g[:, 4:7], np.einsum("bij,bj->bi", R, lab64[:, 4:7]), atol=2e-6)
    np.testing.assert_allclose(lab_g[:, 8:11], np.einsum("bij,bj->bi", R, lab64[:, 8:11]), atol=2e-6)
    np.testing.assert_array_equal(lab_g[:, 3], lab64[:, 3])


@pytest.mark.parametrize("width,precision,tol", [(64, "fp32", TOL_F32), (128, "fp32", TOL_F32),
                                                 (256, "fp32", TOL_F32), (128, "bf16", TOL_BF16),
                                                 (256, "bf16", TOL_BF16), (128, "f16x3", TOL_F32)])
def test_symmetric_pairs_parity(width, precision, tol):
    import torch

    group = _group()
    flat, m = _mlp(width, 21 + width, group)
    c7, c8 = _safe_configs(1500, 22 + width, group)
    out, g = m.pairs(torch.from_numpy(c8).cuda(), precision, grad=True)
    out, g = out.double().cpu().numpy(), g.double().cpu().numpy()
    p = nn.unpack(flat.astype(np.float64), width, sym=group)
    s = torch.as_tensor(c8[:, :3].astype(np.float64))
    q = torch.as_tensor(c8[:, 4:].astype(np.float64))
    E, Fj, ti, tj = nn.predict_labels(p, s, q)
    assert_parity(out[:, 0:3], Fj.numpy(), tol)
    assert_parity(out[:, 4:7], ti.numpy(), tol)
    assert_parity(out[:, 8:11], tj.numpy(), tol)
    assert_parity(out[:, 3], E.detach().numpy(), tol)
    # dE/d(s, q_rel) of the raw configuration
    sq = torch.cat([s, q], 1).requires_grad_(True)
    (gref,) = torch.autograd.grad(nn.config_energy(p, sq[:, :3], sq[:, 3:]).sum(), [sq])
    assert_parity(g[:, 0:3], gref[:, :3].numpy(), tol)
    assert_parity(g[:, 4:8], gref[:, 3:].numpy(), tol)


def test_symmetric_network_is_invariant_on_gpu():
    import torch

    group = _group()
    quats = group[0]
    flat, m = _mlp(128, 31, group)
    c7, c8 = _safe_configs(800, 32, group)
    base = m.pairs(torch.from_numpy(c8).cuda(), "fp32").double().cpu().numpy()
    rng = np.random.default_rng(33)
    for _ in range(4):
        k, j, sg = rng.integers(24), rng.integers(24), rng.choice([1.0, -1.0])
        s2, q2 = symmetry.apply(c8[:, :3].astype(np.float64), c8[:, 4:].astype(np.float64), group,
                                k, sg, j)
        c2 = np.zeros_like(c8)
        c2[:, :3] = s2
        c2[:, 4:] = q2
        out = m.pairs(torch.from_numpy(c2).cuda(), "fp32").double().cpu().numpy()
        R = bodies.qmatrix(quats[k])
        assert_parity(out[:, 3], base[:, 3], TOL_F32)
        assert_parity(out[:, 0:3], sg * base[:, 0:3] @ R.T, TOL_F32)
        assert_parity(out[:, 4:7], base[:, 4:7] @ R.T, TOL_F32)
        assert_parity(out[:, 8:11], base[:, 8:11] @ R.T, TOL_F32)


def _pair_margins(st, L, pairs, group):
    pos = st["pos"][:, :3].astype(np.float64)
    q = st["quat"].astype(np.float64)
    i, j = pairs[:, 0], pairs[:, 1]
    d = pos[j] - pos[i]
    d -= L * np.rint(d / L)
    s = bodies.qrotate(bodies.qconj(q[i]), d)
    qr = bodies.qmul(bodies.qconj(q[i]), q[j])
    _, _, _, mk, mj = symmetry.choose(s, qr, group)
    _, cq = symmetry.canonical(s, qr, group)
    return np.minimum(np.minimum(mk, mj), np.abs(cq[:, 0]))


@pytest.mark.parametrize("precision,tol", [("fp32", TOL_F32), ("bf16", TOL_BF16),
                                           ("f16x3", TOL_F32)])
def test_symmetric_system_forces_parity(precision, tol):
    import oracle

    group = _group()
    st, L, tmpl = make_state(1000, 0.20, 41)
    flat, m = _mlp(128, 42, group)
    s = gpu_system(st, L)
    r = s.forces_nn(m, precision)
    s.sync()
    pos = st["pos"][:, :3].astype(np.float64)
    pairs = oracle.pairs_bruteforce(pos, np.array([L] * 3), bodies.pair_cutoff(tmpl))
    p = nn.unpack(flat.astype(np.float64), 128, sym=group)
    F, T, E, per = nn.forces_nn(p, pos, st["quat"].astype(np.float64), np.array([L] * 3), pairs)
    bad = np.unique(pairs[_pair_margins(st, L, pairs, group) < MARGIN].ravel())
    keep = np.setdiff1d(np.arange(len(pos)), bad)
    assert len(keep) > 0.95 * len(pos)
    assert_parity(r["force"][:, :3].double().cpu().numpy()[keep], F[keep], tol)
    assert_parity(r["torque"][:, :3].double().cpu().numpy()[keep], T[keep], tol)


def _train_setup(width, B, seed):
    import torch

    from paper_2402_12199_gb300 import api

    group = _group()
    flat, m = _mlp(width, seed, group)
    c7, c8 = _safe_configs(B, seed + 1, group)
    B = len(c8)
    rng = np.random.default_rng(seed + 2)
    lab = rng.standard_normal((B, 10))
    l12 = np.zeros((B, 12), np.float32)
    l12[:, 0:3] = lab[:, 1:4]
    l12[:, 3] = lab[:, 0]
    l12[:, 4:7] = lab[:, 4:7]
    l12[:, 8:11] = lab[:, 7:10]
    tr = api.Trainer(m, max(B, 64))
    return group, flat, c8, lab.astype(np.float32), m, tr, torch.from_numpy(c8).cuda(), \
        torch.from_numpy(l12).cuda()


@pytest.mark.parametrize("width,B", [(64, 200), (128, 120)])
def test_symmetric_force_matching_gradient_parity(width, B):
    group, flat, c8, lab, m, tr, c8d, l12 = _train_setup(width, B, 50 + width)
    loss, g = tr.grad(c8d, l12, 0.5, 0.1)
    c7 = np.concatenate([c8[:, :3], c8[:, 4:]], 1).astype(np.float64)
    L_ref, g_ref = nn.force_matching_loss(flat.astype(np.float64), width, 3, c7,
                                          lab.astype(np.float64), 0.5, 0.1, sym=group)
    assert loss == pytest.approx(L_ref, rel=1e-5)
    assert rel_err(g.double().cpu().numpy(), g_ref) < 1e-5


def test_symmetric_weight_vjp_is_second_order_product():
    import torch

    width = 64
    group, flat, c8, lab, m, tr, c8d, l12 = _train_setup(width, 60, 70)
    B = len(c8)
    rng = np.random.default_rng(71)
    u = rng.standard_normal((B, 8)).astype(np.float32)
    u[:, 3] = 0.0
    c = rng.standard_normal(B).astype(np.float32)
    g = tr.weight_vjp(c8d, torch.from_numpy(u).cuda(), torch.from_numpy(c).cuda())
    ft = torch.as_tensor(flat.astype(np.float64)).requires_grad_(True)
    p = nn.unpack(ft, width, sym=group)
    sq = torch.as_tensor(np.concatenate([c8[:, :3], c8[:, 4:]], 1).astype(np.float64)).requires_grad_(True)
    Eh = (nn.config_energy(p, sq[:, :3], sq[:, 3:]) - p["e_shift"]) / p["e_scale"]
    (gsq,) = torch.autograd.grad(Eh.sum(), [sq], create_graph=True)
    uu = torch.as_tensor(np.concatenate([u[:, :3], u[:, 4:]], 1).astype(np.float64))
    J = (gsq * uu).sum() + (torch.as_tensor(c.astype(np.float64)) * Eh).sum()
    (gref,) = torch.autograd.grad(J, [ft])
    gref = gref.numpy().copy()
    gref[:20] = 0.0
    gref[-2:] = 0.0
    assert rel_err(g.double().cpu().numpy(), gref) < 1e-5


def test_symmetric_network_md_conserves_energy():
    from paper_2402_12199_gb300 import api

    group = _group()
    st, L, tmpl = make_state(512, 0.2, 6)
    flat, m = _mlp(128, 80, group)
    s = gpu_system(st, L)
    s.forces_nn(m, "fp32")
    e0 = sum(s.energy())
    s.step(50, 0.002, path=api.RB_PATH_NN, mlp=m, precision="fp32")
    e1 = sum(s.energy())
    s.sync()
    assert np.isfinite(e1) and abs(e1 - e0) < 1e-2 * 512, (e0, e1)
