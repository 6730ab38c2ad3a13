"""GPU parity of the network's smooth energy cutoff (rb_mlp_set_cutoff)
against the FP64 oracle (oracle/nn.py, switch): pair outputs at both
precisions across the switching band, whole-system forces, the training
gradient and the second-order weight product, with the cube's point group
attached as in training.  Configurations within 1e-4 of a boundary of the
canonical choice are left out, as in test_gpu_symmetry.py."""
import numpy as np
import pytest

from oracle import bodies, nn, symmetry
from paper_2402_12199_gb300 import inputs
from tests.helpers import TOL_BF16, TOL_F32, assert_parity, gpu_system, make_state, rel_err

pytestmark = pytest.mark.gpu
MARGIN = 1e-4
R_ON, R_OFF = 8.4, 9.4


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _setup(width, seed):
    from paper_2402_12199_gb300 import api

    group = symmetry.point_group(bodies.cube_template())
    mu, isd = inputs.feature_normalisation(5.0, 9.43)
    flat = inputs.mlp_params(width, 3, seed, mu=mu, inv_sd=isd, e_scale=1.3, e_shift=-0.2)
    m = api.MLP(width, 3)
    m.set_params(flat)
    m.set_symmetry(group[0].astype(np.float32), group[1])
    m.set_cutoff(R_ON, R_OFF)
    p = nn.unpack(flat.astype(np.float64), width, sym=group, cutoff=(R_ON, R_OFF))
    return group, flat, m, p


def _configs(n, seed, group, rho=(R_ON - 0.4, R_OFF + 0.3)):
    c7 = inputs.pair_configs(n, seed, *rho).astype(np.float64)
    _, _, _, mk, mj = symmetry.choose(c7[:, :3], c7[:, 3:], group)
    _, cq = symmetry.canonical(c7[:, :3], c7[:, 3:], group)
    ok = (mk > MARGIN) & (mj > MARGIN) & (np.abs(cq[:, 0]) > MARGIN)
    c7 = c7[ok].astype(np.float32)
    c8 = np.zeros((len(c7), 8), np.float32)
    c8[:, :3] = c7[:, :3]
    c8[:, 4:] = c7[:, 3:]
    return c8


@pytest.mark.parametrize("width,precision,tol", [(128, "fp32", TOL_F32), (128, "bf16", TOL_BF16),
                                                 (256, "bf16", TOL_BF16), (128, "f16x3", TOL_F32)])
def test_switched_pairs_parity(width, precision, tol):
    import torch

    group, flat, m, p = _setup(width, 3 + width)
    c8 = _configs(1200, 4 + width, group)
    out = m.pairs(torch.from_numpy(c8).cuda(), precision).double().cpu().numpy()
    s = torch.as_tensor(c8[:, :3].astype(np.float64))
    q = torch.as_tensor(c8[:, 4:].astype(np.float64))
    E, Fj, ti, tj = nn.predict_labels(p, s, q)
    rho = np.linalg.norm(c8[:, :3].astype(np.float64), axis=1)
    beyond = rho >= R_OFF
    assert beyond.any() and (rho < R_ON).any()
    # beyond r_off: exactly nothing
    assert np.all(out[beyond][:, [0, 1, 2, 3, 4, 5, 6, 8, 9, 10]] == 0.0)
    assert_parity(out[:, 0:3], Fj.numpy(), tol)
    assert_parity(out[:, 4:7], ti.numpy(), tol)
    assert_parity(out[:, 8:11], tj.numpy(), tol)
    assert_parity(out[:, 3], E.detach().numpy(), tol)


def test_switched_system_forces_parity():
    import oracle

    group, flat, m, p = _setup(128, 11)
    st, L, tmpl = make_state(1000, 0.20, 12)
    s = gpu_system(st, L)
    r = s.forces_nn(m, "fp32")
    s.sync()
    pos = st["pos"][:, :3].astype(np.float64)
    qa = st["quat"].astype(np.float64)
    pairs = oracle.pairs_bruteforce(pos, np.array([L] * 3), bodies.pair_cutoff(tmpl))
    F, T, E, per = nn.forces_nn(p, pos, qa, np.array([L] * 3), pairs)
    i, j = pairs[:, 0], pairs[:, 1]
    d = pos[j] - pos[i]
    d -= L * np.rint(d / L)
    sb = bodies.qrotate(bodies.qconj(qa[i]), d)
    qr = bodies.qmul(bodies.qconj(qa[i]), qa[j])
    _, _, _, mk, mj = symmetry.choose(sb, qr, group)
    _, cq = symmetry.canonical(sb, qr, group)
    bad = np.unique(pairs[np.minimum(np.minimum(mk, mj), np.abs(cq[:, 0])) < MARGIN].ravel())
    keep = np.setdiff1d(np.arange(len(pos)), bad)
    assert len(keep) > 0.95 * len(pos)
    assert_parity(r["force"][:, :3].double().cpu().numpy()[keep], F[keep], TOL_F32)
    assert_parity(r["torque"][:, :3].double().cpu().numpy()[keep], T[keep], TOL_F32)


def test_switched_training_gradient_and_weight_vjp():
    import torch

    from paper_2402_12199_gb300 import api

    width = 64
    group, flat, m, p = _setup(width, 21)
    c8 = _configs(220, 22, group)
    B = len(c8)
    rng = np.random.default_rng(23)
    lab = rng.standard_normal((B, 10)) * 0.3
    l12 = np.zeros((B, 12), np.float32)
    l12[:, 0:3] = lab[:, 1:4]
    l12[:, 3] = lab[:, 0]
    l12[:, 4:7] = lab[:, 4:7]
    l12[:, 8:11] = lab[:, 7:10]
    tr = api.Trainer(m, B)
    c8d = torch.from_numpy(c8).cuda()
    loss, g = tr.grad(c8d, torch.from_numpy(l12).cuda(), 0.5, 0.1)
    c7 = np.concatenate([c8[:, :3], c8[:, 4:]], 1).astype(np.float64)
    L_ref, g_ref = nn.force_matching_loss(flat.astype(np.float64), width, 3, c7,
                                          lab.astype(np.float32).astype(np.float64), 0.5, 0.1,
                                          sym=group, cutoff=(R_ON, R_OFF))
    assert loss == pytest.approx(L_ref, rel=1e-5)
    assert rel_err(g.double().cpu().numpy(), g_ref) < 1e-5
    # the second-order product of the switched output S E_hat
    u = rng.standard_normal((B, 8)).astype(np.float32)
    u[:, 3] = 0.0
    c = rng.standard_normal(B).astype(np.float32)
    gv = tr.weight_vjp(c8d, torch.from_numpy(u).cuda(), torch.from_numpy(c).cuda())
    ft = torch.as_tensor(flat.astype(np.float64)).requires_grad_(True)
    sq = torch.as_tensor(c7).requires_grad_(True)
    rho = torch.sqrt((sq[:, :3] ** 2).sum(-1))
    # S E_hat with E_hat the unswitched output before e_scale / e_shift
    pu = nn.unpack(ft, width, sym=group)
    Ehat = (nn.config_energy(pu, sq[:, :3], sq[:, 3:]) - pu["e_shift"]) / pu["e_scale"]
    SEh = nn.switch(rho, R_ON, R_OFF) * Ehat
    (gsq,) = torch.autograd.grad(SEh.sum(), [sq], create_graph=True)
    uu = torch.as_tensor(np.concatenate([u[:, :3], u[:, 4:]], 1).astype(np.float64))
    J = (gsq * uu).sum() + (torch.as_tensor(c.astype(np.float64)) * SEh).sum()
    (gref,) = torch.autograd.grad(J, [ft])
    gref = gref.numpy().copy()
    gref[:20] = 0.0
    gref[-2:] = 0.0
    assert rel_err(gv.double().cpu().numpy(), gref) < 1e-5


def test_switched_network_md_conserves_energy():
    from paper_2402_12199_gb300 import api

    group, flat, m, p = _setup(128, 31)
    st, L, tmpl = make_state(512, 0.2, 6)
    s = gpu_system(st, L)
    s.forces_nn(m, "fp32")
    e0 = sum(s.energy())
    s.step(50, 0.002, path=api.RB_PATH_NN, mlp=m, precision="fp32")
    e1 = sum(s.energy())
    s.sync()
    assert np.isfinite(e1) and abs(e1 - e0) < 1e-2 * 512, (e0, e1)
