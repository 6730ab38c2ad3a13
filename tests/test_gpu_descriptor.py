"""GPU parity of the network on the paper's six numbers of a cube pair
(rb_mlp_set_descriptor RB_DESC_PAPER6; paper SI Sec. 1 for the numbers,
SI Sec. 6 for forces and torques as their energy gradients) against the FP64
oracle (oracle/descriptor.py, oracle/nn.py with desc="paper6"):

- the six numbers themselves (rb_nn_features);
- pair outputs at each precision and width (FP32 SIMT, F16X3, BF16 tensor
  cores at width 128, BF16 and FP32 at width 256), over several tiles with a
  ragged tail;
- whole-system forces and torques, with the smooth cutoff;
- the force-matching weight gradient (the training tangent through the six
  numbers);
- the calls that must be refused.
Configurations within 2e-2 (coordinate units or radians) of a switch of the
description (ties of the frame or face choice, the wrap of alpha_3, and
sin(alpha_1) small, where alpha_2 is undefined) are left out: there FP32 and
FP64 may take different, equally valid descriptions, or the angles' FP32
rounding is amplified by 1 / sin(alpha_1)."""
import math

import numpy as np
import pytest

from oracle import bodies, descriptor, nn, symmetry
from paper_2402_12199_gb300 import inputs
from tests.helpers import TOL_BF16, TOL_F32, assert_parity, gpu_system, make_state, rel_err

pytestmark = pytest.mark.gpu
MARGIN = 2e-2
MU = [6.5, 3.0, 1.5, 1.2, 0.0, 0.8, 0.0, 0.0, 0.0, 0.0]
ISD = [0.6, 0.6, 0.8, 0.7, 0.5, 1.8, 0.0, 0.0, 0.0, 0.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _net(width, seed, cutoff=None):
    from paper_2402_12199_gb300 import api

    flat = inputs.mlp_params(width, 3, seed, mu=MU, inv_sd=ISD, e_scale=1.4, e_shift=-0.3)
    group = symmetry.point_group(bodies.cube_template())
    m = api.MLP(width, 3)
    m.set_params(flat)
    m.set_symmetry(group[0].astype(np.float32), group[1])
    m.set_descriptor("paper6")
    if cutoff:
        m.set_cutoff(*cutoff)
    p = nn.unpack(flat.astype(np.float64), width, desc="paper6", cutoff=cutoff)
    return flat, m, p


def _configs(n, seed, rho=(4.8, 9.6)):
    c7 = inputs.pair_configs(3 * n, seed, *rho).astype(np.float32)
    c64 = c7.astype(np.float64)
    ok = descriptor.margins(c64[:, :3], c64[:, 3:]) > MARGIN
    c7 = c7[ok][:n]
    assert len(c7) == n
    c8 = np.zeros((n, 8), np.float32)
    c8[:, :3] = c7[:, :3]
    c8[:, 4:] = c7[:, 3:]
    return c7.astype(np.float64), c8


def test_six_numbers_match_oracle():
    import torch

    _, m, _ = _net(128, 1)
    c7, c8 = _configs(3000, 2)
    x = m.features(torch.from_numpy(c8).cuda()).double().cpu().numpy()
    ref = descriptor.describe_np(c7[:, :3], c7[:, 3:])
    np.testing.assert_allclose(x[:, :3], ref[:, :3], atol=2e-5)
    np.testing.assert_allclose(x[:, 3:5], ref[:, 3:5], atol=2e-5)
    assert descriptor.angle_gap(x[:, 5], ref[:, 5], 0.5 * math.pi).max() < 2e-5
    assert np.all(x[:, 6:] == 0.0)
    # ranges of the description
    assert np.all((x[:, 0] >= x[:, 1]) & (x[:, 1] >= x[:, 2]) & (x[:, 2] >= 0))
    assert np.all((x[:, 5] >= 0) & (x[:, 5] < 0.5 * math.pi))


@pytest.mark.parametrize("width,precision,tol,n", [(128, "fp32", TOL_F32, 1000),
                                                   (128, "f16x3", TOL_F32, 1000),
                                                   (128, "bf16", TOL_BF16, 1000),
                                                   (256, "bf16", TOL_BF16, 777),
                                                   (256, "fp32", TOL_F32, 300),
                                                   (128, "f16x3", TOL_F32, 5000)])
def test_pairs_parity(width, precision, tol, n):
    import torch

    flat, m, p = _net(width, 3 + width + n, cutoff=(8.4, 9.43))
    c7, c8 = _configs(n, 4 + n)
    out = m.pairs(torch.from_numpy(c8).cuda(), precision).double().cpu().numpy()
    E, Fj, ti, tj = nn.predict_labels(p, torch.as_tensor(c7[:, :3]), torch.as_tensor(c7[:, 3:]))
    assert np.isfinite(out).all()
    assert_parity(out[:, 0:3], Fj.numpy(), tol, "F_j")
    assert_parity(out[:, 4:7], ti.numpy(), tol, "tau_i")
    assert_parity(out[:, 8:11], tj.numpy(), tol, "tau_j")
    assert_parity(out[:, 3], E.detach().numpy(), tol, "E")


@pytest.mark.parametrize("precision,tol", [("fp32", TOL_F32), ("f16x3", TOL_F32), ("bf16", TOL_BF16)])
def test_system_forces_parity(precision, tol):
    import oracle

    flat, m, p = _net(128, 21, cutoff=(8.43, 9.43))
    st, L, tmpl = make_state(1500, 0.20, 22)
    s = gpu_system(st, L)
    r = s.forces_nn(m, precision)
    s.sync()
    pos = st["pos"][:, :3].astype(np.float64)
    qa = st["quat"].astype(np.float64)
    box = np.array([L] * 3)
    pairs = oracle.pairs_bruteforce(pos, box, bodies.pair_cutoff(tmpl))
    F, T, E, per = nn.forces_nn(p, pos, qa, box, pairs)
    i, j = pairs[:, 0], pairs[:, 1]
    d = pos[j] - pos[i]
    d -= L * np.rint(d / L)
    sb = bodies.qrotate(bodies.qconj(qa[i]), d)
    qr = bodies.qmul(bodies.qconj(qa[i]), qa[j])
    bad = np.unique(pairs[descriptor.margins(sb, qr) < MARGIN].ravel())
    keep = np.setdiff1d(np.arange(len(pos)), bad)
    assert len(keep) > 0.5 * len(pos), len(keep)  # about 6 pairs per body, each may be near a switch
    assert_parity(r["force"][:, :3].double().cpu().numpy()[keep], F[keep], tol, "force")
    assert_parity(r["torque"][:, :3].double().cpu().numpy()[keep], T[keep], tol, "torque")


def test_training_gradient_parity():
    import torch

    from paper_2402_12199_gb300 import api

    width = 64
    flat, m, p = _net(width, 31, cutoff=(8.4, 9.43))
    c7, c8 = _configs(200, 32)
    B = len(c8)
    rng = np.random.default_rng(33)
    lab = rng.standard_normal((B, 10)) * 0.3
    l12 = np.zeros((B, 12), np.float32)
    l12[:, 0:3] = lab[:, 1:4]
    l12[:, 3] = lab[:, 0]
    l12[:, 4:7] = lab[:, 4:7]
    l12[:, 8:11] = lab[:, 7:10]
    tr = api.Trainer(m, B)
    loss, g = tr.grad(torch.from_numpy(c8).cuda(), torch.from_numpy(l12).cuda(), 0.5, 0.1)
    L_ref, g_ref = nn.force_matching_loss(flat.astype(np.float64), width, 3, c7,
                                          lab.astype(np.float32).astype(np.float64), 0.5, 0.1,
                                          cutoff=(8.4, 9.43), desc="paper6")
    assert loss == pytest.approx(L_ref, rel=1e-5)
    g = g.double().cpu().numpy()
    # the four constant inputs (mu = inv_sd = 0) give their weights no gradient
    W1 = g[20:20 + width * 10].reshape(width, 10)
    assert np.all(W1[:, 6:] == 0.0)
    assert rel_err(g, g_ref) < 1e-5


def test_refused_without_the_cube_group():
    from paper_2402_12199_gb300 import api

    m = api.MLP(128, 3)
    m.set_params(inputs.mlp_params(128, 3, 1))
    with pytest.raises(api.RBError):
        m.set_descriptor("paper6")
    cyl = symmetry.point_group(bodies.cylinder_template())
    cube = symmetry.point_group(bodies.cube_template())
    m.set_symmetry(cube[0].astype(np.float32), cube[1])
    m.set_descriptor("paper6")
    with pytest.raises(api.RBError):
        m.set_symmetry(cyl[0].astype(np.float32), cyl[1])
    with pytest.raises(api.RBError):
        m.set_symmetry(np.zeros((0, 4), np.float32), False)
    m.set_descriptor("features10")
    m.set_symmetry(cyl[0].astype(np.float32), cyl[1])
