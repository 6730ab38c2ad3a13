"""GPU parity of the training path: the on-device pair sampler (contact
bisection + bead-sum labels), the force-matching loss and its weight
gradient (forward-over-reverse), the second-order weight product behind the
autograd wrapper, and Adam steps, against the FP64 oracle."""
import numpy as np
import pytest

from oracle import bodies, nn, sampler
from paper_2402_12199_gb300 import inputs
from tests.helpers import TOL_F32, assert_parity, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def cube_system(n=8):
    from paper_2402_12199_gb300 import api

    return api.System(n, [40.0] * 3, "cube")


def lab10(lab12):
    """(n, 12) library label layout -> (n, 10) oracle layout (E, F_j, tau_i, tau_j)."""
    lab12 = np.asarray(lab12, dtype=np.float64)
    return np.concatenate([lab12[:, 3:4], lab12[:, 0:3], lab12[:, 4:7], lab12[:, 8:11]], 1)


def cfg7(cfg8):
    cfg8 = np.asarray(cfg8, dtype=np.float64)
    return np.concatenate([cfg8[:, :3], cfg8[:, 4:8]], 1)


@pytest.mark.parametrize("shape,contact", [("cube", None), ("cylinder", None), ("cube", 0.85)])
def test_sampler_matches_oracle(shape, contact):
    import torch

    from paper_2402_12199_gb300 import api

    tmpl = bodies.cube_template() if shape == "cube" else bodies.cylinder_template()
    s = api.System(8, [60.0] * 3, shape)
    u = inputs.sampler_uniforms(48, 5)
    cfg, lab, rc = api.sample_pairs(s, torch.from_numpy(u).cuda(), contact)
    torch.cuda.synchronize()
    cfg, lab, rc = cfg.cpu().numpy(), lab.cpu().numpy(), rc.cpu().numpy()
    d, q = sampler.draws_to_config(u.astype(np.float64))
    np.testing.assert_allclose(cfg[:, 4:8], q, atol=2e-6)
    Rc = bodies.pair_cutoff(tmpl)
    for b in range(0, 48, 6):
        rc_ref = sampler.contact_distance(d[b], q[b], tmpl, Rc, contact or 1.0)
        assert rc[b] == pytest.approx(rc_ref, abs=2e-5)
    rho = np.linalg.norm(cfg[:, :3], axis=1)
    assert np.all(rho >= rc - 1e-4) and np.all(rho <= Rc + 1e-4)
    # labels: the oracle's bead sum at exactly the sampled configurations
    ref = sampler.label_pairs(cfg7(cfg), tmpl)
    got = lab10(lab)
    assert_parity(got[:, 1:4], ref[:, 1:4], TOL_F32)
    assert_parity(got[:, 4:7], ref[:, 4:7], TOL_F32)
    assert_parity(got[:, 7:10], ref[:, 7:10], TOL_F32)
    assert np.abs(got[:, 0] - ref[:, 0]).max() <= TOL_F32 * max(1.0, np.abs(ref[:, 0]).max())


def _setup(width, B, seed, lam_tau=0.5, lam_E=0.1):
    import torch

    from paper_2402_12199_gb300 import api

    mu, isd = inputs.feature_normalisation(5.0, 9.43)
    flat = inputs.mlp_params(width, 3, seed, mu=mu, inv_sd=isd, e_scale=1.3, e_shift=0.2)
    c7 = inputs.pair_configs(B, seed + 1, 5.0, 9.4)
    rng = np.random.default_rng(seed + 2)
    lab = rng.standard_normal((B, 10))
    m = api.MLP(width, 3)
    m.set_params(flat)
    tr = api.Trainer(m, max(B, 64))
    c8 = np.zeros((B, 8), np.float32)
    c8[:, :3] = c7[:, :3]
    c8[:, 4:] = c7[:, 3:]
    l12 = np.zeros((B, 12), np.float32)
    l12[:, 0:3] = lab[:, 1:4]
    l12[:, 3] = lab[:, 0]
    l12[:, 4:7] = lab[:, 4:7]
    l12[:, 8:11] = lab[:, 7:10]
    return flat, c7, lab.astype(np.float32), m, tr, torch.from_numpy(c8).cuda(), torch.from_numpy(l12).cuda()


@pytest.mark.parametrize("width,B,fs,kt", [(64, 200, 0.0, 0.0), (128, 96, 0.0, 0.0),
                                           (128, 1, 0.0, 0.0), (128, 150, 1.5, 0.7)])
def test_force_matching_gradient_parity(width, B, fs, kt):
    flat, c7, lab, m, tr, c8, l12 = _setup(width, B, width + B)
    loss, g = tr.grad(c8, l12, 0.5, 0.1, fs, kt)
    L_ref, g_ref = nn.force_matching_loss(flat.astype(np.float64), width, 3, c7.astype(np.float64),
                                          lab.astype(np.float64), 0.5, 0.1, fs or None, kt or None)
    assert loss == pytest.approx(L_ref, rel=1e-5)
    assert rel_err(g.double().cpu().numpy(), g_ref) < 1e-5


def test_weight_vjp_is_second_order_product():
    import torch

    width, B = 64, 50
    flat, c7, lab, m, tr, c8, l12 = _setup(width, B, 77)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((B, 8)).astype(np.float32)
    u[:, 3] = 0.0
    c = rng.standard_normal(B).astype(np.float32)
    g = tr.weight_vjp(c8, torch.from_numpy(u).cuda(), torch.from_numpy(c).cuda())
    # oracle: d/dW sum_b [u_b . dE_hat/d(s, q) + c_b E_hat] by autograd
    ft = torch.as_tensor(flat.astype(np.float64)).requires_grad_(True)
    p = nn.unpack(ft, width)
    sq = torch.as_tensor(c7.astype(np.float64)).requires_grad_(True)
    Eh = (nn.config_energy(p, sq[:, :3], sq[:, 3:]) - p["e_shift"]) / p["e_scale"]
    (gsq,) = torch.autograd.grad(Eh.sum(), [sq], create_graph=True)
    uu = torch.as_tensor(np.concatenate([u[:, :3], u[:, 4:]], 1).astype(np.float64))
    J = (gsq * uu).sum() + (torch.as_tensor(c.astype(np.float64)) * Eh).sum()
    (gref,) = torch.autograd.grad(J, [ft])
    gref = gref.numpy().copy()
    gref[:20] = 0.0
    gref[-2:] = 0.0
    assert rel_err(g.double().cpu().numpy(), gref) < 1e-5


def test_adam_steps_match_oracle():
    """Two rb_train_step updates against the oracle's Adam (adam_update) on the
    gradients the library reports for the same batches (rb_train_grad, which
    rb_train_step recomputes in the same fixed order), so both sides start
    each step from identical FP32 weights and gradients.  Compared: the weight
    change of each step (FP32 rounding of the weights is ~3e-8 against steps
    of lr = 1e-2) and the untrained entries (normalisation, energy scale and
    shift), which must not move."""
    width, B, lr = 64, 128, 1e-2
    flat, c7, lab, m, tr, c8, l12 = _setup(width, B, 41)
    tr.set_lr(lr)
    _, _, _, _, _, c8b, l12b = _setup(width, B, 42)
    w = m.get_params().astype(np.float64)
    mom = np.zeros_like(w)
    vel = np.zeros_like(w)
    for t, (c, l) in enumerate(((c8, l12), (c8b, l12b)), start=1):
        _, g = tr.grad(c, l, 0.5, 0.1)
        g = g.double().cpu().numpy()
        assert np.median(np.abs(g[20:-2])) > 1e-5  # |g| >> eps: the update is not eps-dominated
        tr.step(c, l, 0.5, 0.1, want_loss=False)
        w_new = m.get_params().astype(np.float64)
        ref, mom, vel = nn.adam_update(w, g, mom, vel, t, lr)
        assert np.array_equal(w_new[:20], w[:20]) and np.array_equal(w_new[-2:], w[-2:])
        assert rel_err(w_new - w, ref - w) < 1e-5, t
        assert np.abs((w_new - w) - (ref - w)).max() < 1e-6, t
        w = w_new


def test_adam_steps_fit_a_teacher():
    """Labels from a teacher network: Adam steps on the student's
    force-matching loss drive the loss down."""
    import torch

    from paper_2402_12199_gb300 import api

    mu, isd = inputs.feature_normalisation(5.0, 9.43)
    teacher = inputs.mlp_params(64, 3, 100, mu=mu, inv_sd=isd)
    student = inputs.mlp_params(64, 3, 101, mu=mu, inv_sd=isd)
    B = 512
    c7 = inputs.pair_configs(B, 102, 5.0, 9.4)
    c8 = np.zeros((B, 8), np.float32)
    c8[:, :3] = c7[:, :3]
    c8[:, 4:] = c7[:, 3:]
    c8 = torch.from_numpy(c8).cuda()
    mt = api.MLP(64, 3)
    mt.set_params(teacher)
    lab = mt.pairs(c8, "fp32")
    ms = api.MLP(64, 3)
    ms.set_params(student)
    tr = api.Trainer(ms, B, lr=3e-3)
    l0 = tr.step(c8, lab, 1.0, 0.1)
    for _ in range(150):
        l1 = tr.step(c8, lab, 1.0, 0.1, want_loss=False)
    l1 = tr.grad(c8, lab, 1.0, 0.1)[0]
    assert l1 < 0.2 * l0, (l0, l1)


def test_autograd_wrapper_double_backward():
    """Force matching through torch autograd on the library's wrapper: the
    gradient of a force-based loss with respect to the parameters equals the
    oracle's."""
    import torch

    from paper_2402_12199_gb300.autograd import NNEnergy

    width, B = 64, 40
    flat, c7, lab, m, tr, c8, l12 = _setup(width, B, 55)
    f = NNEnergy(width, 3, 256)
    params = torch.from_numpy(flat).cuda().requires_grad_(True)
    cfg = c8.clone().requires_grad_(True)
    E = f(cfg, params)
    (G,) = torch.autograd.grad(E.sum(), [cfg], create_graph=True)
    target = torch.from_numpy(np.random.default_rng(1).standard_normal((B, 8))).float().cuda()
    target[:, 3] = 0.0
    loss = ((G - target) ** 2).sum() + 0.3 * (E ** 2).sum()
    (gp,) = torch.autograd.grad(loss, [params])
    # oracle
    ft = torch.as_tensor(flat.astype(np.float64)).requires_grad_(True)
    p = nn.unpack(ft, width)
    sq = torch.as_tensor(c7.astype(np.float64)).requires_grad_(True)
    Eo = nn.config_energy(p, sq[:, :3], sq[:, 3:])
    (Go,) = torch.autograd.grad(Eo.sum(), [sq], create_graph=True)
    t = target.double().cpu()
    t7 = torch.cat([t[:, :3], t[:, 4:]], 1)
    lo = ((Go - t7) ** 2).sum() + 0.3 * (Eo ** 2).sum()
    (gref,) = torch.autograd.grad(lo, [ft])
    gref = gref.numpy().copy()
    gref[:20] = 0.0
    gref[-2:] = 0.0
    g = gp.double().cpu().numpy()
    assert rel_err(g, gref) < 1e-5
