"""GPU parity of the per-component cylinder networks (rb_fnet_*) against the
FP64 oracle (oracle/fnet.py): pair outputs at widths 16, 32, 64 and depths 1
and 3, whole-system forces and torques, the regression gradient on sampled
and bead-labelled cylinder pairs, a short training run, and momentum
conservation of an MD run with these forces.

Configurations within 1e-4 of a boundary of the four-number description
(p_z = 0 or u_z = 0, where a frame axis or cylinder 2's axis turns over;
p_r = 0; the branch cut of phi; theta = 0, where phi has no meaning) are left
out of element-wise comparisons: there FP32 and FP64 may pick different, equally
valid descriptions."""
import numpy as np
import pytest

from oracle import bodies, fnet
from paper_2402_12199_gb300 import inputs
from tests.helpers import TOL_F32, assert_parity, gpu_system, make_state, rel_err

pytestmark = pytest.mark.gpu
MARGIN = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _flat(width, depth, seed):
    rng = np.random.default_rng(seed)
    n = fnet.net_size(width, depth)
    flat = rng.standard_normal(5 * n) / np.sqrt(width)
    for c in range(5):
        o = c * n
        flat[o:o + 4] = [6.0, 3.0, 0.8, 0.0]
        flat[o + 4:o + 8] = [0.3, 0.3, 1.2, 0.5]
        flat[o + n - 2] = 0.7 + 0.1 * c
        flat[o + n - 1] = 0.05 * c
    return flat.astype(np.float32)


def _clear(s, q):
    """Mask of configurations away from the description's boundaries (FP64)."""
    xh, yh, zh, d = fnet.frame(s, q)
    a2 = bodies.qrotate(q, np.broadcast_to([0.0, 0, 1], (len(s), 3)))
    uz = (a2 * zh).sum(1)
    return ((np.abs(s[:, 2]) > MARGIN) & (np.abs(uz) > MARGIN) & (d[:, 0] > MARGIN)
            & (d[:, 2] > 1e-3) & (np.pi - np.abs(d[:, 3]) > MARGIN))


def _configs(n, seed):
    rng = np.random.default_rng(seed)
    direc = rng.standard_normal((n, 3))
    direc /= np.linalg.norm(direc, axis=1, keepdims=True)
    s = direc * rng.uniform(3.0, 11.4, (n, 1))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    s32, q32 = s.astype(np.float32), q.astype(np.float32)
    keep = _clear(s32.astype(np.float64), q32.astype(np.float64))
    return s32[keep], q32[keep]


@pytest.mark.parametrize("width,depth", [(16, 1), (32, 3), (64, 3), (64, 1)])
def test_fnet_pair_outputs_parity(width, depth):
    import torch

    from paper_2402_12199_gb300 import api

    flat = _flat(width, depth, 10 + width + depth)
    f = api.FNet(width, depth)
    f.set_params(flat)
    s, q = _configs(1500, 20 + width)
    cfg = np.zeros((len(s), 8), np.float32)
    cfg[:, :3] = s
    cfg[:, 4:] = q
    out = f.pairs(torch.from_numpy(cfg).cuda()).double().cpu().numpy()
    nets = fnet.unpack(flat.astype(np.float64), width, depth)
    Fj, ti, tj, _ = fnet.predict(nets, s.astype(np.float64), q.astype(np.float64))
    assert_parity(out[:, 0:3], Fj, TOL_F32)
    assert_parity(out[:, 4:7], ti, TOL_F32)
    assert_parity(out[:, 8:11], tj, TOL_F32)
    assert np.all(out[:, [3, 7, 11]] == 0.0)


def test_fnet_system_forces_parity():
    import oracle
    from paper_2402_12199_gb300 import api

    width, depth = 32, 3
    flat = _flat(width, depth, 31)
    f = api.FNet(width, depth)
    f.set_params(flat)
    st, L, tmpl = make_state(400, 0.15, 32, "cylinder")
    s = gpu_system(st, L, "cylinder")
    r = s.forces_fnet(f)
    s.sync()
    pos = st["pos"][:, :3].astype(np.float64)
    quat = st["quat"].astype(np.float64)
    box = np.array([L] * 3)
    pairs = oracle.pairs_bruteforce(pos, box, bodies.pair_cutoff(tmpl))
    i, j = pairs[:, 0], pairs[:, 1]
    R = bodies.min_image(pos[j] - pos[i], box)
    sb = bodies.qrotate(bodies.qconj(quat[i]), R)
    qr = bodies.qmul(bodies.qconj(quat[i]), quat[j])
    bad = np.unique(pairs[~_clear(sb, qr)].ravel())
    keep = np.setdiff1d(np.arange(len(pos)), bad)
    assert len(pairs) > 300 and len(keep) > 0.9 * len(pos)
    F, T = fnet.forces_fnet(fnet.unpack(flat.astype(np.float64), width, depth), pos, quat, box, pairs)
    assert_parity(r["force"][:, :3].double().cpu().numpy()[keep], F[keep], TOL_F32)
    assert_parity(r["torque"][:, :3].double().cpu().numpy()[keep], T[keep], TOL_F32)
    # Newton 3: the total force vanishes (FP32 rounding only)
    tot = r["force"][:, :3].double().sum(0).abs().max().item()
    assert tot < 1e-4 * np.abs(F).sum()


def _sampled(n, seed, contact=None):
    import torch

    from paper_2402_12199_gb300 import api

    s = api.System(8, [60.0] * 3, "cylinder")
    u = inputs.sampler_uniforms(n, seed)
    cfg, lab, _ = api.sample_pairs(s, torch.from_numpy(u).cuda(), contact)
    c = cfg.double().cpu().numpy()
    keep = _clear(c[:, :3], c[:, 4:8])
    idx = torch.from_numpy(np.nonzero(keep)[0]).cuda()
    return cfg[idx].contiguous(), lab[idx].contiguous()


def test_fnet_training_gradient_matches_oracle():
    from paper_2402_12199_gb300 import api

    width, depth = 16, 2
    flat = _flat(width, depth, 41)
    f = api.FNet(width, depth)
    f.set_params(flat)
    cfg, lab = _sampled(700, 42)
    B = cfg.shape[0]
    tr = api.FNetTrainer(f, B)
    c = cfg.double().cpu().numpy()
    lb = lab.double().cpu().numpy()
    for cap, fs in ((0.0, 0.0), (5.0, 0.0), (5.0, 1.5)):  # plain, capped, capped and weighted
        tr.set_cap(cap, fs)
        loss, g = tr.grad(cfg, lab)
        d, t = fnet.targets(c[:, :3], c[:, 4:8], lb[:, 0:3], lb[:, 4:7], cap=cap or None)
        L_ref, g_ref = fnet.loss_and_grad(flat.astype(np.float64), width, depth, d, t,
                                          f_scale=fs or None)
        assert loss == pytest.approx(L_ref, rel=1e-5)
        assert rel_err(g.double().cpu().numpy(), g_ref) < 1e-5


def test_fnet_training_reduces_the_loss():
    from paper_2402_12199_gb300 import api

    width, depth = 32, 3
    f = api.FNet(width, depth)
    flat = _flat(width, depth, 51)
    n = fnet.net_size(width, depth)
    for c in range(5):  # output scale of the bead-sum labels
        flat[c * n + n - 2] = 1.0
        flat[c * n + n - 1] = 0.0
    f.set_params(flat)
    cfg, lab = _sampled(40000, 52, contact=1.2)
    B = 2048
    tr = api.FNetTrainer(f, B, lr=2e-3)
    tr.set_cap(5.0)
    first = tr.grad(cfg[:B], lab[:B])[0]
    for k in range(300):
        o = (k * B) % (cfg.shape[0] - B)
        tr.step(cfg[o:o + B], lab[o:o + B])
    last = tr.grad(cfg[:B], lab[:B])[0]
    assert np.isfinite(last) and last < 0.7 * first, (first, last)


def test_fnet_md_conserves_momentum():
    import torch

    from paper_2402_12199_gb300 import api

    width, depth = 32, 2
    f = api.FNet(width, depth)
    flat = _flat(width, depth, 61)
    n = fnet.net_size(width, depth)
    for c in range(5):  # gentle random forces
        flat[c * n + n - 2] = 0.05
    f.set_params(flat)
    st, L, tmpl = make_state(1000, 0.15, 62, "cylinder")
    s = gpu_system(st, L, "cylinder")
    s.set_skin(0.4)
    p0 = (s.get_state(to_host=True)["vel"][:, :3].astype(np.float64)).sum(0) * s.mass
    s.step_fnet(f, 200, 0.002)
    cur = s.get_state(to_host=True)
    s.sync()
    p1 = cur["vel"][:, :3].astype(np.float64).sum(0) * s.mass
    assert np.all(np.isfinite(cur["pos"]))
    scale = np.abs(cur["vel"][:, :3]).sum() * s.mass
    assert np.abs(p1 - p0).max() < 1e-5 * scale


def test_parameter_change_on_the_network_stream_reaches_the_system():
    """The per-component networks' parameters and kernel image are written on
    their own stream; a system on another stream that evaluates right after a
    change sees the new values (the network's stream is held busy by a bounded
    spin before each device-to-device parameter copy)."""
    import torch

    from paper_2402_12199_gb300 import api

    width, depth = 32, 3
    sets = [torch.from_numpy(_flat(width, depth, seed)).cuda() for seed in (41, 42)]
    st, L, tmpl = make_state(400, 0.15, 32, "cylinder")
    s = gpu_system(st, L, "cylinder")
    ref = []
    for flat in sets:
        f0 = api.FNet(width, depth)
        f0.set_params(flat)
        r = s.forces_fnet(f0)
        s.sync()
        ref.append((r["force"].clone(), r["torque"].clone()))
    assert not torch.equal(ref[0][0], ref[1][0])
    ns = torch.cuda.Stream()
    f = api.FNet(width, depth, stream=ns)
    for k in range(4):
        with torch.cuda.stream(ns):
            torch.cuda._sleep(2_000_000)  # about 1 ms of the network's stream
        f.set_params(sets[k % 2])
        r = s.forces_fnet(f)
        s.sync()
        assert torch.equal(r["force"], ref[k % 2][0]), k
        assert torch.equal(r["torque"], ref[k % 2][1]), k
