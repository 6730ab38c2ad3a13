"""GPU parity of the FP32 pair-network path (features, MLP forward, reverse
pass, geometric adjoint) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import bodies, nn
from paper_2402_12199_gb300 import inputs
from tests.helpers import (TOL_F32, assert_parity, canonical_margin, gpu_system, make_state,
                           oracle_nn, rel_err)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def params(width, seed, depth=3):
    mu, isd = inputs.feature_normalisation(5.0, 9.43)
    return inputs.mlp_params(width, depth, seed, mu=mu, inv_sd=isd, e_scale=1.5, e_shift=-0.2)


def cfg8(cfg7):
    c = np.zeros((len(cfg7), 8), np.float32)
    c[:, :3] = cfg7[:, :3]
    c[:, 4:] = cfg7[:, 3:]
    return c


def oracle_labels(flat, width, cfg7, depth=3):
    import torch

    p = nn.unpack(np.asarray(flat, np.float64), width, depth)
    c = torch.as_tensor(cfg7.astype(np.float64))
    E, Fj, ti, tj = nn.predict_labels(p, c[:, :3], c[:, 3:])
    return E.detach().numpy(), Fj.numpy(), ti.numpy(), tj.numpy()


@pytest.mark.parametrize("width,n", [(128, 4096), (128, 1000), (64, 777), (256, 333), (128, 1)])
def test_nn_pairs_parity(width, n):
    import torch

    from paper_2402_12199_gb300 import api

    flat = params(width, width + n)
    m = api.MLP(width, 3)
    m.set_params(flat)
    cfg7 = inputs.pair_configs(n, 17 + n, 5.0, 9.4)
    out, g = m.pairs(torch.from_numpy(cfg8(cfg7)).cuda(), "fp32", grad=True)
    torch.cuda.synchronize()
    out = out.double().cpu().numpy()
    E, Fj, ti, tj = oracle_labels(flat, width, cfg7)
    assert_parity(out[:, 0:3], Fj, TOL_F32)
    assert_parity(out[:, 4:7], ti, TOL_F32)
    assert_parity(out[:, 8:11], tj, TOL_F32)
    assert np.abs(out[:, 3] - E).max() < TOL_F32 * max(1.0, np.abs(E).max())
    # gradient of E with respect to the raw inputs (s, q_rel)
    sq = torch.as_tensor(cfg7.astype(np.float64)).requires_grad_(True)
    p = nn.unpack(flat.astype(np.float64), width)
    Eo = nn.config_energy(p, sq[:, :3], sq[:, 3:])
    (gref,) = torch.autograd.grad(Eo.sum(), [sq])
    g = g.double().cpu().numpy()
    assert_parity(g[:, 0:3], gref[:, :3].numpy(), TOL_F32)
    assert_parity(g[:, 4:8], gref[:, 3:].numpy(), TOL_F32)


def test_nn_pairs_empty_and_depths():
    import torch

    from paper_2402_12199_gb300 import api

    m = api.MLP(128, 3)
    m.set_params(params(128, 1))
    out = m.pairs(torch.zeros((0, 8), device="cuda"))
    assert out.shape == (0, 12)
    # depth 4 at widths 128 and 256 takes the kernel's smaller weight chunks
    for width, depth in ((64, 1), (64, 2), (64, 4), (128, 1), (128, 4), (256, 4)):
        flat = params(width, depth, depth)
        m = api.MLP(width, depth)
        m.set_params(flat)
        cfg7 = inputs.pair_configs(300, depth, 5.0, 9.4)
        out = m.pairs(torch.from_numpy(cfg8(cfg7)).cuda()).double().cpu().numpy()
        E, Fj, ti, tj = oracle_labels(flat, width, cfg7, depth)
        assert_parity(out[:, 0:3], Fj, TOL_F32)
        assert_parity(out[:, 4:7], ti, TOL_F32)
        assert_parity(out[:, 8:11], tj, TOL_F32)
        assert_parity(out[:, 3], E, TOL_F32)


def test_nn_system_forces_parity_64_cubes():
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(64, 0.10, 1)
    flat = params(128, 2)
    m = api.MLP(128, 3)
    m.set_params(flat)
    s = gpu_system(st, L)
    r = s.forces_nn(m, "fp32", energy=True)
    s.sync()
    F, T, E, per, pairs = oracle_nn(st, L, tmpl, flat, 128)
    assert canonical_margin(st, pairs) > 1e-4
    assert_parity(r["force"][:, :3].double().cpu().numpy(), F, TOL_F32)
    assert_parity(r["torque"][:, :3].double().cpu().numpy(), T, TOL_F32)
    assert abs(r["energy"] - E) < TOL_F32 * np.abs(per).sum()


def test_nn_md_steps_conserve_energy():
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(512, 0.2, 6)
    m = api.MLP(128, 3)
    m.set_params(params(128, 3))
    s = gpu_system(st, L)
    s.forces_nn(m, "fp32")
    e0 = sum(s.energy())
    s.step(50, 0.002, path=api.RB_PATH_NN, mlp=m)
    e1 = sum(s.energy())
    assert abs(e1 - e0) < 1e-3 * 512, (e0, e1)


def test_bead_fallback_for_close_pairs():
    """Pairs closer than rho_min take the bead sum inside the network path:
    rho_min above the cutoff reproduces the bead path exactly; in between, the
    result is the oracle's bead sum on close pairs plus its network on the rest."""
    import oracle
    from oracle import bodies
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(1500, 0.2, 61)
    flat = params(128, 8)
    m = api.MLP(128, 3)
    m.set_params(flat)
    s = gpu_system(st, L)
    ref = s.forces_beads()
    s.set_nn_fallback(100.0)
    r = s.forces_nn(m, "fp32")
    s.sync()
    assert bool((r["force"] == ref["force"]).all()) and bool((r["torque"] == ref["torque"]).all())
    rho_min = 8.2
    s.set_nn_fallback(rho_min)
    r = s.forces_nn(m, "fp32")
    n_fb = s.nn_fallback_count()
    pos = st["pos"][:, :3].astype(np.float64)
    pairs = oracle.pairs_bruteforce(pos, [L] * 3, bodies.pair_cutoff(tmpl))
    d = pos[pairs[:, 1]] - pos[pairs[:, 0]]
    d -= L * np.rint(d / L)
    close = np.linalg.norm(d, axis=1) < rho_min
    assert n_fb == int(close.sum()) and 0 < n_fb < len(pairs)
    Fb, Tb, _, _ = oracle.forces_beads(pos, st["quat"], [L] * 3, tmpl, pairs[close])
    Fn, Tn, _, _, _ = oracle_nn(st, L, tmpl, flat, 128, pairs=pairs[~close])
    assert_parity(r["force"][:, :3].double().cpu().numpy(), Fb + Fn, TOL_F32)
    assert_parity(r["torque"][:, :3].double().cpu().numpy(), Tb + Tn, TOL_F32)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_parameter_change_on_the_network_stream_reaches_the_system(precision):
    """A network's parameters (and its kernel images) are written on the
    network's own stream; a system on another stream that evaluates right after
    the change must see the new values.  The network's stream is held busy by a
    bounded spin before each device-to-device parameter copy, so a system that
    did not wait for it would read the previous parameters."""
    import torch

    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(512, 0.2, 6)
    sets = [torch.from_numpy(params(128, seed)).cuda() for seed in (11, 12)]
    s = gpu_system(st, L)
    ref = []
    for flat in sets:  # each set on a fresh network on the system's own stream
        m0 = api.MLP(128, 3)
        m0.set_params(flat)
        r = s.forces_nn(m0, precision)
        s.sync()
        ref.append((r["force"].clone(), r["torque"].clone()))
    assert not torch.equal(ref[0][0], ref[1][0])
    ns = torch.cuda.Stream()
    m = api.MLP(128, 3, stream=ns)
    for k in range(4):
        with torch.cuda.stream(ns):
            torch.cuda._sleep(2_000_000)  # about 1 ms of the network's stream
        m.set_params(sets[k % 2])
        r = s.forces_nn(m, precision)
        s.sync()
        assert torch.equal(r["force"], ref[k % 2][0]), k
        assert torch.equal(r["torque"], ref[k % 2][1]), k
